// Step a1: superpixel pixel lists (CSR) and statistics, and the per-view
// bilinear sampling textures.
//
// Section III-A: each view is over-segmented into compact superpixels laid out
// as a regular grid with an 8-neighbour system; each superpixel's plane is
// anchored at its centroid and its colour is the mean colour of its pixels
// (Section III-C1).  Eq. 11 needs the minimum colour similarity to the
// neighbours, which is fixed per superpixel and computed here once.
//
// The pixel lists are built without sorting and without atomics on the list
// itself: one block per superpixel scans the superpixel's bounding box in
// row-major order and compacts the matching pixels with a block prefix sum,
// so the list order (row-major) and every sum are deterministic.  The cost is
// the sum of bounding-box areas, about the image area for compact superpixels.
#include "lfd_internal.cuh"

namespace lfd {

// ---------------------------------------------------------------------------
// 1. counts and bounding boxes (warp-aggregated atomics)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_sp_count(Workspace w, int *cnt, int4 *bbox)
{
    const int v = blockIdx.y;
    const ViewDev &vd = w.views[v];
    const int npx = vd.W * vd.H;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = p < npx;
    int l = in ? __ldg(vd.labels + p) : -1;
    const bool ok = in && l >= 0 && l < vd.S;
    if (in && !ok) {
        if (atomicOr(&w.ctr->status, DEV_ERR_LABEL) == 0) {
            w.ctr->bad_view = v;
            w.ctr->bad_index = p;
        }
    }
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (!ok) return;
    const int x = p % vd.W, y = p / vd.W;
    const unsigned grp = __match_any_sync(act, l);
    const int n = __popc(grp);
    const int mnx = (int)__reduce_min_sync(grp, (unsigned)x);
    const int mxx = (int)__reduce_max_sync(grp, (unsigned)x);
    const int mny = (int)__reduce_min_sync(grp, (unsigned)y);
    const int mxy = (int)__reduce_max_sync(grp, (unsigned)y);
    if ((threadIdx.x & 31) == __ffs(grp) - 1) {
        const int gs = vd.sp_base + l;
        atomicAdd(&cnt[gs], n);
        atomicMin(&bbox[gs].x, mnx);
        atomicMin(&bbox[gs].y, mny);
        atomicMax(&bbox[gs].z, mxx);
        atomicMax(&bbox[gs].w, mxy);
    }
}

__global__ void k_sp_bbox_init(int S_total, int *cnt, int4 *bbox)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S_total) {
        cnt[i] = 0;
        bbox[i] = make_int4(0x7fffffff, 0x7fffffff, -1, -1);
    }
}

cudaError_t launch_sp_count(const Workspace &w, int V, int max_px, int *cnt, int4 *bbox, cudaStream_t st)
{
    k_sp_bbox_init<<<(w.S_total + 255) / 256, 256, 0, st>>>(w.S_total, cnt, bbox);
    dim3 grid((max_px + 255) / 256, V);
    k_sp_count<<<grid, 256, 0, st>>>(w, cnt, bbox);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 2. exclusive scan of the counts of each view -> global list offsets
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(1024) k_sp_scan(Workspace w, int V, const int *cnt, int *off)
{
    const int v = blockIdx.x;
    const ViewDev &vd = w.views[v];
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = (int)vd.px_base;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < vd.S; base += 1024) {
        const int s = base + threadIdx.x;
        const int c = s < vd.S ? cnt[vd.sp_base + s] : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int t = warp_tot[lane];
            int ti = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, ti, o);
                if (lane >= o) ti += u;
            }
            warp_tot[lane] = ti - t;   // exclusive prefix of warp totals
        }
        __syncthreads();
        const int excl = carry + warp_tot[wid] + incl - c;
        if (s < vd.S) off[vd.sp_base + s] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + c;
        __syncthreads();
    }
    if (v == V - 1 && threadIdx.x == 0) off[w.S_total] = carry;
}

cudaError_t launch_sp_scan(const Workspace &w, int V, const int *cnt, int *off, cudaStream_t st)
{
    k_sp_scan<<<V, 1024, 0, st>>>(w, V, cnt, off);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 3. ordered compaction of each superpixel's pixels + centroid and colour sums
// ---------------------------------------------------------------------------

struct ColourSum {
    double r, g, b;
};

__device__ __forceinline__ void texel_rgb(int fmt, const void *img, long long pitch, int x, int y, double &r,
                                          double &g, double &b)
{
    const char *row = (const char *)img + (long long)y * pitch;
    if (fmt == LFD_RGBA8) {
        const uchar4 t = ((const uchar4 *)row)[x];
        r = t.x; g = t.y; b = t.z;                       // summed as integers, scaled once at the end
    } else if (fmt == LFD_RGBA_F16) {
        const __half *t = (const __half *)row + 4 * x;
        r = __half2float(t[0]); g = __half2float(t[1]); b = __half2float(t[2]);
    } else if (fmt == LFD_RGBA_BF16) {
        const __nv_bfloat16 *t = (const __nv_bfloat16 *)row + 4 * x;
        r = __bfloat162float(t[0]); g = __bfloat162float(t[1]); b = __bfloat162float(t[2]);
    } else {
        const float4 t = ((const float4 *)row)[x];
        r = t.x; g = t.y; b = t.z;
    }
}

template <typename T>
__device__ __forceinline__ T block_sum256(T v, T *sh)
{
    // fixed tree over 256 threads: deterministic
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + o];
        __syncthreads();
    }
    T r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(256) k_sp_collect(Workspace w, Consts c, const int4 *bbox, const int *cnt,
                                                    unsigned *pix, double2 *cen, int2 *ref, float4 *col)
{
    const int gs = blockIdx.x;
    const int v = w.sp_view[gs];
    const ViewDev &vd = w.views[v];
    const int s = gs - vd.sp_base;
    const int n = cnt[gs];
    __shared__ int warp_cnt[8];
    __shared__ double shd[256];
    __shared__ long long shl[256];
    if (n == 0) {
        if (threadIdx.x == 0) {
            cen[gs] = make_double2(0.0, 0.0);
            ref[gs] = make_int2(0, 0);
            col[gs] = make_float4(0.f, 0.f, 0.f, 1.f);
        }
        return;
    }
    const int4 bb = bbox[gs];
    const int bw = bb.z - bb.x + 1, bh = bb.w - bb.y + 1;
    const long long area = (long long)bw * bh;
    const int base_off = w.sp_off[gs];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long sx = 0, sy = 0;
    double sr = 0, sg = 0, sb = 0;
    int written = 0;
    for (long long b0 = 0; b0 < area; b0 += 256) {
        const long long i = b0 + threadIdx.x;
        int x = 0, y = 0;
        bool f = false;
        if (i < area) {
            x = bb.x + (int)(i % bw);
            y = bb.y + (int)(i / bw);
            f = __ldg(vd.labels + (long long)y * vd.W + x) == s;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_cnt[wid] = __popc(bal);
        __syncthreads();
        int before = 0, tot = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int cw = warp_cnt[k];
            before += k < wid ? cw : 0;
            tot += cw;
        }
        if (f) {
            const int rank = before + __popc(bal & ((1u << lane) - 1u));
            if (written + rank < n) pix[base_off + written + rank] = ((unsigned)y << 16) | (unsigned)x;
            sx += x;
            sy += y;
            double r, g, b;
            texel_rgb(c.fmt, vd.img, vd.pitch, x, y, r, g, b);
            sr += r; sg += g; sb += b;
        }
        written += tot;
        __syncthreads();
    }
    const long long tx = block_sum256<long long>(sx, shl);
    const long long ty = block_sum256<long long>(sy, shl);
    const double tr = block_sum256<double>(sr, shd);
    const double tg = block_sum256<double>(sg, shd);
    const double tb = block_sum256<double>(sb, shd);
    if (threadIdx.x == 0) {
        if (written != n) {
            if (atomicOr(&w.ctr->status, DEV_ERR_COUNT) == 0) {
                w.ctr->bad_view = v;
                w.ctr->bad_index = s;
            }
        }
        const double cx = (double)tx / n, cy = (double)ty / n;
        cen[gs] = make_double2(cx, cy);
        ref[gs] = make_int2(__double2int_rn(cx), __double2int_rn(cy));
        const double sc = (c.fmt == LFD_RGBA8) ? 1.0 / 255.0 : 1.0;
        col[gs] = make_float4((float)(tr * sc / n), (float)(tg * sc / n), (float)(tb * sc / n), 1.0f);
    }
}

cudaError_t launch_sp_collect(const Workspace &w, const Consts &c, const int4 *bbox, const int *cnt, unsigned *pix,
                              double2 *cen, int2 *ref, float4 *col, cudaStream_t st)
{
    k_sp_collect<<<w.S_total, 256, 0, st>>>(w, c, bbox, cnt, pix, cen, ref, col);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 4. minimum colour similarity to the present 8-neighbours (Eq. 11)
// ---------------------------------------------------------------------------

__global__ void k_sp_minw(Workspace w, Consts c, float4 *col)
{
    const int gs = blockIdx.x * blockDim.x + threadIdx.x;
    if (gs >= w.S_total) return;
    const int v = w.sp_view[gs];
    const ViewDev &vd = w.views[v];
    const int s = gs - vd.sp_base;
    const int gx = s % vd.GW, gy = s / vd.GW;
    const float4 cs = col[gs];
    const double k_col = vd.k_col;   // log2(e) / (2 alpha^2): omega = 2^(-|dC|^2 k_col)
    double best = 1.0;
    bool any = false;
    for (int d = 0; d < 8; d++) {
        int dx, dy;
        ring_dir(d, dx, dy);
        const int x = gx + dx, y = gy + dy;
        if (x < 0 || y < 0 || x >= vd.GW || y >= vd.GH) continue;
        const int j = vd.sp_base + y * vd.GW + x;
        if (w.sp_cnt[j] == 0) continue;
        const float4 cj = col[j];
        const double dr = (double)cj.x - cs.x, dg = (double)cj.y - cs.y, db = (double)cj.z - cs.z;
        const double om = exp2(-(dr * dr + dg * dg + db * db) * k_col);
        if (!any || om < best) best = om;
        any = true;
    }
    col[gs].w = (float)(any ? best : 1.0);
}

cudaError_t launch_sp_minw(const Workspace &w, const Consts &c, float4 *col, cudaStream_t st)
{
    k_sp_minw<<<(w.S_total + 127) / 128, 128, 0, st>>>(w, c, col);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 5. sampling textures: per pixel the 2x2 bilinear footprint in one record
// ---------------------------------------------------------------------------
//   RGBA8, F16, BF16: red/green of t00, t10, t01, t11 as     24 B / pixel
//          four 16-bit pairs (16-B records for all entries), then
//          blue of (t00, t01), (t10, t11) as two pairs (8-B records);
//          RGBA8 bytes are stored as exact halves
//   F32: 3 x float4 RGB of t00, t10, t01, t11                48 B / pixel
//   (W + 1) x (H + 1) entries per view, see k_quads

__device__ __forceinline__ unsigned pack_h2(float lo, float hi)
{
    __half2 h = __floats2half2_rn(lo, hi);   // small integers: exact
    return *reinterpret_cast<unsigned *>(&h);
}

// The texture has a border of one quad on the left and top: entry
// (y + 1) (W + 1) + (x + 1) holds the quad of pixel (x, y) for x in [-1, W-1],
// y in [-1, H-1], every texel index clamped to the image.  A bilinear sample
// anywhere in the texture area -1/2 <= x < W - 1/2 then reads the quad at
// floor(x) with no clamping of the coordinates: where a texel is clamped its
// difference to the neighbour is 0, which gives clamp-to-edge exactly.
__global__ void __launch_bounds__(256) k_quads(Workspace w, int fmt)
{
    const int v = blockIdx.y;
    const ViewDev &vd = w.views[v];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int Wp = vd.W + 1;
    if (p >= Wp * (vd.H + 1)) return;
    const int qx = p % Wp - 1, qy = p / Wp - 1;
    const int x = max(qx, 0), y = max(qy, 0);
    const int x1 = min(qx + 1, vd.W - 1), y1 = min(qy + 1, vd.H - 1);
    const char *base = (const char *)vd.img;
    const long long pitch = vd.pitch;
    const char *r0 = base + (long long)y * pitch;
    const char *r1 = base + (long long)y1 * pitch;
    if (fmt == LFD_RGBA8) {
        // the byte texels as halves (0..255 exact) in the FP16 layout below
        const uchar4 *a = (const uchar4 *)r0, *b = (const uchar4 *)r1;
        const uchar4 t00 = a[x], t10 = a[x1], t01 = b[x], t11 = b[x1];
        const long long npx = (long long)Wp * (vd.H + 1);
        ((uint4 *)vd.quad)[p] = make_uint4(pack_h2(t00.x, t00.y), pack_h2(t10.x, t10.y), pack_h2(t01.x, t01.y),
                                           pack_h2(t11.x, t11.y));
        ((uint2 *)((uint4 *)vd.quad + npx))[p] = make_uint2(pack_h2(t00.z, t01.z), pack_h2(t10.z, t11.z));
    } else if (fmt == LFD_RGBA_F16 || fmt == LFD_RGBA_BF16) {
        // a texel is {red|green, blue|alpha} as two 16-bit pairs
        const uint2 *a = (const uint2 *)r0, *b = (const uint2 *)r1;
        const uint2 t00 = a[x], t10 = a[x1], t01 = b[x], t11 = b[x1];
        const long long npx = (long long)Wp * (vd.H + 1);
        ((uint4 *)vd.quad)[p] = make_uint4(t00.x, t10.x, t01.x, t11.x);
        ((uint2 *)((uint4 *)vd.quad + npx))[p] =
            make_uint2((t00.y & 0xffffu) | (t01.y << 16), (t10.y & 0xffffu) | (t11.y << 16));
    } else {
        const float4 *a = (const float4 *)r0, *b = (const float4 *)r1;
        const float4 t00 = a[x], t10 = a[x1], t01 = b[x], t11 = b[x1];
        float4 *q = (float4 *)vd.quad + 3 * (long long)p;
        q[0] = make_float4(t00.x, t00.y, t00.z, t10.x);
        q[1] = make_float4(t10.y, t10.z, t01.x, t01.y);
        q[2] = make_float4(t01.z, t11.x, t11.y, t11.z);
    }
}

cudaError_t launch_quads(const Workspace &w, int V, int max_px, int fmt, cudaStream_t st)
{
    dim3 grid((max_px + 255) / 256, V);       // max_px: largest (W + 1) (H + 1) of the views
    k_quads<<<grid, 256, 0, st>>>(w, fmt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 6. work orders of the persistent launches: a stable counting sort of all
//    superpixels by size class, largest first, index order inside a class.
//    Propagation (mode 0) uses pixel-slot classes ceil(n/32), capped at 16:
//    superpixels of one class run the same compiled evaluation, so the warps
//    resident on an SM at any time execute one code body (measured on the
//    8-view 1024x768 case: 23.3 ms per frame in this order, 47 ms with the
//    classes sorted per view, 53 ms in plain index order, from
//    instruction-fetch stalls).  The sweep (mode 1) has one code body and
//    uses coarser power-of-two classes floor(log2 n): expensive superpixels
//    still go first, while superpixels of similar size keep index order, so
//    concurrently swept superpixels are neighbours and share L2 lines (slot
//    classes there interleaved 14- and 15-pixel grid cells across all views
//    and read 6x more DRAM).  Deterministic.
// ---------------------------------------------------------------------------

//    Inside a class the superpixels go by row band (up to ORDER_BANDS
//    bands of each view's grid rows, a launch-shape option) and then in
//    index order: the superpixels in flight at any time cover the same rows
//    of every view, so the rows of the sampling textures and rasterised maps
//    they gather from (their own band, shifted by the disparity, in each
//    neighbour view) stay in L2 together instead of spanning whole views.
//    The sweep's order is finally partitioned, stably, by sweep class (mode
//    2: the label-count class of each superpixel's light field and the pair
//    form of its view): one sweep launch per class, its CTAs as wide as the
//    class's label count, compiled for the class's pair form.

__device__ __forceinline__ int order_key(const Workspace &w, int gs, int mode, int bands)
{
    if (mode == 2) return w.views[__ldg(w.sp_view + gs)].sclass;
    const int n = __ldg(w.sp_cnt + gs);
    const int cls = mode == 0 ? (n + 31) >> 5 : 31 - __clz(max(n, 1));
    const ViewDev &vd = w.views[__ldg(w.sp_view + gs)];
    const int gy = (gs - vd.sp_base) / vd.GW;
    const int band = min(bands - 1, (int)(((long long)gy * bands) / vd.GH));
    return (ORDER_CLASSES - 1 - min(cls, ORDER_CLASSES - 1)) * ORDER_BANDS + band;   // 0 = largest class, top band
}

__global__ void k_order_hist(Workspace w, int *hist, int mode, int bands, const int *in)
{
    __shared__ int h[ORDER_KEYS];
    for (int k = threadIdx.x; k < ORDER_KEYS; k += blockDim.x) h[k] = 0;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < w.S_total) atomicAdd(&h[order_key(w, in ? __ldg(in + i) : i, mode, bands)], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < ORDER_KEYS; k += blockDim.x)
        if (h[k]) atomicAdd(&hist[k], h[k]);
}

// one CTA of 1024 threads walks the superpixels in tiles of 1024; a
// superpixel's slot is its key's start + the count of equal keys before it
__global__ void __launch_bounds__(1024) k_order_scatter(Workspace w, const int *hist, int *order, int mode, int bands,
                                                        const int *in)
{
    __shared__ int run[ORDER_KEYS];                  // running position per key
    __shared__ int wcnt[32][ORDER_KEYS];             // per-warp counts of the tile
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0) {
        int acc = 0;
        for (int k = 0; k < ORDER_KEYS; k++) {
            run[k] = acc;
            acc += hist[k];
        }
    }
    for (int base = 0; base < w.S_total; base += 1024) {
        for (int i = t; i < 32 * ORDER_KEYS; i += 1024) wcnt[i / ORDER_KEYS][i % ORDER_KEYS] = 0;
        __syncthreads();
        const int pos = base + t;
        const bool ok = pos < w.S_total;
        const int gs = ok ? (in ? __ldg(in + pos) : pos) : 0;
        const int key = ok ? order_key(w, gs, mode, bands) : ORDER_KEYS;   // out-of-range lanes: a key of their own
        const unsigned same = __match_any_sync(0xffffffffu, key);
        const int rank = __popc(same & ((1u << lane) - 1u));
        if (ok && rank == 0) wcnt[wid][key] = __popc(same);
        __syncthreads();
        if (ok) {
            int before = 0;
            for (int u = 0; u < wid; u++) before += wcnt[u][key];
            order[run[key] + before + rank] = gs;
        }
        __syncthreads();
        if (t < ORDER_KEYS) {
            int tot = 0;
            for (int u = 0; u < 32; u++) tot += wcnt[u][t];
            run[t] += tot;
        }
        __syncthreads();
    }
}

cudaError_t launch_sp_order(const Workspace &w, int *order, int *hist, int mode, int bands, const int *in,
                            cudaStream_t st)
{
    bands = max(1, min(bands, ORDER_BANDS));
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * ORDER_KEYS, st);
    if (e != cudaSuccess) return e;
    const int blocks = (w.S_total + 255) / 256;
    k_order_hist<<<blocks, 256, 0, st>>>(w, hist, mode, bands, in);
    k_order_scatter<<<1, 1024, 0, st>>>(w, hist, order, mode, bands, in);
    return cudaGetLastError();
}

}  // namespace lfd
