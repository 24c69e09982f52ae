// lfd_superpixel_stats_noalloc: the superpixel statistics of one view (the
// per-label counts, centroids, mean colours and minimum neighbour colour
// similarity that lfd_set_input builds) computed without allocating any
// memory.
//
// Some callers cannot allocate device memory on the path where they need
// these statistics: code running inside a CUDA graph being captured (stream
// capture forbids cudaMalloc/cudaFree), real-time or embedded loops that have
// a fixed memory plan and may not touch the allocator once started, and hosts
// whose allocator is owned by another framework.  This entry point therefore
// takes only caller-provided inputs and outputs; its scratch (per-label pixel
// counts and bounding boxes) lives in a file-scope device array of a fixed
// size that exists for as long as the library is loaded.
//
// Limits and sharing rules:
//  - at most LFD_NOALLOC_MAX_LABELS (65536) labels per call (grid_w*grid_h);
//  - the scratch array is shared by every call on a device and keeps the last
//    call's contents; each call clears the part it uses first;
//  - calls whose GPU work overlaps (different streams, or different host
//    threads without ordering) race on the scratch array and give wrong
//    results: serialise them;
//  - the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before any stream capture.
#include <mutex>

#include "lfd_internal.cuh"

namespace {

constexpr int NOALLOC_MAX_LABELS = LFD_NOALLOC_MAX_LABELS;
constexpr int NOALLOC_MAX_DEVICES = 64;

struct NoallocScratch {
    int cnt[NOALLOC_MAX_LABELS];
    int4 bbox[NOALLOC_MAX_LABELS];
};

// 1.25 MiB per device, held while the library is loaded
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

std::mutex g_noalloc_mutex;
NoallocScratch *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

__global__ void k_na_clear(NoallocScratch *sc, int S)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S) {
        sc->cnt[i] = 0;
        sc->bbox[i] = make_int4(0x7fffffff, 0x7fffffff, -1, -1);
    }
}

__global__ void __launch_bounds__(256) k_na_count(NoallocScratch *sc, const int *labels, int W, int H, int S)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = p < W * H;
    const int l = in ? __ldg(labels + p) : -1;
    const bool ok = in && l >= 0 && l < S;                   // labels outside the grid are ignored
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (!ok) return;
    const int x = p % W, y = p / W;
    const unsigned grp = __match_any_sync(act, l);
    const int n = __popc(grp);
    const int mnx = (int)__reduce_min_sync(grp, (unsigned)x), mxx = (int)__reduce_max_sync(grp, (unsigned)x);
    const int mny = (int)__reduce_min_sync(grp, (unsigned)y), mxy = (int)__reduce_max_sync(grp, (unsigned)y);
    if ((threadIdx.x & 31) == __ffs(grp) - 1) {
        atomicAdd(&sc->cnt[l], n);
        atomicMin(&sc->bbox[l].x, mnx);
        atomicMin(&sc->bbox[l].y, mny);
        atomicMax(&sc->bbox[l].z, mxx);
        atomicMax(&sc->bbox[l].w, mxy);
    }
}

__device__ __forceinline__ void na_texel(int fmt, const char *row, int x, double &r, double &g, double &b)
{
    if (fmt == LFD_RGBA8) {
        const uchar4 t = ((const uchar4 *)row)[x];
        r = t.x; g = t.y; b = t.z;
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
__device__ __forceinline__ T na_sum256(T v, T *sh)
{
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

// one block per label: sums over the label's bounding box in a fixed order
__global__ void __launch_bounds__(256) k_na_stats(const NoallocScratch *sc, const int *labels, const void *img,
                                                  long long pitch, int fmt, int W, float *stats)
{
    const int s = blockIdx.x;
    const int n = sc->cnt[s];
    __shared__ double shd[256];
    __shared__ long long shl[256];
    float *out = stats + 8 * (long long)s;
    if (n == 0) {   // as the regular path: centroid and colour 0, minw filled in by k_na_minw
        if (threadIdx.x < 8) out[threadIdx.x] = threadIdx.x == 5 ? 1.f : 0.f;
        return;
    }
    const int4 bb = sc->bbox[s];
    const int bw = bb.z - bb.x + 1;
    const long long area = (long long)bw * (bb.w - bb.y + 1);
    long long sx = 0, sy = 0;
    double sr = 0, sg = 0, sb = 0;
    for (long long i = threadIdx.x; i < area; i += 256) {
        const int x = bb.x + (int)(i % bw), y = bb.y + (int)(i / bw);
        if (__ldg(labels + (long long)y * W + x) != s) continue;
        sx += x;
        sy += y;
        double r, g, b;
        na_texel(fmt, (const char *)img + (long long)y * pitch, x, r, g, b);
        sr += r; sg += g; sb += b;
    }
    const long long tx = na_sum256<long long>(sx, shl), ty = na_sum256<long long>(sy, shl);
    const double tr = na_sum256<double>(sr, shd), tg = na_sum256<double>(sg, shd), tb = na_sum256<double>(sb, shd);
    if (threadIdx.x == 0) {
        const double sc_ = fmt == LFD_RGBA8 ? 1.0 / 255.0 : 1.0;
        out[0] = (float)((double)tx / n);
        out[1] = (float)((double)ty / n);
        out[2] = (float)(tr * sc_ / n);
        out[3] = (float)(tg * sc_ / n);
        out[4] = (float)(tb * sc_ / n);
        out[5] = 1.f;
        out[6] = (float)n;
        out[7] = 0.f;
    }
}

// minimum colour similarity to the present (non-empty) 8-neighbours, from the
// colours just written; an empty label gets the value the regular path gives
// it (its colour is 0), so both report the same slot 5 for every label
__global__ void k_na_minw(float *stats, int GW, int GH, double k_col)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= GW * GH) return;
    const float *me = stats + 8 * (long long)s;
    const int gx = s % GW, gy = s / GW;
    const int dxs[8] = {1, 1, 0, -1, -1, -1, 0, 1}, dys[8] = {0, -1, -1, -1, 0, 1, 1, 1};
    double best = 1.0;
    bool any = false;
    for (int d = 0; d < 8; d++) {
        const int x = gx + dxs[d], y = gy + dys[d];
        if (x < 0 || y < 0 || x >= GW || y >= GH) continue;
        const float *nb = stats + 8 * (long long)(y * GW + x);
        if (nb[6] == 0.f) continue;
        const double dr = (double)nb[2] - me[2], dg = (double)nb[3] - me[3], db = (double)nb[4] - me[4];
        const double om = exp2(-(dr * dr + dg * dg + db * db) * k_col);
        if (!any || om < best) best = om;
        any = true;
    }
    // written into a separate slot first would need a second buffer; the
    // neighbours read only colours and counts (slots 2..4, 6), never slot 5
    stats[8 * (long long)s + 5] = (float)(any ? best : 1.0);
}

}  // namespace

extern "C" lfd_status lfd_superpixel_stats_noalloc(const int32_t *labels, const void *image, int32_t width,
                                                   int32_t height, int64_t pitch_bytes, int32_t fmt, int32_t grid_w,
                                                   int32_t grid_h, double alpha, float *stats_out, void *stream)
{
    int texel = fmt == LFD_RGBA8 ? 4 : (fmt == LFD_RGBA_F16 || fmt == LFD_RGBA_BF16) ? 8 : fmt == LFD_RGBA_F32 ? 16 : 0;
    if (!labels || !image || !stats_out || texel == 0) return LFD_ERR_INVALID_ARG;
    if (width < 1 || height < 1 || width > LFD_MAX_DIM || height > LFD_MAX_DIM || grid_w < 1 || grid_h < 1)
        return LFD_ERR_INVALID_ARG;
    if ((long long)grid_w * grid_h > NOALLOC_MAX_LABELS) return LFD_ERR_INVALID_ARG;   // beyond the scratch size
    const long long pitch = pitch_bytes ? pitch_bytes : (long long)width * texel;
    if (pitch < (long long)width * texel || pitch % texel || !(alpha > 0)) return LFD_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return LFD_ERR_CUDA;
    }
    NoallocScratch *sc = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return LFD_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = (NoallocScratch *)p;
        }
        sc = g_noalloc_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int S = grid_w * grid_h;
    const int npx = width * height;
    // An error left pending on this thread by earlier, unrelated work is not
    // this call's: a launch of this call has failed only when the pending
    // error changes from what it was on entry.  (The earlier error stays
    // pending for its owner.)
    const cudaError_t before = cudaPeekAtLastError();
    auto launch_failed = [before]() {
        const cudaError_t e = cudaPeekAtLastError();
        return e != cudaSuccess && e != before;
    };
    const double log2e = 1.4426950408889634;
    k_na_clear<<<(S + 255) / 256, 256, 0, st>>>(sc, S);
    if (!launch_failed()) k_na_count<<<(npx + 255) / 256, 256, 0, st>>>(sc, labels, width, height, S);
    if (!launch_failed()) k_na_stats<<<S, 256, 0, st>>>(sc, labels, image, pitch, fmt, width, stats_out);
    if (!launch_failed())
        k_na_minw<<<(S + 127) / 128, 128, 0, st>>>(stats_out, grid_w, grid_h, log2e / (2.0 * alpha * alpha));
    if (launch_failed()) {
        if (before == cudaSuccess) cudaGetLastError();   // clear only what this call raised
        return LFD_ERR_CUDA;
    }
    return LFD_OK;
}
