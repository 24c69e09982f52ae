// Steps a2-a4: partly randomised fronto-parallel plane sweep (Section III-B).
//
// For superpixel Omega of view v and label k the plane is fronto-parallel at
// inverse depth z_k = 1/d_max + (k + u_k) * delta with u_k uniform in [0,1)
// per superpixel and label (the jitter of Section III-B).  Its cost is
// Eq. 2's double sum over the neighbour views N(v) and the superpixel's
// pixels of the truncated SSD of Eq. 1, sampled bilinearly through the
// plane-induced homography; the lowest cost wins.
//
// Mapping: one CTA per superpixel, one thread per label.  The superpixel's
// pixels are staged in shared memory and read as broadcasts, so every thread
// walks the same pixel list while its own label shifts the projection along
// the epipolar line; neighbouring labels therefore gather from neighbouring
// texels (coalesced, L1-resident).  No reduction is needed per sample: each
// thread owns its label's cost; a single block arg-min ends the CTA.
//
// Homography per (label, view): for the plane g = z_k * gh (gh = (0,0,1) for
// camera-frame sweeps) A = P + q g^T; its superpixel-anchored third column
// (P + q g^T) (ref,1) is composed in FP64 and rounded to FP32.  In the camera
// frame the rest, P (du, dv, 0) on the pixel's offset from the anchor, does not
// depend on the label: it is computed once per pixel and view of a chunk into
// shared memory and each sample adds the label's column (3 FP32 adds).  In the
// world frame the label also scales the pixel terms: 6 FP32 FMAs per sample.
#include "lfd_sample.cuh"

namespace lfd {

constexpr int SWEEP_CHUNK = 128;

// Pair forms of the homography of a (view, neighbour view) pair, the kernels'
// template argument PF:
//   PF_GENERAL  any pair;
//   PF_AFFINE   P row 3 = (0, 0, P22) and q_z = 0 (parallel optical axes at
//               equal depth): the sample's homogeneous coordinate is the same
//               for every pixel of a label;
//   PF_SHIFT    affine with P's upper 2 x 2 block = P22 I as well (rectified
//               parallel cameras with equal intrinsics, e.g. a planar array):
//               a fronto-parallel plane moves every pixel by the same vector
//               (X0, Y0), so the integer part and the bilinear fractions are
//               per label and view, and a sample is an integer offset, a
//               window test on it and the gather.
constexpr int PF_GENERAL = 0, PF_AFFINE = 1, PF_SHIFT = 2;

struct SweepPair {
    float a00, a01, a10, a11, a20, a21;   // FP32 columns 0,1 of P (camera frame: not label dependent)
    int Wi, Hi;
    double pref[3];                       // P (ref,1) in FP64
    double q[3];
    double p0[3], p1[3];                  // columns 0,1 of P in FP64 (world-frame sweeps)
    double icw;                           // 1 / P (ref,1)_z (translation pairs: every label's w)
    const void *tex;
};

template <int THREADS, bool WORLD>
struct SweepShared {
    float2 d[SWEEP_CHUNK];
    float4 ref[SWEEP_CHUNK];
    // camera-frame sweeps: the label-independent part of each pixel's projection into
    // each neighbour view, P (du, dv, 0) (the label adds q z_k at the anchor)
    float4 xyw[WORLD ? 1 : LFD_MAXN][SWEEP_CHUNK];
    SweepPair pair[LFD_MAXN];
    double gh[4];                         // gh and gh.(ref,1)
    float n[3];                           // sweep plane normal (camera frame)
    float bc[THREADS / 32];
    int bk[THREADS / 32];
    int item;
};

// the whole sweep of superpixel gs by one CTA (threads = labels)
template <int FMT, bool WORLD, int THREADS, int PF>
__device__ __forceinline__ void sweep_sp(const Workspace &w, const Consts &c, int gs, SweepShared<THREADS, WORLD> &sh,
                                         float4 *planes, int *label_out, float *cost_out)
{
    const int v = __ldg(w.sp_view + gs);
    const ViewDev &vd = w.views[v];
    if (vd.sweep_skip) return;               // warm-started view: its planes are given
    const int s = gs - vd.sp_base;
    const int n = __ldg(w.sp_cnt + gs);
    if (n == 0) {
        if (threadIdx.x == 0) {
            planes[gs] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (label_out) label_out[gs] = -1;
        }
        return;
    }
    const int2 ref = __ldg(w.sp_ref + gs);
    const int nnb = vd.nnb;
    const int off = __ldg(w.sp_off + gs);
    const void *own_tex = vd.quad;
    const int L = vd.L;

    if (threadIdx.x == 0) {
        // sweep plane normal: fronto-parallel to the camera (gh = (0,0,1)) or to the
        // world z axis; gh = K^-T n / (n . K^-1 (c,1)) so that g = z * gh
        double gh0 = 0.0, gh1 = 0.0, gh2 = 1.0;
        if (WORLD) {
            const double2 cc = __ldg(w.sp_cen + gs);
            const double *Ki = vd.Kinv;
            double nn[3] = {vd.wz[0], vd.wz[1], vd.wz[2]};
            const double ray[3] = {Ki[0] * cc.x + Ki[1] * cc.y + Ki[2], Ki[3] * cc.x + Ki[4] * cc.y + Ki[5],
                                   Ki[6] * cc.x + Ki[7] * cc.y + Ki[8]};
            double nr = nn[0] * ray[0] + nn[1] * ray[1] + nn[2] * ray[2];
            if (nr > 0) { nn[0] = -nn[0]; nn[1] = -nn[1]; nn[2] = -nn[2]; nr = -nr; }
            gh0 = (Ki[0] * nn[0] + Ki[3] * nn[1] + Ki[6] * nn[2]) / nr;
            gh1 = (Ki[1] * nn[0] + Ki[4] * nn[1] + Ki[7] * nn[2]) / nr;
            gh2 = (Ki[2] * nn[0] + Ki[5] * nn[1] + Ki[8] * nn[2]) / nr;
            sh.n[0] = (float)nn[0]; sh.n[1] = (float)nn[1]; sh.n[2] = (float)nn[2];
        } else {
            sh.n[0] = 0.f; sh.n[1] = 0.f; sh.n[2] = -1.f;
        }
        sh.gh[0] = gh0; sh.gh[1] = gh1; sh.gh[2] = gh2;
        sh.gh[3] = gh0 * ref.x + gh1 * ref.y + gh2;
    }
    if (threadIdx.x < nnb) {
        const PairDev &pd = w.pairs[v * LFD_MAXN + threadIdx.x];
        SweepPair sp;
        sp.a00 = pd.Pf[0]; sp.a01 = pd.Pf[1];
        sp.a10 = pd.Pf[3]; sp.a11 = pd.Pf[4];
        sp.a20 = pd.Pf[6]; sp.a21 = pd.Pf[7];
        sp.Wi = pd.Wi; sp.Hi = pd.Hi;
        for (int r = 0; r < 3; r++) {
            sp.pref[r] = pd.P[3 * r] * ref.x + pd.P[3 * r + 1] * ref.y + pd.P[3 * r + 2];
            sp.q[r] = pd.q[r];
            sp.p0[r] = pd.P[3 * r];
            sp.p1[r] = pd.P[3 * r + 1];
        }
        sp.icw = sp.pref[2] > 0.0 ? 1.0 / sp.pref[2] : 0.0;
        sp.tex = pd.quad_i;
        sh.pair[threadIdx.x] = sp;
    }
    __syncthreads();

    const float T = vd.T;
    float best_cost = INFINITY;
    int best_k = 0x7fffffff;
    for (int k0 = 0; k0 < L; k0 += THREADS) {
        const int k = k0 + threadIdx.x;
        const bool active = k < L;
        const double u = vd.jitter ? jitter_u(vd.seed, vd.lf_index, vd.lv, s, active ? k : 0) : 0.5;
        const double z = vd.inv_dmax + ((double)(active ? k : 0) + u) * vd.delta;
        // the label's cost is summed per chunk (at most 128 pixels times the
        // neighbour views) and the chunk sums are added up, which keeps the
        // FP32 sum within ~1e-5 relative for superpixels of any size
        float total = 0.f;
        for (int pc = 0; pc < n; pc += SWEEP_CHUNK) {
            float cost = 0.f;
            const int cn = min(SWEEP_CHUNK, n - pc);
            __syncthreads();
            for (int i = threadIdx.x; i < cn; i += THREADS) {
                const unsigned pk = __ldg(w.sp_pix + off + pc + i);
                const int x = pk & 0xffff, y = pk >> 16;
                sh.d[i] = make_float2((float)(x - ref.x), (float)(y - ref.y));
                const float3 rc = texel_colour<FMT>(own_tex, x, y, vd.W, vd.H);
                float front = 1.f;
                if (WORLD) front = (sh.gh[0] * x + sh.gh[1] * y + sh.gh[2]) > 0.0 ? 1.f : 0.f;
                sh.ref[i] = make_float4(rc.x, rc.y, rc.z, front);
            }
            if (!WORLD) {
                __syncthreads();
                for (int t = threadIdx.x; t < cn * nnb; t += THREADS) {
                    const int j = t / cn, i = t - j * cn;
                    const SweepPair &sp = sh.pair[j];
                    const float2 d = sh.d[i];
                    if (PF == PF_SHIFT) {
                        // the pixel offset and, for 16-bit textures, the pixel's colour in
                        // the texture's format (one broadcast per sample instead of two),
                        // else its offset in view j's sampling texture
                        const int du = (int)d.x, dv = (int)d.y;
                        if constexpr (tex_fmt<FMT>() != LFD_RGBA_F32) {
                            const float4 rc = sh.ref[i];
                            sh.xyw[j][i] = make_float4(__int_as_float(du), __int_as_float(dv),
                                                       __uint_as_float(pack2<tex_fmt<FMT>()>(rc.x, rc.y)),
                                                       __uint_as_float(pack2<tex_fmt<FMT>()>(rc.z, 0.f)));
                        } else {
                            sh.xyw[j][i] = make_float4(__int_as_float(du), __int_as_float(dv),
                                                       __int_as_float(dv * (sp.Wi + 1) + du), 0.f);
                        }
                    } else {
                        sh.xyw[j][i] = make_float4(fmaf(sp.a00, d.x, sp.a01 * d.y), fmaf(sp.a10, d.x, sp.a11 * d.y),
                                                   fmaf(sp.a20, d.x, sp.a21 * d.y), 0.f);
                    }
                }
            }
            __syncthreads();
            for (int j = 0; j < nnb; j++) {
                const SweepPair &sp = sh.pair[j];
                // FP64 composition of the label's homography, anchored at ref
                const double zq0 = z * sp.q[0], zq1 = z * sp.q[1], zq2 = z * sp.q[2];
                const float cx = (float)fma(zq0, sh.gh[3], sp.pref[0]);
                const float cy = (float)fma(zq1, sh.gh[3], sp.pref[1]);
                const float cw = (float)fma(zq2, sh.gh[3], sp.pref[2]);
                float a00 = sp.a00, a01 = sp.a01, a10 = sp.a10, a11 = sp.a11, a20 = sp.a20, a21 = sp.a21;
                if (WORLD) {
                    a00 = (float)fma(zq0, sh.gh[0], sp.p0[0]); a01 = (float)fma(zq0, sh.gh[1], sp.p1[0]);
                    a10 = (float)fma(zq1, sh.gh[0], sp.p0[1]); a11 = (float)fma(zq1, sh.gh[1], sp.p1[1]);
                    a20 = (float)fma(zq2, sh.gh[0], sp.p0[2]); a21 = (float)fma(zq2, sh.gh[1], sp.p1[2]);
                }
                const void *tex = sp.tex;
                const int Wi = sp.Wi, Hi = sp.Hi;
                if (WORLD) {
#pragma unroll 4
                    for (int i = 0; i < cn; i++) {
                        const float2 d = sh.d[i];
                        const float4 rc = sh.ref[i];
                        const float X = fmaf(a00, d.x, fmaf(a01, d.y, cx));
                        const float Y = fmaf(a10, d.x, fmaf(a11, d.y, cy));
                        const float Wz = fmaf(a20, d.x, fmaf(a21, d.y, cw));
                        float t = tssd_sample<FMT>(tex, Wi, Hi, X, Y, Wz, make_float3(rc.x, rc.y, rc.z), T);
                        if (rc.w == 0.f) t = T;
                        cost += t;
                    }
                } else if (PF == PF_SHIFT) {
                    // translation pair: pixel offset (du, dv) samples at (du + X0, dv + Y0);
                    // with ix = du + floor(X0) and fx = X0 - floor(X0) the texture-area
                    // test -1/2 <= ix + fx < Wi - 1/2 is lo <= ix <= lo + Wi - 1, lo = -1
                    // when fx >= 1/2 and 0 otherwise (the same for y)
                    // The shift (X0, Y0) = (cx, cy) / w is split into its integer part and
                    // its fraction in FP64 (w = P (ref,1)_z for every label: q_z = 0), so
                    // the fraction is exact to FP32 rounding of a number below 1 whatever
                    // the image size (an absolute FP32 position near x = 2000 would carry
                    // ~1e-4 px).
                    const float4 *xyw = sh.xyw[WORLD ? 0 : j];
                    const double X0 = fma(zq0, sh.gh[3], sp.pref[0]) * sp.icw;
                    const double Y0 = fma(zq1, sh.gh[3], sp.pref[1]) * sp.icw;
                    if (sp.icw > 0.0 && fabs(X0) < 1e9 && fabs(Y0) < 1e9) {
                        const int ixk = __double2int_rd(X0), iyk = __double2int_rd(Y0);
                        const float fx = (float)(X0 - (double)ixk), fy = (float)(Y0 - (double)iyk);
                        const int ox = ixk + (fx >= 0.5f ? 1 : 0), oy = iyk + (fy >= 0.5f ? 1 : 0);
                        const unsigned spx = (unsigned)(Wi - 1), spy = (unsigned)(Hi - 1);
                        const long long koff = quad_index(ixk, iyk, Wi), npx = quad_entries(Wi, Hi);
#pragma unroll 4
                        for (int i = 0; i < cn; i++) {
                            const float4 q = xyw[i];
                            const int du = __float_as_int(q.x), dv = __float_as_int(q.y);
                            const bool in = (unsigned)(du + ox) <= spx && (unsigned)(dv + oy) <= spy;
                            // branch-free: a sample off the texture area reads entry 0
                            float t;
                            if constexpr (tex_fmt<FMT>() != LFD_RGBA_F32) {
                                const long long e = in ? koff + (dv * (Wi + 1) + du) : 0;
                                t = tssd_quad_href<FMT>(tex, e, npx, fx, fy, __float_as_uint(q.z),
                                                        __float_as_uint(q.w), T);
                            } else {
                                const float4 rc = sh.ref[i];
                                const long long e = in ? koff + __float_as_int(q.z) : 0;
                                t = tssd_quad<FMT>(tex, e, npx, fx, fy, make_float3(rc.x, rc.y, rc.z), T);
                            }
                            cost += in ? t : T;
                        }
                    } else {
                        for (int i = 0; i < cn; i++) cost += T;
                    }
                } else if (PF == PF_AFFINE) {
                    // affine pair: the homogeneous coordinate is cw for every pixel
                    // (P row 3 = (0, 0, P22), q_z = 0), one reciprocal per label and view;
                    // the same arithmetic as the general loop, value for value
                    const float4 *xyw = sh.xyw[WORLD ? 0 : j];
                    const float rw = rcp_approx(cw);
                    if (cw > 0.f) {
#pragma unroll 4
                        for (int i = 0; i < cn; i++) {
                            const float4 q = xyw[i];
                            const float4 rc = sh.ref[i];
                            cost += tssd_at<FMT>(tex, Wi, Hi, (q.x + cx) * rw, (q.y + cy) * rw,
                                                 make_float3(rc.x, rc.y, rc.z), T);
                        }
                    } else {
                        for (int i = 0; i < cn; i++) cost += T;
                    }
                } else {
                    const float4 *xyw = sh.xyw[WORLD ? 0 : j];
#pragma unroll 4
                    for (int i = 0; i < cn; i++) {
                        const float4 q = xyw[i];
                        const float4 rc = sh.ref[i];
                        cost += tssd_sample<FMT>(tex, Wi, Hi, q.x + cx, q.y + cy, q.z + cw,
                                                 make_float3(rc.x, rc.y, rc.z), T);
                    }
                }
            }
            total += cost;
        }
        const float cost = total;
        if (active) {
            if (cost_out) cost_out[(long long)gs * c.L + k] = cost * c.col_scale * c.col_scale;
            if (cost < best_cost) {   // k increases within a thread: strict < keeps the lowest k
                best_cost = cost;
                best_k = k;
            }
        }
    }
    // block arg-min, lowest k on ties
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oc = __shfl_xor_sync(0xffffffffu, best_cost, o);
        const int ok = __shfl_xor_sync(0xffffffffu, best_k, o);
        if (oc < best_cost || (oc == best_cost && ok < best_k)) {
            best_cost = oc;
            best_k = ok;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh.bc[wid] = best_cost;
        sh.bk[wid] = best_k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float bc = sh.bc[0];
        int bk = sh.bk[0];
        for (int i = 1; i < THREADS / 32; i++)
            if (sh.bc[i] < bc || (sh.bc[i] == bc && sh.bk[i] < bk)) {
                bc = sh.bc[i];
                bk = sh.bk[i];
            }
        const double u = vd.jitter ? jitter_u(vd.seed, vd.lf_index, vd.lv, s, bk) : 0.5;
        const double z = vd.inv_dmax + ((double)bk + u) * vd.delta;
        planes[gs] = make_float4((float)(1.0 / z), sh.n[0], sh.n[1], sh.n[2]);
        if (label_out) label_out[gs] = bk;
        atomicAdd(&w.ctr->hyp, (unsigned long long)L);
        atomicAdd(&w.ctr->samples, (unsigned long long)L * n * nnb);
    }
}

// camera-frame sweeps: 6 CTAs of 256 threads (12 of 128) per SM, at most 40
// registers; world-frame sweeps (more FP64 per label) 4, at most 64

// one CTA per superpixel of order_sweep[base .. base + count)
template <int FMT, bool WORLD, int THREADS, int PF>
__global__ void __launch_bounds__(THREADS, (WORLD ? 1024 : 1536) / THREADS) k_sweep(Workspace w, Consts c, int base,
                                                                                     float4 *planes, int *label_out,
                                                                                     float *cost_out)
{
    __shared__ SweepShared<THREADS, WORLD> sh;
    sweep_sp<FMT, WORLD, THREADS, PF>(w, c, __ldg(w.order_sweep + base + blockIdx.x), sh, planes, label_out,
                                       cost_out);
}

// persistent CTAs: superpixels of order_sweep[base .. base + count) taken in
// order (size classes, largest first), queue counter queue[qidx]
template <int FMT, bool WORLD, int THREADS, int PF>
__global__ void __launch_bounds__(THREADS, (WORLD ? 1024 : 1536) / THREADS) k_sweep_persistent(
    Workspace w, Consts c, int base, int count, int qidx, float4 *planes, int *label_out, float *cost_out)
{
    __shared__ SweepShared<THREADS, WORLD> sh;
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(&w.queue[qidx], 1);
        __syncthreads();
        const int item = sh.item;
        __syncthreads();
        if (item >= count) break;
        sweep_sp<FMT, WORLD, THREADS, PF>(w, c, __ldg(w.order_sweep + base + item), sh, planes, label_out, cost_out);
        __syncthreads();
    }
}

template <int FMT, bool WORLD, int THREADS, int PF>
static cudaError_t launch_sweep_a(const Workspace &w, const Consts &c, const LaunchCfg &lc, int base, int count,
                                  int qidx, float4 *planes, int *label, float *cost, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    if (lc.sweep_persistent) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, k_sweep_persistent<FMT, WORLD, THREADS, PF>, THREADS, 0);
        if (e != cudaSuccess) return e;
        const int grid = max(1, min(count, per_sm * lc.num_sms));
        k_sweep_persistent<FMT, WORLD, THREADS, PF><<<grid, THREADS, 0, st>>>(w, c, base, count, qidx, planes,
                                                                               label, cost);
    } else {
        k_sweep<FMT, WORLD, THREADS, PF><<<count, THREADS, 0, st>>>(w, c, base, planes, label, cost);
    }
    return cudaGetLastError();
}

template <int FMT, bool WORLD, int THREADS>
static cudaError_t launch_sweep_t(const Workspace &w, const Consts &c, const LaunchCfg &lc, int base, int count,
                                  int qidx, float4 *planes, int *label, float *cost, cudaStream_t st)
{
    if (!WORLD && c.affine && c.shift)
        return launch_sweep_a<FMT, false, THREADS, PF_SHIFT>(w, c, lc, base, count, qidx, planes, label, cost, st);
    if (!WORLD && c.affine)
        return launch_sweep_a<FMT, false, THREADS, PF_AFFINE>(w, c, lc, base, count, qidx, planes, label, cost, st);
    return launch_sweep_a<FMT, WORLD, THREADS, PF_GENERAL>(w, c, lc, base, count, qidx, planes, label, cost, st);
}

template <int FMT>
static cudaError_t launch_sweep_f(const Workspace &w, const Consts &c, const LaunchCfg &lc, int threads, int base,
                                  int count, int qidx, float4 *planes, int *label, float *cost, cudaStream_t st)
{
    if (c.sweep_frame)   // world-frame sweeps: 128 or 256 threads
        return threads <= 128 ? launch_sweep_t<FMT, true, 128>(w, c, lc, base, count, qidx, planes, label, cost, st)
                              : launch_sweep_t<FMT, true, 256>(w, c, lc, base, count, qidx, planes, label, cost, st);
    switch (threads) {
    case 64: return launch_sweep_t<FMT, false, 64>(w, c, lc, base, count, qidx, planes, label, cost, st);
    case 128: return launch_sweep_t<FMT, false, 128>(w, c, lc, base, count, qidx, planes, label, cost, st);
    case 160: return launch_sweep_t<FMT, false, 160>(w, c, lc, base, count, qidx, planes, label, cost, st);
    case 192: return launch_sweep_t<FMT, false, 192>(w, c, lc, base, count, qidx, planes, label, cost, st);
    case 224: return launch_sweep_t<FMT, false, 224>(w, c, lc, base, count, qidx, planes, label, cost, st);
    default: return launch_sweep_t<FMT, false, 256>(w, c, lc, base, count, qidx, planes, label, cost, st);
    }
}

cudaError_t launch_sweep(const Workspace &w, const Consts &c, const LaunchCfg &lc, int threads, int base, int count,
                         int qidx, float4 *planes, int *label, float *cost, cudaStream_t st)
{
    switch (c.fmt) {
    case LFD_RGBA8: return launch_sweep_f<LFD_RGBA8>(w, c, lc, threads, base, count, qidx, planes, label, cost, st);
    case LFD_RGBA_F16:
        return launch_sweep_f<LFD_RGBA_F16>(w, c, lc, threads, base, count, qidx, planes, label, cost, st);
    case LFD_RGBA_BF16:
        return launch_sweep_f<LFD_RGBA_BF16>(w, c, lc, threads, base, count, qidx, planes, label, cost, st);
    case LFD_RGBA_F32:
        return launch_sweep_f<LFD_RGBA_F32>(w, c, lc, threads, base, count, qidx, planes, label, cost, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lfd
