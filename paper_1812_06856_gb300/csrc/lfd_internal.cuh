// Internal device-side layout and helpers of liblfdepth (sm_103a).
//
// HBM layout of one bound light field (all views of one frame):
//   superpixels are numbered globally, gs = sp_base[v] + s;
//   pixels of all views are numbered globally, px_base[v] + y*W + x.
//   sp_off[gs] .. sp_off[gs+1]   range of sp_pix for superpixel gs
//   sp_pix[]                     packed pixel (y << 16 | x), row-major order per superpixel
//   sp_cnt, sp_ref (rounded centroid), sp_cen (FP64 centroid), sp_col {r,g,b,minw}
//   quad textures                per pixel the 2x2 block (x,y),(x+1,y),(x,y+1),(x+1,y+1),
//                                edges clamped: one load serves a bilinear sample
//   maps                         per pixel float4 {superpixel mean colour, depth value},
//                                written by the rasteriser, gathered by the energy kernel
//   sp_g / sp_rc                 per-superpixel plane coefficients of the current state
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/lfdepth.h"

#define LFD_MAXN LFD_MAX_NEIGHBOR_VIEWS
#define LFD_MAX_RADII 64
#define LFD_MAX_PERTURB 24

namespace lfd {

// status-word bits raised by kernels (read by lfd_synchronize)
enum : int { DEV_ERR_LABEL = 1, DEV_ERR_COUNT = 2 };

struct ViewDev {
    int W, H, GW, GH;
    int S, sp_base;
    long long px_base;
    int nnb;
    int ksize_init, ksteps_init;
    int lf;                  // light field this view belongs to
    double Kinv[9];
    double wz[3];            // world z axis in this camera's frame (R e3), for world-frame sweeps
    const int *labels;       // caller label map (valid during lfd_set_input only)
    const void *img;         // caller image (valid during lfd_set_input only)
    long long pitch;         // its row pitch in bytes
    void *quad;              // sampling texture (format dependent)
    float4 *map;             // rasterised {colour, depth value}
    // parameters of the view's light field
    int L, jitter, lf_index, term_mask;
    int iters, warm_off;
    int lv;                  // index of the view within its light field (jitter key)
    int sweep_skip;          // 1: the view starts from given (warm) planes; the sweep leaves it out
    unsigned long long seed;
    double inv_dmin, inv_dmax, delta;   // delta: inverse-depth bin width
    float T;                 // Eq. 1 truncation in the sampler's colour units squared
    float k_col;             // log2(e) / (2 alpha^2)     (Eq. 7)
    float k_sig;             // log2(e) / (2 sigma^2)     (Eq. 6, Eq. 10)
    float eta;               // Eq. 11
    float xy_lo, xy_hi;      // X/Y split: inverse domain X iff zeta >= D xy_lo; depth domain X iff z <= D xy_hi
    float col_gain;          // sqrt(k_col): scale of the colours in the rasterised maps
    float dep_gain;          // sqrt(k_sig): scale of their depth values
    int perturb_k;           // perturbation samples of the refinement (flagged variant; 0 = off)
    int sclass;              // sweep class: label-count class of its light field x 3 + the pair form of
                             // its neighbour pairs (0 general, 1 affine, 2 translation), see NSCLASS
    double perturb_scale;    // their relative radius at I = 1
};

// view v -> its k-th neighbour view i.  The plane with inverse-depth vector g
// (1/depth(p) = g . (p,1)) induces the homography A(g) = P + q g^T from
// homogeneous pixels of v to homogeneous pixels of i (Section III-B), with
// P = K_i R_rel K_v^-1, q = K_i t_rel, R_rel = R_i R_v^T, t_rel = t_i - R_rel t_v.
// Row 3 of A(g) p is the point's camera-i depth times g.p.
struct PairDev {
    int i, Wi, Hi, pad;
    double P[9];
    double q[3];
    float Pf[9];
    float qf[3];
    const void *quad_i;
    const float4 *map_i;
};

struct DevCounters {
    unsigned long long hyp;
    unsigned long long samples;
    int status;
    int bad_view, bad_index, pad;
};

// parameters shared by every view of a launch (the rest is per view in ViewDev)
struct Consts {
    int V, L, fmt, domain;   // L: label count of single-light-field calls (cost_out stride)
    int sweep_frame;
    int batch_iters;         // 1: a view whose light field has run its iterations passes its plane through
    float col_scale;         // sampler colour units -> [0,1]
    int cand_batch;          // candidate planes per pass (16 or 32; LaunchCfg::prop_batch)
    int affine;              // 1: every pair's homography has third row (0, 0, c) for every plane
                             //    (parallel cameras, common principal depth axis): the sample's depth
                             //    term is constant per (hypothesis, view) and the kernels skip it
    int shift;               // 1: affine, and every pair's P has upper 2 x 2 block P22 I (rectified
                             //    cameras with equal intrinsics): a fronto-parallel sweep plane
                             //    translates the image, the sweep samples at integer offsets plus
                             //    per-label fractions
};

struct Workspace {
    const ViewDev *views;
    const PairDev *pairs;    // [V * LFD_MAXN]
    const int *sp_view;      // [S_total]
    const int *sp_off;       // [S_total + 1]
    const int *sp_cnt;       // [S_total]
    const unsigned *sp_pix;  // [total px]
    const int2 *sp_ref;      // [S_total]
    const double2 *sp_cen;   // [S_total]
    const float4 *sp_col;    // [S_total] {r,g,b,minw}
    const double4_32a *sp_g; // [S_total] plane g (FP64), w = 1 valid
    const float4 *sp_rc;     // [S_total] {g.ref, g0, g1, valid} FP32 (rasteriser)
    const short *radii;      // [V][LFD_MAX_ITER_INDEX + 1][LFD_MAX_RADII]
    const int *radii_cnt;    // [V][LFD_MAX_ITER_INDEX + 1]
    DevCounters *ctr;
    const int *order;        // [S_total] work order: descending pixel-slot class, index order inside
    const int *order_sweep;  // [S_total] sweep work order: descending power-of-two size class, index order inside
    int *queue;              // [32] work-queue counters of persistent launches
    int S_total;
    long long px_total;
};

// arguments of the fusion kernels for one light field (device arrays)
struct FuseArgs {
    int V;                           // views of the light field
    float tau;                       // relative agreement tolerance
    const int *W, *H;                // [V]
    const long long *zoff;           // [V] word offset of reference view r's z-buffer planes
    const float *const *depth_in;    // [V]
    float *const *depth_out;         // [V]
    const float *mats;               // [V * V][12]: M (row-major 3x3) and e of source i -> reference r
    unsigned *zbuf;
};

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Blackwell packed single precision (sm_100 and later): two IEEE binary32
// operations, each rounded to nearest like its scalar form, in one
// instruction (the sweep interpolates red and green as a pair).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pc, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\tmov.b64 pc, {%6, %7};\n\t"
        "fma.rn.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ float2 fmul2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mul.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 fsub2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 dup2(float x) { return make_float2(x, x); }

// exact byte -> float through the 2^23 mantissa trick (byte c of w)
template <int C>
__device__ __forceinline__ float u8_to_f(unsigned w)
{
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | C)) - 8388608.0f;
}

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    // Steele, Lea, Flood (OOPSLA 2014) finaliser of the golden-gamma increment
    unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// uniform [0,1) jitter of label k of superpixel s of view v (Section III-B)
__device__ __forceinline__ double jitter_u(unsigned long long seed, int lf, int v, int s, int k)
{
    unsigned long long key = ((((unsigned long long)lf << 12) + (unsigned long long)v) << 20) + (unsigned long long)s;
    key = (key << 12) + (unsigned long long)k;
    return (double)(splitmix64(seed ^ key) >> 11) * (1.0 / 9007199254740992.0);
}

// uniform [0,1) draw j of the perturbation variant for superpixel s of view v
// (index within its light field) at iteration I
__device__ __forceinline__ double perturb_u(unsigned long long seed, int lf, int v, int s, int I, int j)
{
    unsigned long long key = ((((unsigned long long)lf << 12) + (unsigned long long)v) << 20) + (unsigned long long)s;
    key = (key << 7) + (unsigned long long)I;
    key = (key << 7) + (unsigned long long)j;
    return (double)(splitmix64((seed ^ 0x5045525455524231ULL) ^ key) >> 11) * (1.0 / 9007199254740992.0);
}

// Propagation-kernel cell of candidate m (Eq. 4, Fig. 3a): m = 0 own cell,
// 1..8 the ring E NE N NW W SW S SE (y down), then 8 cells per distinct ray radius.
__device__ __forceinline__ void ring_dir(int d, int &dx, int &dy)
{
    switch (d) {
    case 0: dx = 1; dy = 0; break;
    case 1: dx = 1; dy = -1; break;
    case 2: dx = 0; dy = -1; break;
    case 3: dx = -1; dy = -1; break;
    case 4: dx = -1; dy = 0; break;
    case 5: dx = -1; dy = 1; break;
    case 6: dx = 0; dy = 1; break;
    default: dx = 1; dy = 1; break;
    }
}

// launch shape of the two hot kernels (chosen by the autotuner)
struct LaunchCfg {
    int sweep_threads;       // 128 or 256 threads (labels) per CTA
    int sweep_persistent;    // 1: persistent CTAs over a cost-ordered queue
    int prop_blocks;         // 7 or 8 resident 4-warp CTAs per SM (register budget)
    int prop_persistent;     // 1: persistent warps over a cost-ordered queue
    int num_sms;
    int prop_batch;          // 16 or 32 candidate planes per pass over the neighbour views
    int order_bands;         // 1 or 16 row bands in the work orders
    int prop_coop;           // 1: persistent CTAs whose 4 warps share one superpixel (k_propagate_coop)
};

cudaError_t launch_sp_count(const Workspace &w, int V, int max_px, int *cnt, int4 *bbox, cudaStream_t st);
cudaError_t launch_sp_scan(const Workspace &w, int V, const int *cnt, int *off, cudaStream_t st);
cudaError_t launch_sp_collect(const Workspace &w, const Consts &c, const int4 *bbox, const int *cnt, unsigned *pix,
                              double2 *cen, int2 *ref, float4 *col, cudaStream_t st);
cudaError_t launch_sp_minw(const Workspace &w, const Consts &c, float4 *col, cudaStream_t st);
cudaError_t launch_quads(const Workspace &w, int V, int max_px, int fmt, cudaStream_t st);
// mode 0: pixel-slot classes ceil(n/32) (propagation); mode 1: power-of-two classes floor(log2 n) (sweep)
// keys of the work orders' counting sort: 17 size classes x 16 row bands
constexpr int ORDER_CLASSES = 17;
constexpr int ORDER_BANDS = 16;
constexpr int ORDER_KEYS = ORDER_CLASSES * ORDER_BANDS;
// Label-count classes of the sweep: a light field of L labels is swept by
// CTAs of LCLASS_THREADS[c] threads, the smallest width >= L (256 beyond:
// several passes), so that few threads idle when L is not a multiple of 256.
constexpr int LCLASSES = 6;
constexpr int LCLASS_THREADS[LCLASSES] = {64, 128, 160, 192, 224, 256};
// sweep classes: one sweep launch per (label-count class, pair form) present,
// so that each view of a batch of mixed rigs sweeps with its own pair form
constexpr int NSCLASS = LCLASSES * 3;
constexpr int QUEUE_INTS = 32;          // 4 + NSCLASS <= QUEUE_INTS
inline int label_class(int L)
{
    for (int c = 0; c < LCLASSES; c++)
        if (L <= LCLASS_THREADS[c]) return c;
    return LCLASSES - 1;
}
// mode 0: propagation order (pixel-slot class, band); 1: sweep order
// (power-of-two size class, band); 2: stable partition of `in` by the
// label-count class of each superpixel's light field.  bands: 1 ..
// ORDER_BANDS row bands inside a size class.  in: NULL = index order.
cudaError_t launch_sp_order(const Workspace &w, int *order, int *hist, int mode, int bands, const int *in,
                            cudaStream_t st);  // hist: ORDER_KEYS ints
// sweep of the superpixels order_sweep[base .. base + count) with CTAs of
// `threads` threads (one of LCLASS_THREADS), queue counter queue[qidx]
cudaError_t launch_sweep(const Workspace &w, const Consts &c, const LaunchCfg &lc, int threads, int base, int count,
                         int qidx, float4 *planes, int *label, float *cost, cudaStream_t st);
cudaError_t launch_plane_prep(const Workspace &w, const Consts &c, const float4 *planes, double4_32a *g, float4 *rc,
                              cudaStream_t st);
cudaError_t launch_rasterize(const Workspace &w, const Consts &c, float *const *depth, cudaStream_t st);
cudaError_t launch_propagate(const Workspace &w, const Consts &c, const LaunchCfg &lc, int iter,
                             const float4 *planes_in, float4 *planes_out, int *choice, float *energy,
                             cudaStream_t st);
cudaError_t launch_fuse(const FuseArgs &a, long long zbuf_words, int max_px, cudaStream_t st);
cudaError_t launch_score(const Workspace &w, const Consts &c, const float4 *planes_state, int nq, const lfd_query *q,
                         float *out, cudaStream_t st);
}  // namespace lfd
