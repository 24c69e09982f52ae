// Steps a5-a7: depth rasterisation and the parallel propagation / plane
// refinement of Section III-C and III-E.
//
// Every superpixel of every view is refined at once (Jacobi): the kernels read
// only the previous iteration's planes (planes_in, via sp_g / sp_rc) and the
// maps rasterised from them, and write planes_out.
//
// Energy (Eq. 3): E = E_c * E_s.
//   E_s (Eq. 5-7): colour-weighted mean over the present 8-neighbours j of
//       exp(-(d_j - d_j(plane))^2 / 2 sigma^2), d_j(plane) the hypothesis
//       extrapolated to neighbour j's centroid.  Weights are evaluated as
//       exp(-(a_j - min a)) / sum (same value, no 0/0 in FP32).
//   E_c (Eq. 8): mean over the neighbour views i of V_i + O_i, with
//       S_i (Eq. 9) the mean colour similarity between the superpixel and the
//       view-i superpixel hit by each pixel (nearest pixel), V_i (Eq. 10) =
//       S_i * mean over X of exp(-(D(p) - D_i(p_i))^2 / 2 sigma^2) where X are
//       the pixels whose 3-D point is not behind view i's surface, and O_i
//       (Eq. 11) = eta (1 - min_j omega) when some pixel lies behind it.
//
// Mapping: one warp per superpixel; lanes own pixels (ceil(n/32) slots per
// lane, a compile-time count chosen per superpixel, up to 10 staged in shared
// memory and more streamed), so the gathers of a warp into a neighbour view's
// map fall in a compact footprint.  Hypotheses are scored one after another by
// the whole warp; per view the five sums are reduced with REDUX (counts) and
// butterfly shuffles (sums) in a fixed order, so results are deterministic.
// What does not depend on the view (the FP32 form of the plane and E_s) is
// computed once per candidate, lane-parallel over a batch of 32.
//
// Projection precision: for each (hypothesis, view) the homography applied to
// the superpixel's anchor pixel is composed in FP64 and split into an integer
// pixel (xi, yi) plus FP32 residuals; per pixel only offsets from the anchor
// are evaluated in FP32, which keeps the sub-pixel position exact to ~1e-6 px
// and makes the nearest-pixel choice match an FP64 evaluation except within
// that distance of a rounding boundary.
#include "lfd_sample.cuh"

namespace lfd {

typedef double4_32a dbl4;

constexpr int PROP_WARPS = 4;
constexpr int SLOTS_MAX = 10;   // pixel slots per lane staged in shared memory (320 pixels per warp)


// FP64 reciprocal and reciprocal square root by Newton-Raphson refinement of
// the FP32 hardware estimates (two steps each: y += y (1 - x y) and
// y += y (1/2 - x y^2 / 2)), which leaves ~1 ulp; outside FP32's normal range
// the IEEE operations.  Short code on the low-rate FP64 pipe.
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ double rcp64(double x)
{
    const float a = fabsf((float)x);
    if (!(a >= 1e-30f && a <= 1e30f)) return 1.0 / x;
    double y = (double)rcp_approx((float)x);
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

__device__ __forceinline__ double rsqrt64(double x)
{
    const float a = (float)x;
    if (!(a >= 1e-30f && a <= 1e30f)) return 1.0 / sqrt(x);
    double y = (double)rsqrt_approx(a);
    const double h = 0.5 * x;
    double e = fma(-h * y, y, 0.5);
    y = fma(y, e, y);
    e = fma(-h * y, y, 0.5);
    return fma(y, e, y);
}

// ---------------------------------------------------------------------------
// plane coefficients of a state: g with 1/depth(p) = g . (p,1)
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool plane_to_g(const ViewDev &vd, double d, double nx, double ny, double nz, double cx,
                                           double cy, double &g0, double &g1, double &g2)
{
    g0 = g1 = g2 = 0.0;
    if (!(d > 0.0) || !isfinite(d) || !isfinite(nx) || !isfinite(ny) || !isfinite(nz)) return false;
    const double *K = vd.Kinv;
    const double rx = K[0] * cx + K[1] * cy + K[2];
    const double ry = K[3] * cx + K[4] * cy + K[5];
    const double rz = K[6] * cx + K[7] * cy + K[8];
    const double rho = d * (nx * rx + ny * ry + nz * rz);       // n . X_c
    if (!(fabs(rho) > 0.0) || !isfinite(rho)) return false;
    const double ir = rcp64(rho);
    g0 = (K[0] * nx + K[3] * ny + K[6] * nz) * ir;               // K^-T n / rho
    g1 = (K[1] * nx + K[4] * ny + K[7] * nz) * ir;
    g2 = (K[2] * nx + K[5] * ny + K[8] * nz) * ir;
    return isfinite(g0) && isfinite(g1) && isfinite(g2);
}

__global__ void k_plane_prep(Workspace w, const float4 *planes, dbl4 *g_out, float4 *rc_out)
{
    const int gs = blockIdx.x * blockDim.x + threadIdx.x;
    if (gs >= w.S_total) return;
    const ViewDev &vd = w.views[__ldg(w.sp_view + gs)];
    const float4 p = planes[gs];
    double g0 = 0, g1 = 0, g2 = 0;
    bool ok = false;
    if (__ldg(w.sp_cnt + gs) > 0) {
        const double2 c = w.sp_cen[gs];
        ok = plane_to_g(vd, p.x, p.y, p.z, p.w, c.x, c.y, g0, g1, g2);
    }
    const int2 ref = w.sp_ref[gs];
    dbl4 g;
    g.x = g0; g.y = g1; g.z = g2; g.w = ok ? 1.0 : 0.0;
    g_out[gs] = g;
    rc_out[gs] = make_float4((float)(g0 * ref.x + g1 * ref.y + g2), (float)g0, (float)g1, ok ? 1.f : 0.f);
}

cudaError_t launch_plane_prep(const Workspace &w, const Consts &c, const float4 *planes, double4_32a *g, float4 *rc,
                              cudaStream_t st)
{
    (void)c;
    k_plane_prep<<<(w.S_total + 127) / 128, 128, 0, st>>>(w, planes, g, rc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// rasteriser: warp per superpixel writes {colour, depth value} of its pixels
// ---------------------------------------------------------------------------
//
// The map holds the superpixel's mean colour times sqrt(k_col) and the depth
// value (inverse depth, or depth in the metric domain) times sqrt(k_sig) of
// the view's light field, so that the exponents of Eq. 7 / Eq. 9 and of the
// Gaussian of Eq. 10 are plain squared distances in the energy kernel.  (An
// 8-B texel {depth value, superpixel} with the colours in a table halves the
// gathered bytes but adds a dependent gather per sample: measured 17-19 %
// slower on the 8 x 1024x768 and 16 x 1080p frames.)

__global__ void __launch_bounds__(128) k_rasterize(Workspace w, Consts c, float *const *depth)
{
    const int gs = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (gs >= w.S_total) return;
    const int v = __ldg(w.sp_view + gs);
    const ViewDev &vd = w.views[v];
    const int n = __ldg(w.sp_cnt + gs);
    const int off = __ldg(w.sp_off + gs);
    const float4 rc = w.sp_rc[gs];
    const float4 col = w.sp_col[gs];
    const int2 ref = w.sp_ref[gs];
    const float cgain = vd.col_gain, dgain = vd.dep_gain;
    const float4 cc = make_float4(col.x * cgain, col.y * cgain, col.z * cgain, 0.f);
    float4 *map = vd.map;
    float *dep = depth ? depth[v] : nullptr;
    for (int i = lane; i < n; i += 32) {
        const unsigned pk = __ldg(w.sp_pix + off + i);
        const int x = pk & 0xffff, y = pk >> 16;
        const float inv = fmaf(rc.y, (float)(x - ref.x), fmaf(rc.z, (float)(y - ref.y), rc.x));
        const bool ok = rc.w != 0.f && inv > 0.f && isfinite(inv);
        const float dv = ok ? (c.domain == 0 ? inv : 1.0f / inv) : 0.f;
        const long long p = (long long)y * vd.W + x;
        map[p] = make_float4(cc.x, cc.y, cc.z, dv * dgain);
        if (dep) dep[p] = ok ? 1.0f / inv : 0.f;
    }
}

cudaError_t launch_rasterize(const Workspace &w, const Consts &c, float *const *depth, cudaStream_t st)
{
    const int blocks = (w.S_total + 3) / 4;
    k_rasterize<<<blocks, 128, 0, st>>>(w, c, depth);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// energy evaluation shared by the propagation and score kernels
// ---------------------------------------------------------------------------
//
// Per warp (one superpixel), shared memory holds what does not change across
// hypotheses: for each neighbour view k the homography pieces anchored at an
// integer pixel (xa, ya) near the projection of the superpixel's reference
// pixel under its current plane (composed in FP64, stored in FP32), and for
// each 8-neighbour its depth, centroid and colour weight.  A hypothesis g is
// reduced once, in FP64, to the FP32 quantities of HypF (E_s of Eq. 5-7
// included), lane-parallel over the candidates of a batch; the per-pixel work
// is then FP32 on small quantities only:
//   dg = g.(ref,1) - g_a.(ref,1)  (FP64 difference, rounded once),
//   hw = hw_a + q_z dg,   cx = Ex + Dx dg,   cy = Ey + Dy dg,
//   per pixel offset (du,dv) from ref:
//     Nw = hw + a20 du + a21 dv,  x = xa + (cx + b0 du + b1 dv)/Nw, ...
// which keeps the sub-pixel position of neighbouring hypotheses to ~1e-6 px.

struct alignas(16) SpView {
    float hw_a, qw, Ex, Dx;
    float Ey, Dy;
    int xa_m, ya_m;                      // anchor pixel minus the bits of 1.5 * 2^23 (see energy_sample)
    float Pp00, Pp01, Pp10, Pp11;        // P00 - xa P20, P01 - xa P21, P10 - ya P20, P11 - ya P21
    float P20, P21;
    int Wi, Hi;
    const float4 *map;
    long long pad2;
};

struct alignas(16) SpNb {
    double invd, d, cx, cy;              // neighbour's current depth (inverse, metric) and centroid
    double Px, Py, Pz;                   // its centroid point d K^-1 (c,1) (Fig. 3b vertices)
    float w;                             // colour weight exp(-(a_j - min a))
    int ok;
    float fdx, fdy;                      // c_j - c (own centroid), FP32
    float finvd, fd;                     // invd, d in FP32
};

// the superpixel a warp works on (identical in every lane)
struct WarpSP {
    int gs, v, s, n, off, nnb, gx, gy;
    int2 ref;
    float cr, cg, cb, minw, sum_w;       // colour scaled by sqrt(k_col)
};

struct alignas(16) SpShared {
    // offsets from ref of the first 32*SLOTS_MAX pixels, two slots per entry:
    // px4[32 jp + lane] = (du, du', dv, dv') of pixels lane + 64 jp and lane + 64 jp + 32
    float4 px4[32 * (SLOTS_MAX / 2)];
    WarpSP S;
    SpView view[LFD_MAXN];
    SpNb nb[8];
    double cx, cy, rx, ry, rz, rn, grefa;        // centroid, its ray K^-1(c,1), |ray|, anchor g.(ref,1)
    double best_ig;                              // winning candidate (propagation / refinement)
    double best_dep;                             // depth of the refinement winner
    float bnx, bny, bnz;
    int best_m;
    float k_sig, xy_lo, xy_hi, eta;              // energy constants of the superpixel's light field
    float rdx, rdy;                              // ref - c (anchor pixel minus centroid)
    int term_mask;
};

// FP32 reduction of a hypothesis g (see above): gp(p) = g0 du + g1 dv + gr is
// the hypothesis' inverse depth at pixel p, dgr the anchored offset of
// g.(ref,1), es its smoothness E_s.
struct HypF {
    float g0, g1, gr, dgr, es;
};

// candidate planes of one 32-wide batch (propagation) or the 8 triangles (refinement)
struct alignas(16) CandShared {
    float g0[32], g1[32], gr[32], dgr[32], es[32];
    float ec[32];                        // running sum over views of V_i + O_i (Eq. 8)
    double ig[32];
    float nx[32], ny[32], nz[32];
};

// per-warp records of the 4-warp propagation and score CTAs
__shared__ SpShared g_sh[PROP_WARPS];
__shared__ CandShared g_cs[PROP_WARPS];

// Cooperative propagation (k_propagate_coop): the CTA's 4 warps refine one
// superpixel together, so its record is per CTA; each warp keeps its own
// candidate batch.  The winners of the warps and the candidate index of
// every batch slot meet in CoopShared.
struct CoopShared {
    int item, ok;
    int cnt[PROP_WARPS];                 // valid candidates found by each warp in a round
    int mi[PROP_WARPS][32];              // candidate index m of batch slot (warp, slot)
    float E[PROP_WARPS];                 // each warp's best energy, its m (or t) and plane
    int m[PROP_WARPS];
    double ig[PROP_WARPS];
    float nx[PROP_WARPS], ny[PROP_WARPS], nz[PROP_WARPS];
    unsigned nh[PROP_WARPS];             // hypotheses scored per warp
};
__shared__ SpShared g_shc[1];
__shared__ CoopShared g_co;

// the superpixel record of this warp: its own, or the CTA's in the cooperative form
template <bool COOP>
__device__ __forceinline__ SpShared &sp_shared()
{
    if constexpr (COOP) return g_shc[0];
    else return g_sh[threadIdx.x >> 5];
}

struct Acc {
    unsigned cnt, nx, ny;
    float sw, sg;
};

struct ViewK {
    float hw, a20, a21, cx, b0, b1, cy, c0, c1;
    float xy;
    int xa_m, ya_m, Wi, Hi;
    const float4 *map;
};

// E_s (Eq. 5-7) of plane g for this lane; neighbours in ring order.  The
// plane's inverse depth at c_j is taken relative to its value igc at the own
// centroid, g . (c_j,1) = igc + g0 dx_j + g1 dy_j, so that FP32 suffices: the
// offsets are a few superpixel pitches and no large terms cancel.
template <int DOMAIN>
__device__ __forceinline__ float smoothness(const SpShared &sh, float sum_w, float g0, float g1, float igc)
{
    if (!(sum_w > 0.f)) return 1.f;
    float num = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const SpNb &nb = sh.nb[j];
        if (!nb.ok) continue;
        const float dext = fmaf(g0, nb.fdx, g1 * nb.fdy);          // g . (c_j,1) - igc
        float dl;
        bool has = true;
        if (DOMAIN == 0) {
            dl = (nb.finvd - igc) - dext;
        } else {
            const float ext = igc + dext;
            has = ext > 0.f;
            dl = has ? nb.fd - rcp_approx(ext) : 0.f;
        }
        if (has) num += nb.w * ex2_approx(-dl * dl * sh.k_sig);
    }
    return num * rcp_approx(sum_w);
}

// FP32 form of plane g whose inverse depth at the own centroid is igc
// (g . (c,1), FP64): everything relative to igc, so the only FP64 step left
// is the anchored difference igc - g_a . (ref,1).  The low-rate FP64 pipe of
// this GPU is kept for the few steps that need it.
template <int DOMAIN>
__device__ __noinline__ HypF hyp_prep(const WarpSP &S, const SpShared &sh, double g0, double g1, double igc)
{
    HypF h;
    const float g0f = (float)g0, g1f = (float)g1, igf = (float)igc;
    const float dref = fmaf(g0f, sh.rdx, g1f * sh.rdy);           // g . (ref,1) - igc
    h.g0 = g0f;
    h.g1 = g1f;
    h.gr = igf + dref;
    h.dgr = (float)(igc - sh.grefa) + dref;
    h.es = smoothness<DOMAIN>(sh, S.sum_w, g0f, g1f, igf);
    return h;
}

__device__ __forceinline__ void cand_store(CandShared &cs, int lane, const HypF &h)
{
    cs.g0[lane] = h.g0; cs.g1[lane] = h.g1; cs.gr[lane] = h.gr; cs.dgr[lane] = h.dgr; cs.es[lane] = h.es;
}

__device__ __forceinline__ HypF cand_load(const CandShared &cs, int src)
{
    HypF h;
    h.g0 = cs.g0[src]; h.g1 = cs.g1[src]; h.gr = cs.gr[src]; h.dgr = cs.dgr[src]; h.es = cs.es[src];
    return h;
}

// The part of one pixel-view sample of Eq. 9-11 after the projection:
// nearest pixel, window, gathers, sums.  Branch-free so that the samples of
// an unrolled loop keep their gathers in flight together; `act` false (a
// lane past the superpixel's last pixel) contributes nothing.  Nw: camera-i
// depth times g.p; r = 1/Nw; tx, ty: the offsets from the integer anchor
// plus 1.5 * 2^23 (see below); gp: the hypothesis' inverse depth at the
// pixel; val0 = gp r (inverse-depth domain).  Map colours and depth values
// carry sqrt(k_col) and sqrt(k_sig); the homography rows carry
// 1/sqrt(k_sig) (inverse-depth domain: 1/z_i = gp / Nw comes out scaled) or
// sqrt(k_sig) (metric: z_i = Nw / gp), which leaves the pixel position
// unchanged.
template <int DOMAIN, bool CHECKW = true>
__device__ __forceinline__ void sample_tail(const ViewK &K, bool act, float Nw, float tx, float ty, float gp,
                                            float val0, float cr, float cg, float cb, Acc &a)
{
    // Nearest pixel: adding 1.5 * 2^23 rounds an offset |f| < 2^22 to an
    // integer held in the low mantissa bits (ties to even: the oracle flags
    // an exact .5 as a rounding boundary where either pixel is admissible).
    // The point lies in view i iff that pixel does (-1/2 <= x < W - 1/2);
    // out-of-range or non-finite offsets give out-of-range integers.
    const int ix = __float_as_int(tx) + K.xa_m;
    const int iy = __float_as_int(ty) + K.ya_m;
    const bool ok = act && (gp > 0.f) && (!CHECKW || Nw > 0.f) && ((unsigned)ix < (unsigned)K.Wi) &&
                    ((unsigned)iy < (unsigned)K.Hi);
    const int idx = ok ? iy * K.Wi + ix : 0;                     // in-bounds address either way
    const float4 c = __ldg(K.map + idx);                         // {colour of the superpixel hit, depth value}
    const float tw = c.w;
    const float2 drg = fsub2(make_float2(c.x, c.y), make_float2(cr, cg));   // red, green as a packed pair
    const float2 d2 = fmul2(drg, drg);
    const float db = c.z - cb;
    const float om = ex2_approx(-fmaf(db, db, d2.x + d2.y));             // Eq. 9 summand
    a.cnt += ok ? 1u : 0u;
    a.sw += ok ? om : 0.f;
    const bool has = ok && tw > 0.f;
    float val;
    bool inX;
    if (DOMAIN == 0) {
        val = val0;                                              // 1 / z_i(P), scaled
        inX = has && val >= tw * K.xy;
    } else {
        val = Nw * rcp_approx(gp);                               // z_i(P), scaled
        inX = has && val <= tw * K.xy;
    }
    const float dd = val - tw;
    const float G = ex2_approx(-dd * dd);                        // Eq. 10 summand
    a.nx += inX ? 1u : 0u;
    a.sg += inX ? G : 0.f;
    a.ny += (has && !inX) ? 1u : 0u;
}

constexpr float ROUND_MAGIC = 12582912.0f;                      // 1.5 * 2^23

// one sample: projection of pixel offset (du, dv) into view i, then the
// tail.  AFF (affine pair: a20 = a21 = 0, so Nw = hw for every pixel): Nw and
// r = 1/hw come from the caller, which has checked hw > 0 once; the values
// are those of the general form, which computes hw + 0 du + 0 dv.
template <int DOMAIN, bool AFF = false>
__device__ __forceinline__ void energy_sample(const ViewK &K, bool act, float du, float dv, float gp, float cr,
                                              float cg, float cb, Acc &a, float r_aff = 0.f)
{
    const float Nw = AFF ? K.hw : fmaf(K.a20, du, fmaf(K.a21, dv, K.hw));   // camera-i depth * g.p
    const float ex = fmaf(K.b0, du, fmaf(K.b1, dv, K.cx));
    const float ey = fmaf(K.c0, du, fmaf(K.c1, dv, K.cy));
    const float r = AFF ? r_aff : rcp_approx(Nw);
    sample_tail<DOMAIN, !AFF>(K, act, Nw, fmaf(ex, r, ROUND_MAGIC), fmaf(ey, r, ROUND_MAGIC), gp, gp * r, cr, cg,
                              cb, a);
}

// The view terms V_i + O_i (Eq. 9-11) of every candidate of `mask` (a batch
// held in the warp's CandShared), added to cs.ec[candidate] in view order.
// The loop runs view-outer, candidate-inner: the candidates of one batch
// project the superpixel to nearly the same region of a neighbour view, so
// that region's map texels are reused from L1 across the batch.  SL pixel
// slots per lane; unless MASK_ALL, every slot but the last is full
// (n > 32 (SL - 1)).  With REC (one candidate), lane 0 writes the per-view
// terms of lfd_score to `rec`.  Lane c keeps candidate c's running sum in a
// register (the reduced terms are identical in every lane), so the loop has
// no divergent store.
template <int DOMAIN, int SL, bool MASK_ALL = false, bool REC = false, bool AFF = false, bool COOP = false>
__device__ __noinline__ void view_terms(const Workspace &w, unsigned mask, float *rec)
{
    const int lane = threadIdx.x & 31;
    const SpShared &sh = sp_shared<COOP>();
    CandShared &cs = g_cs[threadIdx.x >> 5];
    const WarpSP S = sh.S;
    float ec = cs.ec[lane];
    for (int k = 0; k < S.nnb; k++) {
        const SpView &sv = sh.view[k];
        unsigned mm = mask;
        while (mm) {
            const int src = __ffs(mm) - 1;
            mm &= mm - 1;
            const HypF h = cand_load(cs, src);
            ViewK K;
            K.hw = fmaf(sv.qw, h.dgr, sv.hw_a);
            K.cx = fmaf(sv.Dx, h.dgr, sv.Ex);
            K.cy = fmaf(sv.Dy, h.dgr, sv.Ey);
            K.b0 = fmaf(sv.Dx, h.g0, sv.Pp00);
            K.b1 = fmaf(sv.Dx, h.g1, sv.Pp01);
            K.c0 = fmaf(sv.Dy, h.g0, sv.Pp10);
            K.c1 = fmaf(sv.Dy, h.g1, sv.Pp11);
            K.a20 = fmaf(sv.qw, h.g0, sv.P20);
            K.a21 = fmaf(sv.qw, h.g1, sv.P21);
            K.xa_m = sv.xa_m; K.ya_m = sv.ya_m; K.Wi = sv.Wi; K.Hi = sv.Hi;
            K.map = sv.map;
            K.xy = DOMAIN == 0 ? sh.xy_lo : sh.xy_hi;
            Acc a = {0u, 0u, 0u, 0.f, 0.f};
            // affine pair: one reciprocal for every pixel; a plane behind
            // camera i there (hw <= 0) has no valid pixel
            const float r_aff = AFF ? rcp_approx(K.hw) : 0.f;
            if (!AFF || K.hw > 0.f) {
                // slots j and j + 1 come from one shared-memory load; every slot
                // but the last is full unless MASK_ALL
#pragma unroll
                for (int jp = 0; jp < (SL + 1) / 2; jp++) {
                    const int j0 = 2 * jp, j1 = 2 * jp + 1;
                    const float4 d = sh.px4[32 * jp + lane];
                    energy_sample<DOMAIN, AFF>(K, (!MASK_ALL && j0 + 1 < SL) || lane + 32 * j0 < S.n, d.x, d.z,
                                               fmaf(h.g0, d.x, fmaf(h.g1, d.z, h.gr)), S.cr, S.cg, S.cb, a, r_aff);
                    if (j1 < SL)
                        energy_sample<DOMAIN, AFF>(K, (!MASK_ALL && j1 + 1 < SL) || lane + 32 * j1 < S.n, d.y, d.w,
                                                   fmaf(h.g0, d.y, fmaf(h.g1, d.w, h.gr)), S.cr, S.cg, S.cb, a,
                                                   r_aff);
                }
                if (SL == SLOTS_MAX) {
#pragma unroll 2
                    for (int i = 32 * SL + lane; i < S.n; i += 32) {    // pixels beyond the staged slots
                        const unsigned pk = __ldg(w.sp_pix + S.off + i);
                        const float du = (float)((int)(pk & 0xffff) - S.ref.x);
                        const float dv = (float)((int)(pk >> 16) - S.ref.y);
                        energy_sample<DOMAIN, AFF>(K, true, du, dv, fmaf(h.g0, du, fmaf(h.g1, dv, h.gr)), S.cr, S.cg,
                                                   S.cb, a, r_aff);
                    }
                }
            }
            unsigned cnt, nx;
            if (S.n < 65536) {    // counts fit 16 bits: one REDUX for |Omega_i| and |X_i|
                const unsigned cx2 = __reduce_add_sync(0xffffffffu, a.cnt | (a.nx << 16));
                cnt = cx2 & 0xffffu;
                nx = cx2 >> 16;
            } else {
                cnt = __reduce_add_sync(0xffffffffu, a.cnt);
                nx = __reduce_add_sync(0xffffffffu, a.nx);
            }
            const unsigned ny = __reduce_add_sync(0xffffffffu, a.ny);
            const float sw = warp_sum(a.sw), sg = warp_sum(a.sg);
            const float Si = cnt > 0 ? sw * rcp_approx((float)cnt) : 0.f;                      // Eq. 9
            const float Vi = (cnt > 0 && nx > 0) ? Si * (sg * rcp_approx((float)nx)) : 0.f;    // Eq. 10
            const float Oi = (ny > 0 && (sh.term_mask & 4)) ? sh.eta * (1.f - S.minw) : 0.f;   // Eq. 11
            ec += lane == src ? Vi + Oi : 0.f;
            if (REC && lane == 0) {
                float *r = rec + LFD_TERMS_HEAD + k * LFD_TERMS_PER_VIEW;
                r[0] = Si; r[1] = Vi; r[2] = Oi; r[3] = (float)cnt; r[4] = (float)nx; r[5] = (float)ny;
            }
        }
    }
    cs.ec[lane] = ec;
    __syncwarp();
}

// E = E_c E_s (Eq. 3, Eq. 8) of candidate src after view_terms
__device__ __forceinline__ float cand_energy(const SpShared &sh, const CandShared &cs, int nnb, int src)
{
    const float Ec = nnb > 0 ? cs.ec[src] * rcp_approx((float)nnb) : 0.f;
    return ((sh.term_mask & 2) ? Ec : 1.f) * ((sh.term_mask & 1) ? cs.es[src] : 1.f);
}

// Warp-wide set-up of a superpixel: registers (pixels, colour) and the warp's
// shared record.  Returns false for an empty superpixel.  `ga` is the anchor
// plane (the current plane when valid).
template <int DOMAIN>
__device__ bool setup_sp(const Workspace &w, const float4 *planes_in, int gs, int lane, WarpSP &S, SpShared &sh,
                         bool ga_valid, double ga0, double ga1, double ga2)
{
    S.gs = gs;
    S.v = __ldg(w.sp_view + gs);
    const ViewDev &vd = w.views[S.v];
    S.s = gs - vd.sp_base;
    S.n = __ldg(w.sp_cnt + gs);
    if (S.n == 0) return false;
    S.off = __ldg(w.sp_off + gs);
    S.nnb = vd.nnb;
    S.gx = S.s % vd.GW;
    S.gy = S.s / vd.GW;
    S.ref = w.sp_ref[gs];
    const float4 col = w.sp_col[gs];
    S.minw = col.w;
    const double2 cc = w.sp_cen[gs];
    const double *Ki = vd.Kinv;
    const double rx = Ki[0] * cc.x + Ki[1] * cc.y + Ki[2];
    const double ry = Ki[3] * cc.x + Ki[4] * cc.y + Ki[5];
    const double rz = Ki[6] * cc.x + Ki[7] * cc.y + Ki[8];
    const double grefa = ga_valid ? ga0 * S.ref.x + ga1 * S.ref.y + ga2 : 0.5 * (vd.inv_dmin + vd.inv_dmax);
    if (lane == 0) {
        sh.k_sig = vd.k_sig;
        sh.xy_lo = vd.xy_lo;
        sh.xy_hi = vd.xy_hi;
        sh.eta = vd.eta;
        sh.term_mask = vd.term_mask;
        sh.cx = cc.x; sh.cy = cc.y;
        sh.rdx = (float)(S.ref.x - cc.x);
        sh.rdy = (float)(S.ref.y - cc.y);
        sh.rx = rx; sh.ry = ry; sh.rz = rz;
        const double rn2 = rx * rx + ry * ry + rz * rz;
        sh.rn = rn2 * rsqrt64(rn2);
        sh.grefa = grefa;
    }

    // neighbour j = lane (E_s and the triangles of Fig. 3b)
    float a = INFINITY;
    if (lane < 8) {
        SpNb nb;
        nb.invd = nb.d = nb.cx = nb.cy = nb.Px = nb.Py = nb.Pz = 0.0;
        nb.ok = 0;
        nb.w = 0.f;
        nb.fdx = nb.fdy = nb.finvd = nb.fd = 0.f;
        int dx, dy;
        ring_dir(lane, dx, dy);
        const int x = S.gx + dx, y = S.gy + dy;
        if (x >= 0 && y >= 0 && x < vd.GW && y < vd.GH) {
            const int j = vd.sp_base + y * vd.GW + x;
            if (__ldg(w.sp_cnt + j) > 0) {
                const float4 pj = planes_in[j];
                if (pj.x > 0.f && isfinite(pj.x)) {
                    nb.ok = 1;
                    const float4 cj = w.sp_col[j];
                    const float dr = cj.x - col.x, dg = cj.y - col.y, db = cj.z - col.z;
                    a = fmaf(dr, dr, fmaf(dg, dg, db * db)) * vd.k_col;
                    const double2 c2 = w.sp_cen[j];
                    nb.d = pj.x;
                    nb.invd = rcp64((double)pj.x);
                    nb.cx = c2.x;
                    nb.cy = c2.y;
                    nb.fdx = (float)(c2.x - cc.x);
                    nb.fdy = (float)(c2.y - cc.y);
                    nb.finvd = (float)nb.invd;
                    nb.fd = pj.x;
                    nb.Px = nb.d * (Ki[0] * c2.x + Ki[1] * c2.y + Ki[2]);
                    nb.Py = nb.d * (Ki[3] * c2.x + Ki[4] * c2.y + Ki[5]);
                    nb.Pz = nb.d * (Ki[6] * c2.x + Ki[7] * c2.y + Ki[8]);
                }
            }
        }
        sh.nb[lane] = nb;
    }
    float amin = a;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amin = fminf(amin, __shfl_xor_sync(0xffffffffu, amin, o));
    float wgt = (lane < 8 && a < INFINITY) ? ex2_approx(-(a - amin)) : 0.f;
    if (lane < 8) sh.nb[lane].w = wgt;
    wgt += __shfl_xor_sync(0xffffffffu, wgt, 4);
    wgt += __shfl_xor_sync(0xffffffffu, wgt, 2);
    wgt += __shfl_xor_sync(0xffffffffu, wgt, 1);
    S.sum_w = __shfl_sync(0xffffffffu, wgt, 0);
    const float cgain = vd.col_gain;             // the map colours carry the same factor
    S.cr = col.x * cgain; S.cg = col.y * cgain; S.cb = col.z * cgain;

    // neighbour view k = lane: homography pieces anchored at an integer pixel (FP64 -> FP32)
    if (lane < S.nnb) {
        const PairDev &pd = w.pairs[S.v * LFD_MAXN + lane];
        const double pr0 = pd.P[0] * S.ref.x + pd.P[1] * S.ref.y + pd.P[2];
        const double pr1 = pd.P[3] * S.ref.x + pd.P[4] * S.ref.y + pd.P[5];
        const double pr2 = pd.P[6] * S.ref.x + pd.P[7] * S.ref.y + pd.P[8];
        const double hx = fma(pd.q[0], grefa, pr0), hy = fma(pd.q[1], grefa, pr1), hw = fma(pd.q[2], grefa, pr2);
        double xa = 0.0, ya = 0.0;
        if (hw > 0.0) {
            const double ihw = rcp64(hw);
            xa = floor(hx * ihw);
            ya = floor(hy * ihw);
            xa = fmin(fmax(xa, -1048576.0), 1048576.0);
            ya = fmin(fmax(ya, -1048576.0), 1048576.0);
        }
        // rows scaled so that gp / Nw (or Nw / gp) carries sqrt(k_sig), see energy_sample
        const double rs = DOMAIN == 0 ? rcp64((double)vd.dep_gain) : (double)vd.dep_gain;
        SpView sv;
        sv.hw_a = (float)(hw * rs);
        sv.qw = (float)(pd.q[2] * rs);
        sv.Ex = (float)((hx - xa * hw) * rs);
        sv.Ey = (float)((hy - ya * hw) * rs);
        sv.Dx = (float)((pd.q[0] - xa * pd.q[2]) * rs);
        sv.Dy = (float)((pd.q[1] - ya * pd.q[2]) * rs);
        sv.Pp00 = (float)((pd.P[0] - xa * pd.P[6]) * rs);
        sv.Pp01 = (float)((pd.P[1] - xa * pd.P[7]) * rs);
        sv.Pp10 = (float)((pd.P[3] - ya * pd.P[6]) * rs);
        sv.Pp11 = (float)((pd.P[4] - ya * pd.P[7]) * rs);
        sv.P20 = (float)(pd.P[6] * rs);
        sv.P21 = (float)(pd.P[7] * rs);
        sv.xa_m = (int)xa - 0x4B400000;      // |xa| <= 2^20: no overflow
        sv.ya_m = (int)ya - 0x4B400000;
        sv.Wi = pd.Wi;
        sv.Hi = pd.Hi;
        sv.map = pd.map_i;
        sv.pad2 = 0;
        sh.view[lane] = sv;
    }

    // pixel offsets of the first 32*SLOTS_MAX pixels (zero past the last pixel)
#pragma unroll
    for (int jp = 0; jp < SLOTS_MAX / 2; jp++) {
        float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
        const int i0 = lane + 64 * jp, i1 = i0 + 32;
        if (i0 < S.n) {
            const unsigned pk = __ldg(w.sp_pix + S.off + i0);
            d.x = (float)((int)(pk & 0xffff) - S.ref.x);
            d.z = (float)((int)(pk >> 16) - S.ref.y);
        }
        if (i1 < S.n) {
            const unsigned pk = __ldg(w.sp_pix + S.off + i1);
            d.y = (float)((int)(pk & 0xffff) - S.ref.x);
            d.w = (float)((int)(pk >> 16) - S.ref.y);
        }
        sh.px4[32 * jp + lane] = d;
    }
    if (lane == 0) sh.S = S;
    __syncwarp();
    return true;
}

// Refinement candidate t (Fig. 3b): the normal of the triangle of the own
// centroid at depth dnew and ring neighbours t, t+1 at their depths, facing
// the camera; false for a missing vertex, a degenerate or a grazing
// triangle.  The plane goes to slot `slot` of the warp's CandShared.
template <int DOMAIN, bool COOP = false>
__device__ __noinline__ bool triangle_candidate(const ViewDev &vd, double dnew, double ignew, int t, int slot)
{
    const SpShared &sh = sp_shared<COOP>();
    CandShared &cs = g_cs[threadIdx.x >> 5];
    const SpNb &A = sh.nb[t];
    const SpNb &B = sh.nb[(t + 1) & 7];
    if (!A.ok || !B.ok) return false;
    const double P0x = dnew * sh.rx, P0y = dnew * sh.ry, P0z = dnew * sh.rz;
    const double e1x = A.Px - P0x, e1y = A.Py - P0y, e1z = A.Pz - P0z;
    const double e2x = B.Px - P0x, e2y = B.Py - P0y, e2z = B.Pz - P0z;
    double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    const double nn2 = nx * nx + ny * ny + nz * nz;
    const double l12 = (e1x * e1x + e1y * e1y + e1z * e1z) * (e2x * e2x + e2y * e2y + e2z * e2z);
    if (!(nn2 > 0.0 && nn2 >= 1e-24 * l12)) return false;               // |n| >= 1e-12 |e1| |e2|
    const double inn = rsqrt64(nn2);
    nx *= inn; ny *= inn; nz *= inn;
    if (nx * P0x + ny * P0y + nz * P0z > 0.0) { nx = -nx; ny = -ny; nz = -nz; }   // face the camera
    cs.nx[slot] = (float)nx; cs.ny[slot] = (float)ny; cs.nz[slot] = (float)nz;
    cs.ig[slot] = dnew;
    if (!(fabs(nx * sh.rx + ny * sh.ry + nz * sh.rz) >= 0.1 * sh.rn)) return false;   // not grazing
    double tg0 = 0, tg1 = 0, tg2 = 0;
    if (!plane_to_g(vd, dnew, nx, ny, nz, sh.cx, sh.cy, tg0, tg1, tg2)) return false;
    cand_store(cs, slot, hyp_prep<DOMAIN>(sh.S, sh, tg0, tg1, ignew));   // g . (c,1) = 1 / dnew
    return true;
}

// Perturbation sample k (flagged variant, not in the paper) of the plane
// (dnew, n) at iteration I into CandShared slot `slot`: depth scaled by
// 1 + r (2u - 1) and normal moved by r (2u - 1) per component, r =
// perturb_scale 2^(1 - I), draws from perturb_u; false when the depth leaves
// [d_min, d_max] or the plane is grazing.
template <int DOMAIN, bool COOP = false>
__device__ __noinline__ bool perturb_candidate(const ViewDev &vd, double dnew, double n0, double n1, double n2, int I,
                                               int k, int slot)
{
    const SpShared &sh = sp_shared<COOP>();
    CandShared &cs = g_cs[threadIdx.x >> 5];
    const double rad = ldexp(vd.perturb_scale, 1 - I);
    double u[4];
    for (int j = 0; j < 4; j++) u[j] = perturb_u(vd.seed, vd.lf_index, vd.lv, sh.S.s, I, 4 * k + j);
    const double dp = dnew * (1.0 + rad * (2.0 * u[0] - 1.0));
    double nx = n0 + rad * (2.0 * u[1] - 1.0), ny = n1 + rad * (2.0 * u[2] - 1.0), nz = n2 + rad * (2.0 * u[3] - 1.0);
    const double nn2 = nx * nx + ny * ny + nz * nz;
    if (!(nn2 > 0.0)) return false;
    const double inn = rsqrt64(nn2);
    nx *= inn; ny *= inn; nz *= inn;
    if (nx * sh.rx + ny * sh.ry + nz * sh.rz > 0.0) { nx = -nx; ny = -ny; nz = -nz; }   // face the camera
    const double ip = rcp64(dp);
    if (!(ip >= vd.inv_dmax && ip <= vd.inv_dmin)) return false;                      // d in [d_min, d_max]
    if (!(fabs(nx * sh.rx + ny * sh.ry + nz * sh.rz) >= 0.1 * sh.rn)) return false;   // not grazing
    double tg0 = 0, tg1 = 0, tg2 = 0;
    if (!plane_to_g(vd, dp, nx, ny, nz, sh.cx, sh.cy, tg0, tg1, tg2)) return false;
    cand_store(cs, slot, hyp_prep<DOMAIN>(sh.S, sh, tg0, tg1, ip));    // g . (c,1) = 1 / dp
    cs.nx[slot] = (float)nx; cs.ny[slot] = (float)ny; cs.nz[slot] = (float)nz;
    cs.ig[slot] = dp;
    return true;
}

// slots per lane for a superpixel of n pixels (the instantiated counts)
__device__ __forceinline__ int slot_class(int n)
{
    const int s = (n + 31) >> 5;
    return s <= 1 ? 1 : (s <= 8 ? s : SLOTS_MAX);
}

// ---------------------------------------------------------------------------
// propagation + refinement
// ---------------------------------------------------------------------------

// one Jacobi update of superpixel gs by one warp (iteration `iter`, 1-based),
// its pixels in SL slots per lane
template <int DOMAIN, int SL, bool AFF>
__device__ __noinline__ void propagate_sp(const Workspace &w, int iter, int gs, const float4 *planes_in,
                                          float4 *planes_out, int *choice, float *energy, int batch)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    SpShared &sh = g_sh[wid];
    CandShared &cs = g_cs[wid];
    const WarpSP &S = sh.S;                  // read from shared memory where used: nothing to spill
    const dbl4 gc = w.sp_g[gs];
    const ViewDev &vd = w.views[S.v];
    unsigned n_hyp = 0;
    float Ebest = -INFINITY;
    if (lane == 0) {
        sh.best_m = 0;
        sh.best_ig = 0.0;
    }

    // m = 0: the current plane; m >= 1: the propagation kernel (Eq. 4, Fig. 3a)
    const int ii = min(iter + vd.warm_off, LFD_MAX_ITER_INDEX);
    const int nr = w.radii_cnt[S.v * (LFD_MAX_ITER_INDEX + 1) + ii];
    const short *rad = w.radii + ((long long)S.v * (LFD_MAX_ITER_INDEX + 1) + ii) * LFD_MAX_RADII;
    const int M = 9 + 8 * nr;
    // candidates m = base .. base + batch - 1 (lane m - base), scored together
    for (int base = 0; base < M; base += batch) {
        const int m = base + lane;
        bool ok = false;
        double g0 = 0.0, g1 = 0.0, igc = 0.0;
        if (lane >= batch) {
        } else if (m == 0) {
            ok = gc.w != 0.0;
            g0 = gc.x; g1 = gc.y;
            igc = gc.x * sh.cx + gc.y * sh.cy + gc.z;
        } else if (m < M) {
            int dx, dy;
            if (m <= 8) {
                ring_dir(m - 1, dx, dy);
            } else {
                const int t = m - 9;
                const int r = rad[t >> 3];
                ring_dir(t & 7, dx, dy);
                dx *= r;
                dy *= r;
            }
            const int x = S.gx + dx, y = S.gy + dy;
            if (x >= 0 && y >= 0 && x < vd.GW && y < vd.GH) {
                const int j = vd.sp_base + y * vd.GW + x;
                if (__ldg(w.sp_cnt + j) > 0) {
                    const dbl4 gj = w.sp_g[j];
                    const double ig = gj.x * sh.cx + gj.y * sh.cy + gj.z;   // candidate's inverse depth at own centroid
                    ok = gj.w != 0.0 && ig > 0.0 && ig >= vd.inv_dmax && ig <= vd.inv_dmin;
                    const float4 pj = planes_in[j];
                    const double cosr = fabs(pj.y * sh.rx + pj.z * sh.ry + pj.w * sh.rz);
                    ok = ok && cosr >= 0.1 * sh.rn;                          // not grazing
                    g0 = gj.x; g1 = gj.y; igc = ig;
                    cs.ig[lane] = ig;
                    cs.nx[lane] = pj.y; cs.ny[lane] = pj.z; cs.nz[lane] = pj.w;
                }
            }
        }
        if (ok) cand_store(cs, lane, hyp_prep<DOMAIN>(S, sh, g0, g1, igc));
        cs.ec[lane] = 0.f;
        unsigned mask = __ballot_sync(0xffffffffu, ok);
        __syncwarp();
        if (mask) view_terms<DOMAIN, SL, false, false, AFF>(w, mask, nullptr);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const float E = cand_energy(sh, cs, S.nnb, src);
            n_hyp++;
            if (E > Ebest) {
                Ebest = E;
                if (lane == 0 && base + src > 0) {
                    sh.best_m = base + src;
                    sh.best_ig = cs.ig[src];
                    sh.bnx = cs.nx[src];
                    sh.bny = cs.ny[src];
                    sh.bnz = cs.nz[src];
                }
            }
        }
        __syncwarp();
    }
    const float Eprop = Ebest;
    const int best_m = sh.best_m;

    // refinement step: normals of the eight ring triangles (Fig. 3b)
    int best_t = -1;
    const double dnew = best_m > 0 ? rcp64(sh.best_ig) : (double)planes_in[gs].x;
    const double ignew = best_m > 0 ? sh.best_ig : rcp64(dnew);
    if (Ebest > -INFINITY && dnew > 0.0) {
        bool ok = false;
        if (lane < 8) {
            ok = triangle_candidate<DOMAIN>(vd, dnew, ignew, lane, lane);
        } else if (lane < 8 + vd.perturb_k) {           // flagged variant: random planes around (dnew, n)
            double n0, n1, n2;
            if (best_m > 0) {
                n0 = sh.bnx; n1 = sh.bny; n2 = sh.bnz;
            } else {
                const float4 cur = planes_in[gs];
                n0 = cur.y; n1 = cur.z; n2 = cur.w;
            }
            ok = perturb_candidate<DOMAIN>(vd, dnew, n0, n1, n2, ii, lane - 8, lane);
        }
        cs.ec[lane] = 0.f;
        unsigned mask = __ballot_sync(0xffffffffu, ok);
        __syncwarp();
        if (mask) view_terms<DOMAIN, SL, false, false, AFF>(w, mask, nullptr);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const float E = cand_energy(sh, cs, S.nnb, src);
            n_hyp++;
            if (E > Ebest) {
                Ebest = E;
                best_t = src;
                if (lane == 0) {
                    sh.bnx = cs.nx[src];
                    sh.bny = cs.ny[src];
                    sh.bnz = cs.nz[src];
                    sh.best_dep = cs.ig[src];
                }
            }
        }
    }
    if (lane == 0) {
        float4 out = planes_in[gs];
        if (best_t >= 0 || best_m > 0)
            out = make_float4((float)(best_t >= 0 ? sh.best_dep : dnew), sh.bnx, sh.bny, sh.bnz);
        planes_out[gs] = out;
        if (choice) { choice[2 * gs] = best_m; choice[2 * gs + 1] = best_t; }
        if (energy) { energy[2 * gs] = Eprop; energy[2 * gs + 1] = Ebest; }
        atomicAdd(&w.ctr->hyp, (unsigned long long)n_hyp);
        atomicAdd(&w.ctr->samples, (unsigned long long)n_hyp * S.n * S.nnb);
    }
}

// set-up and slot-count dispatch of one superpixel; each slot count is a
// separate (not inlined) function, so that every variant gets its own
// register allocation
template <int DOMAIN, bool AFF>
__device__ __forceinline__ void propagate_one(const Workspace &w, const Consts &c, int iter, int gs, int lane,
                                              const float4 *planes_in, float4 *planes_out, int *choice,
                                              float *energy)
{
    SpShared &sh = g_sh[threadIdx.x >> 5];
    {
        const ViewDev &vd0 = w.views[__ldg(w.sp_view + gs)];
        if (c.batch_iters && iter > vd0.iters) {   // this light field has finished: carry its plane through
            if (lane == 0) {
                planes_out[gs] = planes_in[gs];
                if (choice) { choice[2 * gs] = 0; choice[2 * gs + 1] = -1; }
                if (energy) { energy[2 * gs] = -INFINITY; energy[2 * gs + 1] = -INFINITY; }
            }
            return;
        }
    }
    const dbl4 gc = w.sp_g[gs];
    WarpSP S;
    if (!setup_sp<DOMAIN>(w, planes_in, gs, lane, S, sh, gc.w != 0.0, gc.x, gc.y, gc.z)) {
        if (lane == 0) {
            planes_out[gs] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (choice) { choice[2 * gs] = -1; choice[2 * gs + 1] = -1; }
            if (energy) { energy[2 * gs] = -INFINITY; energy[2 * gs + 1] = -INFINITY; }
        }
        return;
    }
    switch (slot_class(S.n)) {
    case 1: propagate_sp<DOMAIN, 1, AFF>(w, iter, gs, planes_in, planes_out, choice, energy, c.cand_batch); break;
    case 2: propagate_sp<DOMAIN, 2, AFF>(w, iter, gs, planes_in, planes_out, choice, energy, c.cand_batch); break;
    case 3: propagate_sp<DOMAIN, 3, AFF>(w, iter, gs, planes_in, planes_out, choice, energy, c.cand_batch); break;
    case 4: propagate_sp<DOMAIN, 4, AFF>(w, iter, gs, planes_in, planes_out, choice, energy, c.cand_batch); break;
    case 5: propagate_sp<DOMAIN, 5, AFF>(w, iter, gs, planes_in, planes_out, choice, energy, c.cand_batch); break;
    case 6: propagate_sp<DOMAIN, 6, AFF>(w, iter, gs, planes_in, planes_out, choice, energy, c.cand_batch); break;
    case 7: propagate_sp<DOMAIN, 7, AFF>(w, iter, gs, planes_in, planes_out, choice, energy, c.cand_batch); break;
    case 8: propagate_sp<DOMAIN, 8, AFF>(w, iter, gs, planes_in, planes_out, choice, energy, c.cand_batch); break;
    default: propagate_sp<DOMAIN, SLOTS_MAX, AFF>(w, iter, gs, planes_in, planes_out, choice, energy, c.cand_batch); break;
    }
}

// ---------------------------------------------------------------------------
// cooperative propagation: the CTA's 4 warps update one superpixel
// ---------------------------------------------------------------------------
//
// The same candidates, energies and choice as propagate_sp, split across the
// warps of the CTA: in rounds of up to 128 candidates every thread tests one
// candidate m, the valid ones are numbered in m order across the CTA and
// candidate c goes to warp c mod 4, batch slot c / 4; each warp scores its
// batch with view_terms, and the warps' winners are merged (highest energy,
// lowest m on ties: the first maximum in m order, as the sequential scan
// takes it).  The refinement candidates t go to warp t mod 4 the same way.
// Every candidate's energy is computed by one warp with the code of the
// per-warp form, so the results are the same bit for bit.  The point is
// locality: the warps of a CTA reproject one superpixel into the same
// neighbour view at the same time, so an SM's resident warps gather from 8
// footprints instead of 32 and the candidates reuse them from L1.
template <int DOMAIN, int SL, bool AFF>
__device__ __noinline__ void propagate_sp_coop(const Workspace &w, int iter, int gs, const float4 *planes_in,
                                               float4 *planes_out, int *choice, float *energy)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    SpShared &sh = g_shc[0];
    CandShared &cs = g_cs[wid];
    CoopShared &co = g_co;
    const WarpSP &S = sh.S;
    const dbl4 gc = w.sp_g[gs];
    const ViewDev &vd = w.views[S.v];
    unsigned n_hyp = 0;

    const int ii = min(iter + vd.warm_off, LFD_MAX_ITER_INDEX);
    const int nr = w.radii_cnt[S.v * (LFD_MAX_ITER_INDEX + 1) + ii];
    const short *rad = w.radii + ((long long)S.v * (LFD_MAX_ITER_INDEX + 1) + ii) * LFD_MAX_RADII;
    const int M = 9 + 8 * nr;
    float Ebest = -INFINITY;                 // this warp's best; its candidate in co.*[wid]
    if (lane == 0) co.m[wid] = -1;
    for (int base = 0; base < M; base += 32 * PROP_WARPS) {
        const int m = base + threadIdx.x;
        bool ok = false;
        double g0 = 0.0, g1 = 0.0, igc = 0.0;
        float nx = 0.f, ny = 0.f, nz = 0.f;
        if (m == 0) {
            ok = gc.w != 0.0;
            g0 = gc.x; g1 = gc.y;
            igc = gc.x * sh.cx + gc.y * sh.cy + gc.z;
        } else if (m < M) {
            int dx, dy;
            if (m <= 8) {
                ring_dir(m - 1, dx, dy);
            } else {
                const int t = m - 9;
                const int r = rad[t >> 3];
                ring_dir(t & 7, dx, dy);
                dx *= r;
                dy *= r;
            }
            const int x = S.gx + dx, y = S.gy + dy;
            if (x >= 0 && y >= 0 && x < vd.GW && y < vd.GH) {
                const int j = vd.sp_base + y * vd.GW + x;
                if (__ldg(w.sp_cnt + j) > 0) {
                    const dbl4 gj = w.sp_g[j];
                    const double ig = gj.x * sh.cx + gj.y * sh.cy + gj.z;   // candidate's inverse depth at own centroid
                    ok = gj.w != 0.0 && ig > 0.0 && ig >= vd.inv_dmax && ig <= vd.inv_dmin;
                    const float4 pj = planes_in[j];
                    const double cosr = fabs(pj.y * sh.rx + pj.z * sh.ry + pj.w * sh.rz);
                    ok = ok && cosr >= 0.1 * sh.rn;                          // not grazing
                    g0 = gj.x; g1 = gj.y; igc = ig;
                    nx = pj.y; ny = pj.z; nz = pj.w;
                }
            }
        }
        // number the valid candidates of the round in m order across the CTA
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) co.cnt[wid] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int k = 0; k < PROP_WARPS; k++) {
            const int ck = co.cnt[k];
            before += k < wid ? ck : 0;
            total += ck;
        }
        if (ok) {
            const int cidx = before + __popc(bal & ((1u << lane) - 1u));
            const int dw = cidx & (PROP_WARPS - 1), slot = cidx / PROP_WARPS;
            CandShared &dst = g_cs[dw];
            cand_store(dst, slot, hyp_prep<DOMAIN>(S, sh, g0, g1, igc));
            dst.ig[slot] = igc;
            dst.nx[slot] = nx; dst.ny[slot] = ny; dst.nz[slot] = nz;
            dst.ec[slot] = 0.f;
            co.mi[dw][slot] = m;
        }
        __syncthreads();
        const int nw = total > wid ? (total - wid + PROP_WARPS - 1) / PROP_WARPS : 0;
        unsigned mask = nw >= 32 ? 0xffffffffu : ((1u << nw) - 1u);
        if (mask) view_terms<DOMAIN, SL, false, false, AFF, true>(w, mask, nullptr);
        int sbest = -1;
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const float E = cand_energy(sh, cs, S.nnb, src);
            n_hyp++;
            if (E > Ebest) {
                Ebest = E;
                sbest = src;
            }
        }
        if (sbest >= 0 && lane == 0) {       // the round's winner of this warp: keep its plane
            co.E[wid] = Ebest;
            co.m[wid] = co.mi[wid][sbest];
            co.ig[wid] = cs.ig[sbest];
            co.nx[wid] = cs.nx[sbest]; co.ny[wid] = cs.ny[sbest]; co.nz[wid] = cs.nz[sbest];
        }
        __syncthreads();                     // the batches are refilled next round
    }
    // merge: highest energy, lowest m on ties
    float Eprop = -INFINITY;
    int wm = -1;
#pragma unroll
    for (int k = 0; k < PROP_WARPS; k++) {
        const float e = co.E[k];
        if (co.m[k] >= 0 && (wm < 0 || e > Eprop || (e == Eprop && co.m[k] < co.m[wm]))) {
            Eprop = e;
            wm = k;
        }
    }
    const int best_m = wm >= 0 ? co.m[wm] : 0;
    const double best_ig = wm >= 0 ? co.ig[wm] : 0.0;
    float pnx = 0.f, pny = 0.f, pnz = 0.f;
    if (best_m > 0) { pnx = co.nx[wm]; pny = co.ny[wm]; pnz = co.nz[wm]; }
    __syncthreads();                         // the records are reused by the refinement

    // refinement step: normals of the eight ring triangles (Fig. 3b), candidate t
    // in warp t mod 4, slot t / 4
    int best_t = -1;
    float Efinal = Eprop;
    double tdep = 0.0;
    float tnx = 0.f, tny = 0.f, tnz = 0.f;
    const double dnew = best_m > 0 ? rcp64(best_ig) : (double)planes_in[gs].x;
    const double ignew = best_m > 0 ? best_ig : rcp64(dnew);
    if (Eprop > -INFINITY && dnew > 0.0) {
        const int t = PROP_WARPS * lane + wid;
        bool ok = false;
        if (t < 8) {
            ok = triangle_candidate<DOMAIN, true>(vd, dnew, ignew, t, lane);
        } else if (t < 8 + vd.perturb_k) {   // flagged variant: random planes around (dnew, n)
            double n0, n1, n2;
            if (best_m > 0) {
                n0 = pnx; n1 = pny; n2 = pnz;
            } else {
                const float4 cur = planes_in[gs];
                n0 = cur.y; n1 = cur.z; n2 = cur.w;
            }
            ok = perturb_candidate<DOMAIN, true>(vd, dnew, n0, n1, n2, ii, t - 8, lane);
        }
        cs.ec[lane] = 0.f;
        unsigned mask = __ballot_sync(0xffffffffu, ok);
        __syncwarp();
        if (mask) view_terms<DOMAIN, SL, false, false, AFF, true>(w, mask, nullptr);
        float Et = -INFINITY;
        int st = -1;
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const float E = cand_energy(sh, cs, S.nnb, src);
            n_hyp++;
            if (E > Et) {
                Et = E;
                st = src;
            }
        }
        if (lane == 0) {
            co.E[wid] = Et;
            co.m[wid] = st >= 0 ? PROP_WARPS * st + wid : -1;
            co.ig[wid] = st >= 0 ? cs.ig[st] : 0.0;
            co.nx[wid] = st >= 0 ? cs.nx[st] : 0.f;
            co.ny[wid] = st >= 0 ? cs.ny[st] : 0.f;
            co.nz[wid] = st >= 0 ? cs.nz[st] : 0.f;
        }
        __syncthreads();
        // the refinement winner must beat the propagation's energy; lowest t on ties
        int wt = -1;
        float Emax = -INFINITY;
#pragma unroll
        for (int k = 0; k < PROP_WARPS; k++) {
            const float e = co.E[k];
            if (co.m[k] >= 0 && (wt < 0 || e > Emax || (e == Emax && co.m[k] < co.m[wt]))) {
                Emax = e;
                wt = k;
            }
        }
        if (wt >= 0 && Emax > Eprop) {
            best_t = co.m[wt];
            Efinal = Emax;
            tdep = co.ig[wt];
            tnx = co.nx[wt]; tny = co.ny[wt]; tnz = co.nz[wt];
        }
    }
    if (lane == 0) co.nh[wid] = n_hyp;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned nh = 0;
        for (int k = 0; k < PROP_WARPS; k++) nh += co.nh[k];
        float4 out = planes_in[gs];
        if (best_t >= 0)
            out = make_float4((float)tdep, tnx, tny, tnz);
        else if (best_m > 0)
            out = make_float4((float)dnew, pnx, pny, pnz);
        planes_out[gs] = out;
        if (choice) { choice[2 * gs] = best_m; choice[2 * gs + 1] = best_t; }
        if (energy) { energy[2 * gs] = Eprop; energy[2 * gs + 1] = Efinal; }
        atomicAdd(&w.ctr->hyp, (unsigned long long)nh);
        atomicAdd(&w.ctr->samples, (unsigned long long)nh * S.n * S.nnb);
    }
}

// set-up (by warp 0) and slot-count dispatch of one superpixel for the CTA
template <int DOMAIN, bool AFF>
__device__ __forceinline__ void propagate_one_coop(const Workspace &w, const Consts &c, int iter, int gs,
                                                   const float4 *planes_in, float4 *planes_out, int *choice,
                                                   float *energy)
{
    const int lane = threadIdx.x & 31;
    {
        const ViewDev &vd0 = w.views[__ldg(w.sp_view + gs)];
        if (c.batch_iters && iter > vd0.iters) {   // this light field has finished: carry its plane through
            if (threadIdx.x == 0) {
                planes_out[gs] = planes_in[gs];
                if (choice) { choice[2 * gs] = 0; choice[2 * gs + 1] = -1; }
                if (energy) { energy[2 * gs] = -INFINITY; energy[2 * gs + 1] = -INFINITY; }
            }
            return;
        }
    }
    SpShared &sh = g_shc[0];
    if (threadIdx.x < 32) {
        const dbl4 gc = w.sp_g[gs];
        WarpSP S;
        const bool ok = setup_sp<DOMAIN>(w, planes_in, gs, lane, S, sh, gc.w != 0.0, gc.x, gc.y, gc.z);
        if (lane == 0) g_co.ok = ok;
    }
    __syncthreads();
    if (!g_co.ok) {
        if (threadIdx.x == 0) {
            planes_out[gs] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (choice) { choice[2 * gs] = -1; choice[2 * gs + 1] = -1; }
            if (energy) { energy[2 * gs] = -INFINITY; energy[2 * gs + 1] = -INFINITY; }
        }
        return;
    }
    switch (slot_class(sh.S.n)) {
    case 1: propagate_sp_coop<DOMAIN, 1, AFF>(w, iter, gs, planes_in, planes_out, choice, energy); break;
    case 2: propagate_sp_coop<DOMAIN, 2, AFF>(w, iter, gs, planes_in, planes_out, choice, energy); break;
    case 3: propagate_sp_coop<DOMAIN, 3, AFF>(w, iter, gs, planes_in, planes_out, choice, energy); break;
    case 4: propagate_sp_coop<DOMAIN, 4, AFF>(w, iter, gs, planes_in, planes_out, choice, energy); break;
    case 5: propagate_sp_coop<DOMAIN, 5, AFF>(w, iter, gs, planes_in, planes_out, choice, energy); break;
    case 6: propagate_sp_coop<DOMAIN, 6, AFF>(w, iter, gs, planes_in, planes_out, choice, energy); break;
    case 7: propagate_sp_coop<DOMAIN, 7, AFF>(w, iter, gs, planes_in, planes_out, choice, energy); break;
    case 8: propagate_sp_coop<DOMAIN, 8, AFF>(w, iter, gs, planes_in, planes_out, choice, energy); break;
    default: propagate_sp_coop<DOMAIN, SLOTS_MAX, AFF>(w, iter, gs, planes_in, planes_out, choice, energy); break;
    }
}

// persistent CTAs: one superpixel per CTA at a time, from the cost-ordered queue
template <int DOMAIN, int MINB, bool AFF>
__global__ void __launch_bounds__(32 * PROP_WARPS, MINB) k_propagate_coop(const __grid_constant__ Workspace w, Consts c,
                                                                          int iter, const float4 *planes_in,
                                                                          float4 *planes_out, int *choice,
                                                                          float *energy)
{
    for (;;) {
        if (threadIdx.x == 0) g_co.item = atomicAdd(&w.queue[1], 1);
        __syncthreads();
        const int item = g_co.item;
        if (item >= w.S_total) break;
        propagate_one_coop<DOMAIN, AFF>(w, c, iter, __ldg(w.order + item), planes_in, planes_out, choice, energy);
        __syncthreads();                     // every thread is done with this superpixel's records
    }
}

template <int DOMAIN, int MINB, bool AFF>
__global__ void __launch_bounds__(32 * PROP_WARPS, MINB) k_propagate(const __grid_constant__ Workspace w, Consts c, int iter,
                                                                     const float4 *planes_in, float4 *planes_out,
                                                                     int *choice, float *energy)
{
    const int item = blockIdx.x * PROP_WARPS + (threadIdx.x >> 5);
    if (item >= w.S_total) return;
    propagate_one<DOMAIN, AFF>(w, c, iter, __ldg(w.order + item), threadIdx.x & 31, planes_in, planes_out, choice,
                               energy);
}

// persistent warps: superpixels taken from the cost-ordered queue, most expensive first
template <int DOMAIN, int MINB, bool AFF>
__global__ void __launch_bounds__(32 * PROP_WARPS, MINB) k_propagate_persistent(const __grid_constant__ Workspace w, Consts c, int iter,
                                                                                const float4 *planes_in,
                                                                                float4 *planes_out, int *choice,
                                                                                float *energy)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&w.queue[1], 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= w.S_total) break;
        propagate_one<DOMAIN, AFF>(w, c, iter, __ldg(w.order + item), lane, planes_in, planes_out, choice, energy);
        __syncwarp();
    }
}

template <int DOMAIN, int MINB, bool AFF>
static cudaError_t launch_propagate_t(const Workspace &w, const Consts &c, const LaunchCfg &lc, int iter,
                                      const float4 *planes_in, float4 *planes_out, int *choice, float *energy,
                                      cudaStream_t st)
{
    if (lc.prop_persistent && lc.prop_coop) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, k_propagate_coop<DOMAIN, MINB, AFF>, 32 * PROP_WARPS, 0);
        if (e != cudaSuccess) return e;
        const int grid = max(1, min(w.S_total, per_sm * lc.num_sms));
        k_propagate_coop<DOMAIN, MINB, AFF><<<grid, 32 * PROP_WARPS, 0, st>>>(w, c, iter, planes_in, planes_out,
                                                                              choice, energy);
    } else if (lc.prop_persistent) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, k_propagate_persistent<DOMAIN, MINB, AFF>, 32 * PROP_WARPS, 0);
        if (e != cudaSuccess) return e;
        const int warps = (w.S_total + PROP_WARPS - 1) / PROP_WARPS;
        const int grid = max(1, min(warps, per_sm * lc.num_sms));
        k_propagate_persistent<DOMAIN, MINB, AFF><<<grid, 32 * PROP_WARPS, 0, st>>>(w, c, iter, planes_in,
                                                                                    planes_out, choice, energy);
    } else {
        const int blocks = (w.S_total + PROP_WARPS - 1) / PROP_WARPS;
        k_propagate<DOMAIN, MINB, AFF><<<blocks, 32 * PROP_WARPS, 0, st>>>(w, c, iter, planes_in, planes_out, choice,
                                                                           energy);
    }
    return cudaGetLastError();
}

template <int DOMAIN, int MINB>
static cudaError_t launch_propagate_m(const Workspace &w, const Consts &c, const LaunchCfg &lc, int iter,
                                      const float4 *planes_in, float4 *planes_out, int *choice, float *energy,
                                      cudaStream_t st)
{
    return c.affine ? launch_propagate_t<DOMAIN, MINB, true>(w, c, lc, iter, planes_in, planes_out, choice, energy, st)
                    : launch_propagate_t<DOMAIN, MINB, false>(w, c, lc, iter, planes_in, planes_out, choice, energy,
                                                              st);
}

cudaError_t launch_propagate(const Workspace &w, const Consts &c0, const LaunchCfg &lc, int iter,
                             const float4 *planes_in, float4 *planes_out, int *choice, float *energy,
                             cudaStream_t st)
{
    Consts c = c0;
    c.cand_batch = lc.prop_batch == 16 ? 16 : 32;
    const bool eight = lc.prop_blocks >= 8;
    if (c.domain == 0)
        return eight ? launch_propagate_m<0, 8>(w, c, lc, iter, planes_in, planes_out, choice, energy, st)
                     : launch_propagate_m<0, 7>(w, c, lc, iter, planes_in, planes_out, choice, energy, st);
    return eight ? launch_propagate_m<1, 8>(w, c, lc, iter, planes_in, planes_out, choice, energy, st)
                 : launch_propagate_m<1, 7>(w, c, lc, iter, planes_in, planes_out, choice, energy, st);
}

// ---------------------------------------------------------------------------
// per-hypothesis terms (lfd_score)
// ---------------------------------------------------------------------------

template <int FMT, int DOMAIN>
__global__ void __launch_bounds__(128) k_score(const __grid_constant__ Workspace w, Consts c, const float4 *planes_state, int nq,
                                               const lfd_query *q, float *out)
{
    const int qi = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (qi >= nq) return;
    const lfd_query Q = q[qi];
    float *rec = out + (long long)qi * LFD_TERMS_STRIDE;
    if (lane < LFD_TERMS_STRIDE) rec[lane] = 0.f;
    if (lane + 32 < LFD_TERMS_STRIDE) rec[lane + 32] = 0.f;
    __syncwarp();
    const int gs = w.views[Q.view].sp_base + Q.sp;
    SpShared &sh = g_sh[threadIdx.x >> 5];
    const ViewDev &vd = w.views[Q.view];
    double g0, g1, g2;
    bool okp = false;
    if (__ldg(w.sp_cnt + gs) > 0) {
        const double2 cq = w.sp_cen[gs];
        okp = plane_to_g(vd, Q.d, Q.nx, Q.ny, Q.nz, cq.x, cq.y, g0, g1, g2);
    }
    if (!okp) {
        if (lane == 0) rec[0] = -INFINITY;
        return;
    }
    const dbl4 gc = w.sp_g[gs];
    WarpSP S;
    setup_sp<DOMAIN>(w, planes_state, gs, lane, S, sh, gc.w != 0.0, gc.x, gc.y, gc.z);
    __syncwarp();
    CandShared &cs = g_cs[threadIdx.x >> 5];
    cs.ec[lane] = 0.f;
    if (lane == 0) cand_store(cs, 0, hyp_prep<DOMAIN>(S, sh, g0, g1, g0 * sh.cx + g1 * sh.cy + g2));
    __syncwarp();
    view_terms<DOMAIN, SLOTS_MAX, true, true>(w, 1u, rec);
    if (lane == 0) {
        const float E = cand_energy(sh, cs, S.nnb, 0);
        rec[0] = E; rec[1] = cs.es[0]; rec[2] = S.nnb > 0 ? cs.ec[0] / (float)S.nnb : 0.f;
    }
    // truncated SSD sum of Eq. 2 for this plane (lanes over pixels)
    const double gref = g0 * S.ref.x + g1 * S.ref.y + g2;
    float tsum = 0.f;
    for (int k = 0; k < S.nnb; k++) {
        const PairDev &pd = w.pairs[S.v * LFD_MAXN + k];
        double pref[3], a[6];
        for (int r = 0; r < 3; r++) {
            pref[r] = pd.P[3 * r] * S.ref.x + pd.P[3 * r + 1] * S.ref.y + pd.P[3 * r + 2];
            a[2 * r] = fma(pd.q[r], g0, pd.P[3 * r]);
            a[2 * r + 1] = fma(pd.q[r], g1, pd.P[3 * r + 1]);
        }
        const float cx = (float)fma(pd.q[0], gref, pref[0]);
        const float cy = (float)fma(pd.q[1], gref, pref[1]);
        const float cw = (float)fma(pd.q[2], gref, pref[2]);
        const float a00 = (float)a[0], a01 = (float)a[1], a10 = (float)a[2], a11 = (float)a[3], a20 = (float)a[4],
                    a21 = (float)a[5];
        for (int i = lane; i < S.n; i += 32) {
            const unsigned pk = __ldg(w.sp_pix + S.off + i);
            const int x = pk & 0xffff, y = pk >> 16;
            const float du = (float)(x - S.ref.x), dv = (float)(y - S.ref.y);
            const float3 rc = texel_colour<FMT>(vd.quad, x, y, vd.W, vd.H);
            const float gp = (float)(g0 * x + g1 * y + g2);
            float t = vd.T;
            if (gp > 0.f) {
                const float X = fmaf(a00, du, fmaf(a01, dv, cx));
                const float Y = fmaf(a10, du, fmaf(a11, dv, cy));
                const float Wz = fmaf(a20, du, fmaf(a21, dv, cw));
                t = tssd_sample<FMT>(pd.quad_i, pd.Wi, pd.Hi, X, Y, Wz, rc, vd.T);
            }
            tsum += t;
        }
    }
    tsum = warp_sum(tsum);
    if (lane == 0) rec[3] = tsum * c.col_scale * c.col_scale;
}

cudaError_t launch_score(const Workspace &w, const Consts &c, const float4 *planes_state, int nq, const lfd_query *q,
                         float *out, cudaStream_t st)
{
    const int blocks = (nq + 3) / 4;
#define LFD_SCORE_CASE(F)                                                                                   \
    case F:                                                                                                 \
        if (c.domain == 0) k_score<F, 0><<<blocks, 128, 0, st>>>(w, c, planes_state, nq, q, out);           \
        else k_score<F, 1><<<blocks, 128, 0, st>>>(w, c, planes_state, nq, q, out);                         \
        break;
    switch (c.fmt) {
        LFD_SCORE_CASE(LFD_RGBA8)
        LFD_SCORE_CASE(LFD_RGBA_F16)
        LFD_SCORE_CASE(LFD_RGBA_BF16)
        LFD_SCORE_CASE(LFD_RGBA_F32)
    default: return cudaErrorInvalidValue;
    }
#undef LFD_SCORE_CASE
    return cudaGetLastError();
}

}  // namespace lfd
