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
// Mapping: one warp per superpixel; lanes own pixels (8 per lane in
// registers, more streamed), so the gathers of a warp into a neighbour view's
// map fall in a compact footprint.  Hypotheses are scored one after another by
// the whole warp; per view the five sums are reduced with REDUX (counts) and
// butterfly shuffles (sums) in a fixed order, so results are deterministic.
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
constexpr int PM = 8;   // pixels per lane held in registers (256 per warp)

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
    g0 = (K[0] * nx + K[3] * ny + K[6] * nz) / rho;              // K^-T n / rho
    g1 = (K[1] * nx + K[4] * ny + K[7] * nz) / rho;
    g2 = (K[2] * nx + K[5] * ny + K[8] * nz) / rho;
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

__global__ void __launch_bounds__(128) k_rasterize(Workspace w, Consts c, OutPtrs depth, int has_depth)
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
    float4 *map = vd.map;
    float *dep = has_depth ? depth.p[v] : nullptr;
    for (int i = lane; i < n; i += 32) {
        const unsigned pk = __ldg(w.sp_pix + off + i);
        const int x = pk & 0xffff, y = pk >> 16;
        const float inv = fmaf(rc.y, (float)(x - ref.x), fmaf(rc.z, (float)(y - ref.y), rc.x));
        const bool ok = rc.w != 0.f && inv > 0.f && isfinite(inv);
        const float dv = ok ? (c.domain == 0 ? inv : 1.0f / inv) : 0.f;
        const long long p = (long long)y * vd.W + x;
        map[p] = make_float4(col.x, col.y, col.z, dv);
        if (dep) dep[p] = ok ? 1.0f / inv : 0.f;
    }
}

cudaError_t launch_rasterize(const Workspace &w, const Consts &c, const OutPtrs *depth, cudaStream_t st)
{
    OutPtrs none = {};
    const int blocks = (w.S_total + 3) / 4;
    k_rasterize<<<blocks, 128, 0, st>>>(w, c, depth ? *depth : none, depth ? 1 : 0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// energy evaluation shared by the propagation and score kernels
// ---------------------------------------------------------------------------

struct WarpSP {
    int gs, v, s, n, off, nnb, gx, gy;
    int2 ref;
    float cr, cg, cb, minw;
    double cx, cy;
    double rx, ry, rz, rn;       // own centroid ray K^-1 (c,1) and its length
    // neighbour j = lane (< 8) for E_s and the triangles of Fig. 3b
    bool nb_ok;
    float nb_w;                  // colour weight exp(-(a_j - min a))
    double nb_d, nb_invd, nb_cx, nb_cy;
    double Px, Py, Pz;           // neighbour centroid point d_j K^-1 (c_j,1)
    float sum_w;
    // neighbour view k = lane (< nnb)
    double pref0, pref1, pref2, q0, q1, q2;
    float P00, P01, P10, P11, P20, P21, q0f, q1f, q2f;
    int Wi, Hi;
    const float4 *map;
    // pixels of the first chunk
    float du[PM], dv[PM];
};

struct ViewK {
    float hw, a20, a21, cx, b0, b1, cy, c0, c1;
    int xi, yi, Wi, Hi;
    const float4 *map;
};

struct Acc {
    unsigned cnt, nx, ny;
    float sw, sg;
};

template <int DOMAIN>
__device__ __forceinline__ void energy_sample(const ViewK &K, float du, float dv, float gp, float cr, float cg, float cb,
                                              const Consts &c, Acc &a)
{
    if (!(gp > 0.f)) return;                                     // 3-D point not in front of camera v
    const float Nw = fmaf(K.a20, du, fmaf(K.a21, dv, K.hw));     // camera-i depth * g.p
    const float ex = fmaf(K.b0, du, fmaf(K.b1, dv, K.cx));
    const float ey = fmaf(K.c0, du, fmaf(K.c1, dv, K.cy));
    const float r = rcp_approx(Nw);
    const float fx = ex * r, fy = ey * r;                        // offsets from the integer anchor
    const bool ok = (Nw > 0.f) && (fx >= (float)(-K.xi)) && (fx <= (float)(K.Wi - 1 - K.xi)) &&
                    (fy >= (float)(-K.yi)) && (fy <= (float)(K.Hi - 1 - K.yi));
    if (!ok) return;
    const int ix = K.xi + __float2int_rd(fx + 0.5f);             // nearest pixel floor(x + 0.5)
    const int iy = K.yi + __float2int_rd(fy + 0.5f);
    const float4 t = __ldg(K.map + (long long)iy * K.Wi + ix);
    a.cnt++;
    const float dr = t.x - cr, dg = t.y - cg, db = t.z - cb;
    a.sw += ex2_approx(-fmaf(dr, dr, fmaf(dg, dg, db * db)) * c.k_col);    // Eq. 9 summand
    if (t.w > 0.f) {
        float val;
        bool inX;
        if (DOMAIN == 0) {
            val = gp * r;                                        // 1 / z_i(P)
            inX = val >= t.w * c.xy_lo;
        } else {
            val = Nw * rcp_approx(gp);                           // z_i(P)
            inX = val <= t.w * c.xy_hi;
        }
        if (inX) {
            const float dd = val - t.w;
            a.nx++;
            a.sg += ex2_approx(-dd * dd * c.k_sig);              // Eq. 10 summand
        } else {
            a.ny++;
        }
    }
}

// E(g) for the warp's superpixel; all lanes return the same value.  When
// `rec` is non-null lane 0 writes the terms record of lfd_score.
template <int DOMAIN>
__device__ float evaluate(const Workspace &w, const Consts &c, const WarpSP &S, double g0, double g1, double g2,
                          int lane, float *rec)
{
    const double gref = g0 * S.ref.x + g1 * S.ref.y + g2;
    const float g0f = (float)g0, g1f = (float)g1, grf = (float)gref;

    // ---- smoothness (Eq. 5-7) on lanes 0..7
    float num = 0.f;
    if (lane < 8 && S.nb_ok) {
        const double ext = g0 * S.nb_cx + g1 * S.nb_cy + g2;     // plane's inverse depth at c_j
        float dl;
        bool has = true;
        if (DOMAIN == 0) {
            dl = (float)(S.nb_invd - ext);
        } else {
            has = ext > 0.0;
            dl = has ? (float)(S.nb_d - 1.0 / ext) : 0.f;
        }
        num = has ? S.nb_w * ex2_approx(-dl * dl * c.k_sig) : 0.f;
    }
    num += __shfl_xor_sync(0xffffffffu, num, 4);
    num += __shfl_xor_sync(0xffffffffu, num, 2);
    num += __shfl_xor_sync(0xffffffffu, num, 1);
    num = __shfl_sync(0xffffffffu, num, 0);
    const float Es = S.sum_w > 0.f ? num / S.sum_w : 1.f;

    // ---- per neighbour-view anchored homography (lane k composes view k)
    ViewK mine;
    if (lane < S.nnb) {
        const double hx = fma(S.q0, gref, S.pref0);
        const double hy = fma(S.q1, gref, S.pref1);
        const double hw = fma(S.q2, gref, S.pref2);
        const float hwf = (float)hw;
        float xa = (float)hx / hwf, ya = (float)hy / hwf;
        xa = fminf(fmaxf(xa, -1048576.f), 1048576.f);
        ya = fminf(fmaxf(ya, -1048576.f), 1048576.f);
        int xi = __float2int_rd(xa), yi = __float2int_rd(ya);
        if (!(hwf == hwf)) { xi = 0; yi = 0; }
        mine.hw = hwf;
        mine.cx = (float)fma(-(double)xi, hw, hx);
        mine.cy = (float)fma(-(double)yi, hw, hy);
        const float a00 = fmaf(S.q0f, g0f, S.P00), a01 = fmaf(S.q0f, g1f, S.P01);
        const float a10 = fmaf(S.q1f, g0f, S.P10), a11 = fmaf(S.q1f, g1f, S.P11);
        mine.a20 = fmaf(S.q2f, g0f, S.P20);
        mine.a21 = fmaf(S.q2f, g1f, S.P21);
        mine.b0 = fmaf(-(float)xi, mine.a20, a00);
        mine.b1 = fmaf(-(float)xi, mine.a21, a01);
        mine.c0 = fmaf(-(float)yi, mine.a20, a10);
        mine.c1 = fmaf(-(float)yi, mine.a21, a11);
        mine.xi = xi;
        mine.yi = yi;
    }

    float gp[PM];
#pragma unroll
    for (int j = 0; j < PM; j++) gp[j] = fmaf(g0f, S.du[j], fmaf(g1f, S.dv[j], grf));

    float ec = 0.f;
    for (int k = 0; k < S.nnb; k++) {
        ViewK K;
        K.hw = __shfl_sync(0xffffffffu, mine.hw, k);
        K.a20 = __shfl_sync(0xffffffffu, mine.a20, k);
        K.a21 = __shfl_sync(0xffffffffu, mine.a21, k);
        K.cx = __shfl_sync(0xffffffffu, mine.cx, k);
        K.b0 = __shfl_sync(0xffffffffu, mine.b0, k);
        K.b1 = __shfl_sync(0xffffffffu, mine.b1, k);
        K.cy = __shfl_sync(0xffffffffu, mine.cy, k);
        K.c0 = __shfl_sync(0xffffffffu, mine.c0, k);
        K.c1 = __shfl_sync(0xffffffffu, mine.c1, k);
        K.xi = __shfl_sync(0xffffffffu, mine.xi, k);
        K.yi = __shfl_sync(0xffffffffu, mine.yi, k);
        K.Wi = __shfl_sync(0xffffffffu, S.Wi, k);
        K.Hi = __shfl_sync(0xffffffffu, S.Hi, k);
        K.map = (const float4 *)__shfl_sync(0xffffffffu, (unsigned long long)S.map, k);
        Acc a = {0u, 0u, 0u, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < PM; j++)
            if (lane + 32 * j < S.n) energy_sample<DOMAIN>(K, S.du[j], S.dv[j], gp[j], S.cr, S.cg, S.cb, c, a);
        for (int i = 32 * PM + lane; i < S.n; i += 32) {          // pixels beyond the register chunk
            const unsigned pk = __ldg(w.sp_pix + S.off + i);
            const float du = (float)((int)(pk & 0xffff) - S.ref.x), dv = (float)((int)(pk >> 16) - S.ref.y);
            energy_sample<DOMAIN>(K, du, dv, fmaf(g0f, du, fmaf(g1f, dv, grf)), S.cr, S.cg, S.cb, c, a);
        }
        const unsigned cnt = __reduce_add_sync(0xffffffffu, a.cnt);
        const unsigned nx = __reduce_add_sync(0xffffffffu, a.nx);
        const unsigned ny = __reduce_add_sync(0xffffffffu, a.ny);
        const float sw = warp_sum(a.sw), sg = warp_sum(a.sg);
        const float Si = cnt > 0 ? sw / (float)cnt : 0.f;                                  // Eq. 9
        const float Vi = (cnt > 0 && nx > 0) ? Si * (sg / (float)nx) : 0.f;                // Eq. 10
        const float Oi = (ny > 0 && (c.term_mask & 4)) ? c.eta * (1.f - S.minw) : 0.f;     // Eq. 11
        ec += Vi + Oi;
        if (rec && lane == 0) {
            float *r = rec + LFD_TERMS_HEAD + k * LFD_TERMS_PER_VIEW;
            r[0] = Si; r[1] = Vi; r[2] = Oi; r[3] = (float)cnt; r[4] = (float)nx; r[5] = (float)ny;
        }
    }
    const float Ec = S.nnb > 0 ? ec / (float)S.nnb : 0.f;                                  // Eq. 8
    const float E = ((c.term_mask & 2) ? Ec : 1.f) * ((c.term_mask & 1) ? Es : 1.f);      // Eq. 3
    if (rec && lane == 0) {
        rec[0] = E; rec[1] = Es; rec[2] = Ec;
    }
    return E;
}

// warp-wide set-up of the superpixel context; returns false for an empty superpixel
__device__ bool setup_sp(const Workspace &w, const Consts &c, const float4 *planes_in, int gs, int lane, WarpSP &S)
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
    S.cr = col.x; S.cg = col.y; S.cb = col.z; S.minw = col.w;
    const double2 cc = w.sp_cen[gs];
    S.cx = cc.x; S.cy = cc.y;
    const double *Ki = vd.Kinv;
    S.rx = Ki[0] * cc.x + Ki[1] * cc.y + Ki[2];
    S.ry = Ki[3] * cc.x + Ki[4] * cc.y + Ki[5];
    S.rz = Ki[6] * cc.x + Ki[7] * cc.y + Ki[8];
    S.rn = sqrt(S.rx * S.rx + S.ry * S.ry + S.rz * S.rz);

    // neighbour j = lane
    S.nb_ok = false;
    S.nb_w = 0.f;
    S.nb_d = S.nb_invd = S.nb_cx = S.nb_cy = 0.0;
    S.Px = S.Py = S.Pz = 0.0;
    float a = INFINITY;
    if (lane < 8) {
        int dx, dy;
        ring_dir(lane, dx, dy);
        const int x = S.gx + dx, y = S.gy + dy;
        if (x >= 0 && y >= 0 && x < vd.GW && y < vd.GH) {
            const int j = vd.sp_base + y * vd.GW + x;
            if (__ldg(w.sp_cnt + j) > 0) {
                const float4 pj = planes_in[j];
                if (pj.x > 0.f && isfinite(pj.x)) {
                    S.nb_ok = true;
                    const float4 cj = w.sp_col[j];
                    const float dr = cj.x - S.cr, dg = cj.y - S.cg, db = cj.z - S.cb;
                    a = fmaf(dr, dr, fmaf(dg, dg, db * db)) * c.k_col;
                    const double2 c2 = w.sp_cen[j];
                    S.nb_d = pj.x;
                    S.nb_invd = 1.0 / (double)pj.x;
                    S.nb_cx = c2.x;
                    S.nb_cy = c2.y;
                    const double rjx = Ki[0] * c2.x + Ki[1] * c2.y + Ki[2];
                    const double rjy = Ki[3] * c2.x + Ki[4] * c2.y + Ki[5];
                    const double rjz = Ki[6] * c2.x + Ki[7] * c2.y + Ki[8];
                    S.Px = S.nb_d * rjx; S.Py = S.nb_d * rjy; S.Pz = S.nb_d * rjz;
                }
            }
        }
    }
    float amin = a;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amin = fminf(amin, __shfl_xor_sync(0xffffffffu, amin, o));
    S.nb_w = S.nb_ok ? ex2_approx(-(a - amin)) : 0.f;
    float sw = S.nb_w;
    sw += __shfl_xor_sync(0xffffffffu, sw, 4);
    sw += __shfl_xor_sync(0xffffffffu, sw, 2);
    sw += __shfl_xor_sync(0xffffffffu, sw, 1);
    S.sum_w = __shfl_sync(0xffffffffu, sw, 0);

    // neighbour view k = lane
    S.map = nullptr;
    S.Wi = S.Hi = 0;
    S.pref0 = S.pref1 = S.pref2 = S.q0 = S.q1 = S.q2 = 0.0;
    S.P00 = S.P01 = S.P10 = S.P11 = S.P20 = S.P21 = S.q0f = S.q1f = S.q2f = 0.f;
    if (lane < S.nnb) {
        const PairDev &pd = w.pairs[S.v * LFD_MAXN + lane];
        S.pref0 = pd.P[0] * S.ref.x + pd.P[1] * S.ref.y + pd.P[2];
        S.pref1 = pd.P[3] * S.ref.x + pd.P[4] * S.ref.y + pd.P[5];
        S.pref2 = pd.P[6] * S.ref.x + pd.P[7] * S.ref.y + pd.P[8];
        S.q0 = pd.q[0]; S.q1 = pd.q[1]; S.q2 = pd.q[2];
        S.P00 = pd.Pf[0]; S.P01 = pd.Pf[1];
        S.P10 = pd.Pf[3]; S.P11 = pd.Pf[4];
        S.P20 = pd.Pf[6]; S.P21 = pd.Pf[7];
        S.q0f = pd.qf[0]; S.q1f = pd.qf[1]; S.q2f = pd.qf[2];
        S.Wi = pd.Wi; S.Hi = pd.Hi;
        S.map = pd.map_i;
    }

    // pixels of the register chunk
#pragma unroll
    for (int j = 0; j < PM; j++) {
        const int i = lane + 32 * j;
        if (i < S.n) {
            const unsigned pk = __ldg(w.sp_pix + S.off + i);
            S.du[j] = (float)((int)(pk & 0xffff) - S.ref.x);
            S.dv[j] = (float)((int)(pk >> 16) - S.ref.y);
        } else {
            S.du[j] = 0.f;
            S.dv[j] = 0.f;
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// propagation + refinement
// ---------------------------------------------------------------------------

template <int DOMAIN>
__global__ void __launch_bounds__(32 * PROP_WARPS) k_propagate(Workspace w, Consts c, int iter_eff,
                                                               const float4 *planes_in, float4 *planes_out,
                                                               int *choice, float *energy)
{
    const int gs = blockIdx.x * PROP_WARPS + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (gs >= w.S_total) return;
    WarpSP S;
    if (!setup_sp(w, c, planes_in, gs, lane, S)) {
        if (lane == 0) {
            planes_out[gs] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (choice) { choice[2 * gs] = -1; choice[2 * gs + 1] = -1; }
            if (energy) { energy[2 * gs] = -INFINITY; energy[2 * gs + 1] = -INFINITY; }
        }
        return;
    }
    const ViewDev &vd = w.views[S.v];
    unsigned long long n_hyp = 0;

    // current plane
    const float4 cur = planes_in[gs];
    const dbl4 gc = w.sp_g[gs];
    float Ebest = -INFINITY;
    if (gc.w != 0.0) {
        Ebest = evaluate<DOMAIN>(w, c, S, gc.x, gc.y, gc.z, lane, nullptr);
        n_hyp++;
    }
    int best_m = 0;
    double best_ig = 0.0;
    float bnx = cur.y, bny = cur.z, bnz = cur.w;

    // propagation step: candidate planes of the kernel (Eq. 4, Fig. 3a)
    const int ii = min(iter_eff, LFD_MAX_ITER_INDEX);
    const int nr = w.radii_cnt[S.v * (LFD_MAX_ITER_INDEX + 1) + ii];
    const short *rad = w.radii + ((long long)S.v * (LFD_MAX_ITER_INDEX + 1) + ii) * LFD_MAX_RADII;
    const int M = 9 + 8 * nr;
    for (int base = 1; base < M; base += 32) {
        const int m = base + lane;
        bool ok = m < M;
        double cg0 = 0, cg1 = 0, cg2 = 0, ig = 0;
        float cnx = 0, cny = 0, cnz = 0;
        if (ok) {
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
            ok = x >= 0 && y >= 0 && x < vd.GW && y < vd.GH;
            if (ok) {
                const int j = vd.sp_base + y * vd.GW + x;
                ok = __ldg(w.sp_cnt + j) > 0;
                if (ok) {
                    const dbl4 gj = w.sp_g[j];
                    ok = gj.w != 0.0;
                    cg0 = gj.x; cg1 = gj.y; cg2 = gj.z;
                    ig = cg0 * S.cx + cg1 * S.cy + cg2;              // candidate's inverse depth at own centroid
                    ok = ok && ig > 0.0 && ig >= c.inv_dmax && ig <= c.inv_dmin;
                    const float4 pj = planes_in[j];
                    cnx = pj.y; cny = pj.z; cnz = pj.w;
                    const double cosr = fabs(cnx * S.rx + cny * S.ry + cnz * S.rz) / S.rn;
                    ok = ok && cosr >= 0.1;                          // not grazing
                }
            }
        }
        unsigned mask = __ballot_sync(0xffffffffu, ok);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const double h0 = __shfl_sync(0xffffffffu, cg0, src);
            const double h1 = __shfl_sync(0xffffffffu, cg1, src);
            const double h2 = __shfl_sync(0xffffffffu, cg2, src);
            const float E = evaluate<DOMAIN>(w, c, S, h0, h1, h2, lane, nullptr);
            n_hyp++;
            if (E > Ebest) {
                Ebest = E;
                best_m = base + src;
                best_ig = __shfl_sync(0xffffffffu, ig, src);
                bnx = __shfl_sync(0xffffffffu, cnx, src);
                bny = __shfl_sync(0xffffffffu, cny, src);
                bnz = __shfl_sync(0xffffffffu, cnz, src);
            }
        }
    }
    const float Eprop = Ebest;

    // refinement step: normals of the eight ring triangles (Fig. 3b)
    int best_t = -1;
    double dnew = best_m > 0 ? 1.0 / best_ig : (double)cur.x;
    if (Ebest > -INFINITY && dnew > 0.0) {
        const double P0x = dnew * S.rx, P0y = dnew * S.ry, P0z = dnew * S.rz;
        const int nxt = (lane + 1) & 7;
        const double Qx = __shfl_sync(0xffffffffu, S.Px, nxt);
        const double Qy = __shfl_sync(0xffffffffu, S.Py, nxt);
        const double Qz = __shfl_sync(0xffffffffu, S.Pz, nxt);
        const bool ok_b = __shfl_sync(0xffffffffu, S.nb_ok, nxt);
        bool ok = lane < 8 && S.nb_ok && ok_b;
        double tg0 = 0, tg1 = 0, tg2 = 0;
        float tnx = 0, tny = 0, tnz = 0;
        if (ok) {
            const double e1x = S.Px - P0x, e1y = S.Py - P0y, e1z = S.Pz - P0z;
            const double e2x = Qx - P0x, e2y = Qy - P0y, e2z = Qz - P0z;
            double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
            const double nn = sqrt(nx * nx + ny * ny + nz * nz);
            const double l1 = sqrt(e1x * e1x + e1y * e1y + e1z * e1z), l2 = sqrt(e2x * e2x + e2y * e2y + e2z * e2z);
            ok = nn > 0.0 && nn >= 1e-12 * l1 * l2;
            if (ok) {
                nx /= nn; ny /= nn; nz /= nn;
                if (nx * P0x + ny * P0y + nz * P0z > 0.0) { nx = -nx; ny = -ny; nz = -nz; }   // face the camera
                ok = fabs(nx * S.rx + ny * S.ry + nz * S.rz) / S.rn >= 0.1;                  // not grazing
                if (ok) ok = plane_to_g(vd, dnew, nx, ny, nz, S.cx, S.cy, tg0, tg1, tg2);
                tnx = (float)nx; tny = (float)ny; tnz = (float)nz;
            }
        }
        unsigned mask = __ballot_sync(0xffffffffu, ok);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const double h0 = __shfl_sync(0xffffffffu, tg0, src);
            const double h1 = __shfl_sync(0xffffffffu, tg1, src);
            const double h2 = __shfl_sync(0xffffffffu, tg2, src);
            const float E = evaluate<DOMAIN>(w, c, S, h0, h1, h2, lane, nullptr);
            n_hyp++;
            if (E > Ebest) {
                Ebest = E;
                best_t = src;
                bnx = __shfl_sync(0xffffffffu, tnx, src);
                bny = __shfl_sync(0xffffffffu, tny, src);
                bnz = __shfl_sync(0xffffffffu, tnz, src);
            }
        }
    }
    if (lane == 0) {
        float4 out = cur;
        if (best_t >= 0 || best_m > 0) out = make_float4((float)dnew, bnx, bny, bnz);
        planes_out[gs] = out;
        if (choice) { choice[2 * gs] = best_m; choice[2 * gs + 1] = best_t; }
        if (energy) { energy[2 * gs] = Eprop; energy[2 * gs + 1] = Ebest; }
        atomicAdd(&w.ctr->hyp, n_hyp);
        atomicAdd(&w.ctr->samples, n_hyp * (unsigned long long)S.n * S.nnb);
    }
}

cudaError_t launch_propagate(const Workspace &w, const Consts &c, int iter_eff, const float4 *planes_in,
                             float4 *planes_out, int *choice, float *energy, cudaStream_t st)
{
    const int blocks = (w.S_total + PROP_WARPS - 1) / PROP_WARPS;
    if (c.domain == 0)
        k_propagate<0><<<blocks, 32 * PROP_WARPS, 0, st>>>(w, c, iter_eff, planes_in, planes_out, choice, energy);
    else
        k_propagate<1><<<blocks, 32 * PROP_WARPS, 0, st>>>(w, c, iter_eff, planes_in, planes_out, choice, energy);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// per-hypothesis terms (lfd_score)
// ---------------------------------------------------------------------------

template <int FMT, int DOMAIN>
__global__ void __launch_bounds__(128) k_score(Workspace w, Consts c, const float4 *planes_state, int nq,
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
    WarpSP S;
    if (!setup_sp(w, c, planes_state, gs, lane, S)) {
        if (lane == 0) rec[0] = -INFINITY;
        return;
    }
    const ViewDev &vd = w.views[S.v];
    double g0, g1, g2;
    if (!plane_to_g(vd, Q.d, Q.nx, Q.ny, Q.nz, S.cx, S.cy, g0, g1, g2)) {
        if (lane == 0) rec[0] = -INFINITY;
        return;
    }
    __syncwarp();
    evaluate<DOMAIN>(w, c, S, g0, g1, g2, lane, rec);
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
            const float3 rc = texel_colour<FMT>(vd.quad, (long long)y * vd.W + x);
            const float gp = (float)(g0 * x + g1 * y + g2);
            float t = c.T;
            if (gp > 0.f) {
                const float X = fmaf(a00, du, fmaf(a01, dv, cx));
                const float Y = fmaf(a10, du, fmaf(a11, dv, cy));
                const float Wz = fmaf(a20, du, fmaf(a21, dv, cw));
                t = tssd_sample<FMT>(pd.quad_i, pd.Wi, pd.Hi, X, Y, Wz, rc, c.T);
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
