/*
 * FP64 CPU oracle for the superpixel plane-sweep + parallel propagation depth
 * method of Chuchvara, Barsi and Gotchev, "Fast and Accurate Depth Estimation
 * from Sparse Light Fields" (arXiv 1812.06856), Section III.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file; it is used by tests/, by __graft_entry__.smoke() and by the
 * cpu_baseline / reference leg of bench.py.  It shares no code, header, table or
 * helper with the CUDA path: every geometric step (relative pose, projection,
 * plane-from-depth-and-normal, kernel offsets, neighbour views, jitter hash) is
 * written here a second time from its definition.
 *
 * Plain loops, double precision, the paper's order:
 *   view -> superpixel -> hypothesis -> neighbour view -> pixel.
 * Superpixels are processed in parallel with pthreads; this is legal because
 * every update reads only the previous iteration's state (Jacobi scheme,
 * Section III-E) and each superpixel's result is computed by one thread in a
 * fixed order, so the result does not depend on the thread count.
 *
 * Readings of points the paper leaves open (each one also a flag):
 *  - SSD of a pixel (Eq. 1): sum over R,G,B of squared differences, values in
 *    [0,1]; the superpixel is the patch.
 *  - sub-pixel sampling: a projection (x, y) lies in view i iff it is in
 *    front of both cameras and on the image's texture area,
 *    -1/2 <= x < W - 1/2 and -1/2 <= y < H - 1/2 (pixel centres at integers),
 *    i.e. iff its nearest pixel floor(x + 1/2), floor(y + 1/2) is a pixel of
 *    view i; TSSD samples bilinearly with the coordinates clamped to the
 *    outermost pixel centres (clamp to edge), Eq. 9/10 take that nearest
 *    pixel.  This is the domain of a texture sampled by GLSL, the paper's
 *    implementation (Section III-E).
 *  - out-of-view pixels: sweep adds T; refinement leaves them out of view i's
 *    sums; V_i = O_i = 0 when no pixel projects validly; V_i = 0 when X is
 *    empty; the 1/N of Eq. 8 counts every neighbour view.
 *  - neighbour views: the K = min(V-1, max) nearest camera centres.
 *  - sweep plane: fronto-parallel in the reference camera frame n = (0,0,-1)
 *    (flag: world frame).
 *  - jitter: one uniform sample per inverse-depth bin from splitmix64.
 *  - plane model: a 3-D plane in camera coordinates through d * K^-1 (c,1)
 *    with unit normal n; "interpolated/extrapolated depth" is that plane's
 *    depth along a pixel's ray.
 *  - energy is maximised; a candidate replaces the current plane only when its
 *    energy is strictly greater (first maximum in candidate order).
 *  - Gaussians of Eq. 6 and Eq. 10 in inverse depth by default (flag: metric),
 *    sigma = 2 x bin width; alpha = 0.1 on RGB in [0,1].
 *  - D(p) of Eq. 10 is the depth of the 3-D point in camera i; D(p^i) is view
 *    i's rasterised depth at the nearest pixel; pixels whose rasterised depth
 *    is invalid take part in neither X nor Y.
 *  - C^i of Eq. 9 is the mean colour of the view-i superpixel hit.
 *  - Eq. 11's minimum runs over the present 8-neighbours only (1 if none).
 *  - propagation kernel (Fig. 3a, Eq. 4) in superpixel grid cells; normal
 *    candidates from the 8 ring triangles (Fig. 3b).
 *  - candidate validity: interpolated depth inside [d_min, d_max] and not a
 *    grazing plane (|n . ray| >= 0.1).
 *
 * Margin flags: where a discrete decision (validity window, nearest-pixel
 * rounding, the X/Y split of Eq. 10/11, candidate validity) is within
 * `margin_px` pixels or `margin_rel` relative of its threshold, the oracle
 * marks the hypothesis, because an FP32 implementation may legitimately take
 * the other branch there.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 8

/* ------------------------------------------------------------------------ */
/* Public structures (mirrored by oracle/oracle.py with ctypes)             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t V;
    const int32_t *W, *H, *GW, *GH;   /* [V] */
    const double *K, *R, *t;           /* [V*9], [V*9], [V*3]; x_cam = R X + t */
    const double *rgb;                 /* concatenated views, each H*W*3 in [0,1] */
    const int32_t *labels;             /* concatenated views, each H*W */
    double d_min, d_max;
    int32_t L;
    double T, sigma, alpha, eta;
    int32_t kernel_size_init;          /* pixels; 0 => min(W,H) */
    double kernel_step_sp;             /* kernel step in superpixels (5) */
    int32_t max_neighbor_views;        /* 0 => 8 */
    int32_t depth_domain;              /* 0 inverse depth, 1 metric depth */
    int32_t jitter;                    /* 1 on, 0 => bin centres */
    int32_t term_mask;                 /* bit0 smoothness, bit1 consistency, bit2 occlusion */
    int32_t sweep_frame;               /* 0 camera, 1 world */
    uint64_t seed;
    int32_t lf_index;
    double xy_eps;                     /* relative tolerance of the X/Y split */
    int32_t warm_iter_offset;
    int32_t perturb_samples;           /* flagged variant: random plane samples per refinement (0 = off) */
    double perturb_scale;              /* their relative radius at I = 1, halved per iteration */
    int32_t threads;
    double margin_px, margin_rel;
} orc_input;

/* per-hypothesis terms.  *_lo / *_hi bound the value over every outcome an
 * implementation may legitimately reach at margin-flagged decisions; they
 * equal the nominal value when nothing is flagged. */
typedef struct {
    double E, Es, Ec, tssd;
    double E_lo, E_hi, Ec_lo, Ec_hi, tssd_lo, tssd_hi;
    double S[ORC_MAXN], Vt[ORC_MAXN], O[ORC_MAXN];
    double S_lo[ORC_MAXN], S_hi[ORC_MAXN], V_lo[ORC_MAXN], V_hi[ORC_MAXN], O_lo[ORC_MAXN], O_hi[ORC_MAXN];
    int32_t nvalid[ORC_MAXN], nx[ORC_MAXN], ny[ORC_MAXN], nflag[ORC_MAXN];
    int32_t nviews;
    int32_t flag_tssd, flag_energy;
} orc_terms;

typedef struct {
    int W, H, GW, GH, S;
    double K[9], Kinv[9], R[9], t[3], C[3];
    const double *rgb;
    const int32_t *lab;
    int sp_base;
    int64_t *cnt;
    int32_t *off, *pix;                /* CSR, row-major pixel order inside each superpixel */
    double *cen, *col, *minw;          /* [S*2], [S*3], [S] */
    int nnb;
    int nb[ORC_MAXN];
    double Rrel[ORC_MAXN][9], trel[ORC_MAXN][3];
    int ksize_init, ksteps_init;
} orc_view;

typedef struct {
    orc_input in;
    int V, S_total;
    orc_view *views;
    double delta;                      /* inverse-depth bin width */
    double sigma;                      /* Gaussian sigma in the chosen domain */
    /* state used by energy evaluation */
    const double *planes;              /* [S_total*4] */
    double **maps;                     /* per view H*W rasterised depth (domain), 0 invalid */
} orc_ctx;

/* ------------------------------------------------------------------------ */
/* small linear algebra                                                     */
/* ------------------------------------------------------------------------ */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static void matvec(const double *A, const double *x, double *y)
{
    for (int r = 0; r < 3; r++) y[r] = A[3 * r] * x[0] + A[3 * r + 1] * x[1] + A[3 * r + 2] * x[2];
}

static void matTvec(const double *A, const double *x, double *y)
{
    for (int c = 0; c < 3; c++) y[c] = A[c] * x[0] + A[3 + c] * x[1] + A[6 + c] * x[2];
}

static int inv3(const double *A, double *B)
{
    double c00 = A[4] * A[8] - A[5] * A[7];
    double c01 = A[5] * A[6] - A[3] * A[8];
    double c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(fabs(det) > 0.0) || !isfinite(det)) return 0;
    double id = 1.0 / det;
    B[0] = c00 * id;
    B[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    B[3] = c01 * id;
    B[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    B[6] = c02 * id;
    B[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* jitter: splitmix64 (Steele, Lea, Flood 2014)                            */
/* ------------------------------------------------------------------------ */

uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Uniform [0,1) offset of label k of superpixel s of view v (Section III-B):
 * key = ((lf * 2^12 + v) * 2^20 + s) * 2^12 + k  (mod 2^64). */
double orc_jitter_u(uint64_t seed, int32_t lf, int32_t v, int32_t s, int32_t k)
{
    uint64_t key = (((((uint64_t)lf << 12) + (uint64_t)v) << 20) + (uint64_t)s);
    key = (key << 12) + (uint64_t)k;
    return (double)(orc_splitmix64(seed ^ key) >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------ */
/* propagation kernel offsets (Fig. 3a, Eq. 4)                              */
/* ------------------------------------------------------------------------ */

static const int RING_DX[8] = {1, 1, 0, -1, -1, -1, 0, 1};   /* E NE N NW W SW S SE (y down) */
static const int RING_DY[8] = {0, -1, -1, -1, 0, 1, 1, 1};

/* Offsets of iteration I (1-based): the current superpixel (0,0), the eight
 * immediate neighbours, then along each of the eight compass rays the cells at
 * r_k = max(1, floor(k * Size_I / Steps_I + 0.5)), k = 1..Steps_I, with
 * Size_I = Size_init / I and Steps_I = max(1, floor(Steps_init / I)).  Repeats
 * are dropped keeping the first occurrence.  Writes dx,dy pairs; returns the
 * count (or the required count if cap is too small). */
int32_t orc_kernel_offsets(int32_t size_init, int32_t steps_init, int32_t I, int32_t *dxdy, int32_t cap)
{
    int n = 0;
    int32_t tmp[2 * 4096];
    tmp[0] = 0; tmp[1] = 0; n = 1;
    for (int d = 0; d < 8; d++) { tmp[2 * n] = RING_DX[d]; tmp[2 * n + 1] = RING_DY[d]; n++; }
    if (size_init >= 1 && I >= 1) {
        double size_I = (double)size_init / (double)I;
        int steps_I = steps_init / I;
        if (steps_I < 1) steps_I = 1;
        for (int k = 1; k <= steps_I; k++) {
            int r = (int)floor((double)k * size_I / (double)steps_I + 0.5);
            if (r < 1) r = 1;
            for (int d = 0; d < 8; d++) {
                int dx = RING_DX[d] * r, dy = RING_DY[d] * r, dup = 0;
                for (int m = 0; m < n; m++)
                    if (tmp[2 * m] == dx && tmp[2 * m + 1] == dy) { dup = 1; break; }
                if (!dup && n < 4096) { tmp[2 * n] = dx; tmp[2 * n + 1] = dy; n++; }
            }
        }
    }
    if (dxdy && n <= cap) memcpy(dxdy, tmp, sizeof(int32_t) * 2 * n);
    return n;
}

/* ------------------------------------------------------------------------ */
/* context                                                                  */
/* ------------------------------------------------------------------------ */

static double omega(const orc_ctx *c, const double *ca, const double *cb)
{
    double d0 = ca[0] - cb[0], d1 = ca[1] - cb[1], d2 = ca[2] - cb[2];
    double a = c->in.alpha;
    return exp(-(d0 * d0 + d1 * d1 + d2 * d2) / (2.0 * a * a));   /* Eq. 7 */
}

/* Neighbour views: the K nearest camera centres, nearer first; distances equal
 * within a relative 1e-9 keep the lower view index first. */
static void neighbour_views(orc_ctx *c)
{
    int V = c->V;
    int K = c->in.max_neighbor_views > 0 ? c->in.max_neighbor_views : ORC_MAXN;
    if (K > ORC_MAXN) K = ORC_MAXN;
    if (K > V - 1) K = V - 1;
    for (int v = 0; v < V; v++) {
        orc_view *w = &c->views[v];
        double dist[256];
        int used[256];
        for (int i = 0; i < V; i++) {
            double d[3] = {c->views[i].C[0] - w->C[0], c->views[i].C[1] - w->C[1], c->views[i].C[2] - w->C[2]};
            dist[i] = sqrt(dot3(d, d));
            used[i] = (i == v);
        }
        for (int r = 0; r < K; r++) {
            int best = -1;
            for (int i = 0; i < V; i++) {
                if (used[i]) continue;
                if (best < 0 || dist[i] < dist[best] * (1.0 - 1e-9)) best = i;
            }
            used[best] = 1;
            w->nb[r] = best;
        }
        w->nnb = K;
        for (int k = 0; k < K; k++) {
            const orc_view *wi = &c->views[w->nb[k]];
            /* R_rel = R_i R_v^T, t_rel = t_i - R_rel t_v */
            for (int r = 0; r < 3; r++)
                for (int q = 0; q < 3; q++) {
                    double s = 0;
                    for (int m = 0; m < 3; m++) s += wi->R[3 * r + m] * w->R[3 * q + m];
                    w->Rrel[k][3 * r + q] = s;
                }
            double rt[3];
            matvec(w->Rrel[k], w->t, rt);
            for (int r = 0; r < 3; r++) w->trel[k][r] = wi->t[r] - rt[r];
        }
    }
}

/* Superpixel statistics (Section III-A, III-C1): pixel lists, centroid, mean
 * colour, and the minimum colour similarity to the present 8-neighbours used
 * by the occlusion term (Eq. 11). */
static void superpixel_stats(orc_ctx *c, orc_view *w)
{
    int S = w->S, N = w->W * w->H;
    w->cnt = calloc(S, sizeof(int64_t));
    w->off = calloc(S + 1, sizeof(int32_t));
    w->pix = malloc(sizeof(int32_t) * (N > 0 ? N : 1));
    w->cen = calloc(2 * S, sizeof(double));
    w->col = calloc(3 * S, sizeof(double));
    w->minw = calloc(S, sizeof(double));
    for (int p = 0; p < N; p++) w->cnt[w->lab[p]]++;
    for (int s = 0; s < S; s++) w->off[s + 1] = w->off[s] + (int32_t)w->cnt[s];
    int32_t *fill = calloc(S, sizeof(int32_t));
    for (int p = 0; p < N; p++) {
        int s = w->lab[p];
        w->pix[w->off[s] + fill[s]++] = p;
        w->cen[2 * s] += (double)(p % w->W);
        w->cen[2 * s + 1] += (double)(p / w->W);
        for (int ch = 0; ch < 3; ch++) w->col[3 * s + ch] += w->rgb[3 * (size_t)p + ch];
    }
    free(fill);
    for (int s = 0; s < S; s++) {
        if (w->cnt[s] == 0) continue;
        w->cen[2 * s] /= (double)w->cnt[s];
        w->cen[2 * s + 1] /= (double)w->cnt[s];
        for (int ch = 0; ch < 3; ch++) w->col[3 * s + ch] /= (double)w->cnt[s];
    }
    for (int s = 0; s < S; s++) {
        int gx = s % w->GW, gy = s / w->GW;
        double m = 1.0;
        int any = 0;
        for (int d = 0; d < 8; d++) {
            int x = gx + RING_DX[d], y = gy + RING_DY[d];
            if (x < 0 || y < 0 || x >= w->GW || y >= w->GH) continue;
            int j = y * w->GW + x;
            if (w->cnt[j] == 0) continue;
            double om = omega(c, &w->col[3 * s], &w->col[3 * j]);
            if (!any || om < m) m = om;
            any = 1;
        }
        w->minw[s] = any ? m : 1.0;
    }
}

void *orc_create(const orc_input *in)
{
    if (!in || in->V < 2) return NULL;
    orc_ctx *c = calloc(1, sizeof(orc_ctx));
    c->in = *in;
    c->V = in->V;
    c->views = calloc(in->V, sizeof(orc_view));
    size_t px = 0;
    int sb = 0;
    for (int v = 0; v < in->V; v++) {
        orc_view *w = &c->views[v];
        w->W = in->W[v]; w->H = in->H[v]; w->GW = in->GW[v]; w->GH = in->GH[v];
        w->S = w->GW * w->GH;
        memcpy(w->K, in->K + 9 * v, sizeof(w->K));
        memcpy(w->R, in->R + 9 * v, sizeof(w->R));
        memcpy(w->t, in->t + 3 * v, sizeof(w->t));
        if (!inv3(w->K, w->Kinv)) { free(c->views); free(c); return NULL; }
        matTvec(w->R, w->t, w->C);                     /* C = -R^T t */
        for (int r = 0; r < 3; r++) w->C[r] = -w->C[r];
        w->rgb = in->rgb + 3 * px;
        w->lab = in->labels + px;
        w->sp_base = sb;
        px += (size_t)w->W * w->H;
        sb += w->S;
        superpixel_stats(c, w);
        double pitch = sqrt((double)w->W * w->H / ((double)w->GW * w->GH));
        int size_px = in->kernel_size_init > 0 ? in->kernel_size_init : (w->W < w->H ? w->W : w->H);
        w->ksize_init = (int)floor((double)size_px / pitch);
        w->ksteps_init = (int)floor((double)w->ksize_init / in->kernel_step_sp + 0.5);
    }
    c->S_total = sb;
    neighbour_views(c);
    c->delta = (1.0 / in->d_min - 1.0 / in->d_max) / (double)in->L;
    if (in->sigma > 0) c->sigma = in->sigma;
    else if (in->depth_domain == 0) c->sigma = 2.0 * c->delta;
    else c->sigma = 2.0 * (in->d_max - in->d_min) / (double)in->L;
    c->maps = calloc(in->V, sizeof(double *));
    for (int v = 0; v < in->V; v++) c->maps[v] = calloc((size_t)c->views[v].W * c->views[v].H, sizeof(double));
    return c;
}

void orc_destroy(void *h)
{
    orc_ctx *c = h;
    if (!c) return;
    for (int v = 0; v < c->V; v++) {
        orc_view *w = &c->views[v];
        free(w->cnt); free(w->off); free(w->pix); free(w->cen); free(w->col); free(w->minw);
        free(c->maps[v]);
    }
    free(c->maps);
    free(c->views);
    free(c);
}

/* accessors for tests */
int32_t orc_num_sp(void *h, int32_t v) { return ((orc_ctx *)h)->views[v].S; }
int32_t orc_sp_base(void *h, int32_t v) { return ((orc_ctx *)h)->views[v].sp_base; }
double orc_sigma(void *h) { return ((orc_ctx *)h)->sigma; }
double orc_delta(void *h) { return ((orc_ctx *)h)->delta; }

void orc_sp_stats(void *h, int32_t v, int64_t *cnt, double *cen, double *col, double *minw, int32_t *off, int32_t *pix)
{
    orc_view *w = &((orc_ctx *)h)->views[v];
    if (cnt) memcpy(cnt, w->cnt, sizeof(int64_t) * w->S);
    if (cen) memcpy(cen, w->cen, sizeof(double) * 2 * w->S);
    if (col) memcpy(col, w->col, sizeof(double) * 3 * w->S);
    if (minw) memcpy(minw, w->minw, sizeof(double) * w->S);
    if (off) memcpy(off, w->off, sizeof(int32_t) * (w->S + 1));
    if (pix) memcpy(pix, w->pix, sizeof(int32_t) * (size_t)w->W * w->H);
}

int32_t orc_neighbor_views(void *h, int32_t v, int32_t *out)
{
    orc_view *w = &((orc_ctx *)h)->views[v];
    for (int k = 0; k < w->nnb; k++) out[k] = w->nb[k];
    return w->nnb;
}

void orc_kernel_params(void *h, int32_t v, int32_t *size_init, int32_t *steps_init)
{
    orc_view *w = &((orc_ctx *)h)->views[v];
    *size_init = w->ksize_init;
    *steps_init = w->ksteps_init;
}

/* ------------------------------------------------------------------------ */
/* plane model (Section III-A, III-C)                                       */
/* ------------------------------------------------------------------------ */

/* The plane of a superpixel with centroid (cu,cv): it contains the point
 * X_c = d * K^-1 (cu,cv,1) and has unit normal n (camera frame).  Its inverse
 * depth along the ray of pixel p is g . (p,1) with g = K^-T n / (n . X_c).
 * Returns 0 when the plane is not usable (d <= 0, n . X_c == 0, non-finite). */
static int plane_g(const orc_view *w, double d, const double *n, double cu, double cv, double *g)
{
    if (!(d > 0) || !isfinite(d)) return 0;
    double p[3] = {cu, cv, 1.0}, ray[3], Xc[3];
    matvec(w->Kinv, p, ray);
    for (int r = 0; r < 3; r++) Xc[r] = d * ray[r];
    double rho = dot3(n, Xc);
    if (!(fabs(rho) > 0) || !isfinite(rho)) return 0;
    double kn[3];
    matTvec(w->Kinv, n, kn);
    for (int r = 0; r < 3; r++) g[r] = kn[r] / rho;
    return isfinite(g[0]) && isfinite(g[1]) && isfinite(g[2]);
}

/* depth of the plane along the ray of (u,v); 0 if the plane is behind/edge-on */
double orc_plane_depth(void *h, int32_t v, double d, double nx, double ny, double nz, double cu, double cv, double u, double vv)
{
    orc_ctx *c = h;
    double n[3] = {nx, ny, nz}, g[3];
    if (!plane_g(&c->views[v], d, n, cu, cv, g)) return 0.0;
    double ig = g[0] * u + g[1] * vv + g[2];
    if (!(ig > 0)) return 0.0;
    double D = 1.0 / ig;
    /* depth = z of the 3-D point D * K^-1 (u,v,1); K is pinhole so K^-1 row 3 = (0,0,1) */
    double p[3] = {u, vv, 1.0}, ray[3];
    matvec(c->views[v].Kinv, p, ray);
    return D * ray[2];
}

/* Projection of pixel (u,v) of view w, lying on the plane with inverse-depth
 * vector g, into the k-th neighbour view: 3-D point X = K^-1 (u,v,1) / (g.(u,v,1)),
 * X_i = R_rel X + t_rel, pixel = K_i X_i / z_i.  (The composition is the
 * plane-induced homography of Section III-B.) */
typedef struct { int front; double x, y, zi, gp; } proj_t;

static void project(const orc_ctx *c, const orc_view *w, int k, const double *g, double u, double v, proj_t *o)
{
    const orc_view *wi = &c->views[w->nb[k]];
    double p[3] = {u, v, 1.0}, ray[3], X[3], Xi[3], q[3];
    o->gp = dot3(g, p);
    o->front = 0;
    o->x = o->y = o->zi = 0;
    if (!(o->gp > 0)) return;
    matvec(w->Kinv, p, ray);
    double D = 1.0 / o->gp;
    for (int r = 0; r < 3; r++) X[r] = D * ray[r];
    matvec(w->Rrel[k], X, Xi);
    for (int r = 0; r < 3; r++) Xi[r] += w->trel[k][r];
    o->zi = Xi[2];
    if (!(o->zi > 0)) return;
    matvec(wi->K, Xi, q);
    o->x = q[0] / q[2];
    o->y = q[1] / q[2];
    o->front = 1;
}

int32_t orc_project_pixel(void *h, int32_t v, int32_t k, double d, double nx, double ny, double nz,
                          double cu, double cv, double u, double vv, double *out3)
{
    orc_ctx *c = h;
    orc_view *w = &c->views[v];
    double n[3] = {nx, ny, nz}, g[3];
    if (!plane_g(w, d, n, cu, cv, g)) return 0;
    proj_t pr;
    project(c, w, k, g, u, vv, &pr);
    out3[0] = pr.x; out3[1] = pr.y; out3[2] = pr.zi;
    return pr.front;
}

static int in_window(const orc_view *wi, double x, double y)
{
    return x >= -0.5 && x < (double)wi->W - 0.5 && y >= -0.5 && y < (double)wi->H - 0.5;
}

/* within `m` pixels of a window edge, so that FP32 could decide the other way */
static int near_window_edge(const orc_view *wi, double x, double y, double m)
{
    double x0 = -0.5, y0 = -0.5, x1 = (double)wi->W - 0.5, y1 = (double)wi->H - 0.5;
    int xin = x > x0 - m && x < x1 + m, yin = y > y0 - m && y < y1 + m;
    int xe = fabs(x - x0) < m || fabs(x - x1) < m;
    int ye = fabs(y - y0) < m || fabs(y - y1) < m;
    return (xe && yin) || (ye && xin);
}

/* bilinear interpolation of view colour at (x,y), the coordinates clamped to
 * [0, W-1] x [0, H-1] first (clamp to edge) */
static void bilinear(const orc_view *wi, double x, double y, double *out)
{
    x = x < 0.0 ? 0.0 : (x > (double)(wi->W - 1) ? (double)(wi->W - 1) : x);
    y = y < 0.0 ? 0.0 : (y > (double)(wi->H - 1) ? (double)(wi->H - 1) : y);
    int x0 = (int)floor(x), y0 = (int)floor(y);
    int x1 = x0 + 1 < wi->W ? x0 + 1 : wi->W - 1;
    int y1 = y0 + 1 < wi->H ? y0 + 1 : wi->H - 1;
    double fx = x - x0, fy = y - y0;
    const double *c00 = wi->rgb + 3 * ((size_t)y0 * wi->W + x0);
    const double *c10 = wi->rgb + 3 * ((size_t)y0 * wi->W + x1);
    const double *c01 = wi->rgb + 3 * ((size_t)y1 * wi->W + x0);
    const double *c11 = wi->rgb + 3 * ((size_t)y1 * wi->W + x1);
    for (int ch = 0; ch < 3; ch++)
        out[ch] = (1 - fy) * ((1 - fx) * c00[ch] + fx * c10[ch]) + fy * ((1 - fx) * c01[ch] + fx * c11[ch]);
}

void orc_bilinear_image(const double *rgb, int32_t W, int32_t H, double x, double y, double *out)
{
    orc_view w;
    memset(&w, 0, sizeof(w));
    w.rgb = rgb; w.W = W; w.H = H;
    bilinear(&w, x, y, out);
}

/* ------------------------------------------------------------------------ */
/* photo-consistency of the sweep: Eq. 1 and the inner sums of Eq. 2       */
/* ------------------------------------------------------------------------ */

/* truncated SSD between the reference pixel colour and view i sampled at (x,y) */
static double tssd_at(const orc_ctx *c, const orc_view *wi, const double *ref, double x, double y)
{
    double smp[3];
    bilinear(wi, x, y, smp);
    double ssd = 0;
    for (int ch = 0; ch < 3; ch++) ssd += (ref[ch] - smp[ch]) * (ref[ch] - smp[ch]);
    return ssd < c->in.T ? ssd : c->in.T;                                       /* Eq. 1 */
}

/* Sum over neighbour views and superpixel pixels of TSSD (inner sums of Eq. 2).
 * A projection that leaves view i or falls behind a camera costs T.  [lo,hi]
 * bound the sum over both outcomes of window decisions within margin_px. */
static double tssd_cost(const orc_ctx *c, const orc_view *w, int s, const double *g, int *flag, double *lo, double *hi)
{
    double cost = 0.0, clo = 0.0, chi = 0.0, T = c->in.T, m = c->in.margin_px;
    *flag = 0;
    for (int k = 0; k < w->nnb; k++) {
        const orc_view *wi = &c->views[w->nb[k]];
        for (int q = w->off[s]; q < w->off[s + 1]; q++) {
            int p = w->pix[q];
            double u = p % w->W, v = p / w->W;
            const double *ref = w->rgb + 3 * (size_t)p;
            proj_t pr;
            project(c, w, k, g, u, v, &pr);
            int valid = pr.front && in_window(wi, pr.x, pr.y);
            double nominal = valid ? tssd_at(c, wi, ref, pr.x, pr.y) : T;
            cost += nominal;
            if (pr.front && near_window_edge(wi, pr.x, pr.y, m)) {
                double alt = tssd_at(c, wi, ref, pr.x, pr.y);      /* sampled as if inside */
                clo += alt < T ? alt : T;
                chi += T;
                *flag = 1;
            } else {
                clo += nominal;
                chi += nominal;
            }
        }
    }
    if (lo) *lo = clo;
    if (hi) *hi = chi;
    return cost;
}

/* ------------------------------------------------------------------------ */
/* energy (Eq. 3 - 11)                                                      */
/* ------------------------------------------------------------------------ */

static int nearest(double x)   /* floor(x + 0.5) */
{
    return (int)floor(x + 0.5);
}

static double domain_value_of_inv(const orc_ctx *c, double inv)
{
    return c->in.depth_domain == 0 ? inv : 1.0 / inv;
}

/* outcome of one projected pixel sampled at (x,y) in view i */
typedef struct { int valid, inX, inY; double om, G; } outcome_t;

/* Eq. 9 and Eq. 10 summands for one pixel: validity, colour similarity of the
 * view-i superpixel hit at the nearest pixel, and the X/Y split against view
 * i's rasterised depth (force: -1 nominal comparison, 0 force Y, 1 force X). */
static void sample_outcome(const orc_ctx *c, const orc_view *wi, const double *map, const double *Cs,
                           double x, double y, double zval, int force, outcome_t *o)
{
    memset(o, 0, sizeof(*o));
    if (!in_window(wi, x, y)) return;
    int xi = nearest(x), yi = nearest(y);
    size_t pi = (size_t)yi * wi->W + xi;
    o->valid = 1;
    o->om = omega(c, Cs, &wi->col[3 * wi->lab[pi]]);
    double Di = map[pi];
    if (!(Di > 0)) return;
    double eps = c->in.xy_eps;
    int inX;
    if (force >= 0) inX = force;
    else if (c->in.depth_domain == 0) inX = zval >= Di / (1.0 + eps);   /* z_i <= D_i (1 + eps) */
    else inX = zval <= Di * (1.0 + eps);
    if (inX) {
        double dd = zval - Di;
        o->inX = 1;
        o->G = exp(-dd * dd / (2.0 * c->sigma * c->sigma));
    } else {
        o->inY = 1;
    }
}

/* E(g) for superpixel s of view w under the current state (planes + maps). */
static void energy(const orc_ctx *c, const orc_view *w, int s, const double *g, orc_terms *o)
{
    memset(o, 0, sizeof(*o));
    const double sig2 = 2.0 * c->sigma * c->sigma;
    const double *Cs = &w->col[3 * s];
    int gx = s % w->GW, gy = s / w->GW;
    double mpx = c->in.margin_px, mrel = c->in.margin_rel;

    /* smoothness, Eq. 5-7 */
    double num = 0, den = 0;
    for (int dI = 0; dI < 8; dI++) {
        int x = gx + RING_DX[dI], y = gy + RING_DY[dI];
        if (x < 0 || y < 0 || x >= w->GW || y >= w->GH) continue;
        int j = y * w->GW + x;
        if (w->cnt[j] == 0) continue;
        const double *pl = &c->planes[4 * (size_t)(w->sp_base + j)];
        if (!(pl[0] > 0)) continue;
        double wj = omega(c, Cs, &w->col[3 * j]);
        double ext = g[0] * w->cen[2 * j] + g[1] * w->cen[2 * j + 1] + g[2];   /* plane inverse depth at c_j */
        double sj;
        if (c->in.depth_domain == 0) {
            double dd = 1.0 / pl[0] - ext;
            sj = exp(-dd * dd / sig2);
        } else {
            if (ext > 0) { double dd = pl[0] - 1.0 / ext; sj = exp(-dd * dd / sig2); }
            else sj = 0.0;
        }
        num += wj * sj;
        den += wj;
    }
    o->Es = den > 0 ? num / den : 1.0;

    /* consistency, Eq. 8-11 */
    double ec = 0, ec_lo = 0, ec_hi = 0;
    o->nviews = w->nnb;
    double Oocc = (c->in.term_mask & 4) ? c->in.eta * (1.0 - w->minw[s]) : 0.0;
    for (int k = 0; k < w->nnb; k++) {
        const orc_view *wi = &c->views[w->nb[k]];
        const double *map = c->maps[w->nb[k]];
        /* nominal sums and their bounds over flagged alternatives */
        double nv = 0, sw = 0, nx = 0, sg = 0, ny = 0;
        double nv_l = 0, sw_l = 0, nx_l = 0, sg_l = 0, ny_l = 0;
        double nv_h = 0, sw_h = 0, nx_h = 0, sg_h = 0, ny_h = 0;
        int nflag = 0;
        for (int q = w->off[s]; q < w->off[s + 1]; q++) {
            int p = w->pix[q];
            double u = p % w->W, v = p / w->W;
            proj_t pr;
            project(c, w, k, g, u, v, &pr);
            if (!pr.front) continue;
            double zval = domain_value_of_inv(c, 1.0 / pr.zi);              /* D(p) in the domain */
            outcome_t o0;
            sample_outcome(c, wi, map, Cs, pr.x, pr.y, zval, -1, &o0);
            nv += o0.valid; sw += o0.om; nx += o0.inX; sg += o0.G; ny += o0.inY;
            /* flagged decisions: window edge, nearest-pixel rounding, X/Y split */
            double fxr = pr.x + 0.5 - floor(pr.x + 0.5), fyr = pr.y + 0.5 - floor(pr.y + 0.5);
            int fl = near_window_edge(wi, pr.x, pr.y, mpx) ||
                     (o0.valid && (fxr < mpx || fxr > 1 - mpx || fyr < mpx || fyr > 1 - mpx));
            double alts_x[5] = {pr.x, pr.x - mpx, pr.x + mpx, pr.x - mpx, pr.x + mpx};
            double alts_y[5] = {pr.y, pr.y - mpx, pr.y - mpx, pr.y + mpx, pr.y + mpx};
            int na = fl ? 5 : 1;
            double l[5] = {1e300, 1e300, 1e300, 1e300, 1e300}, h[5] = {-1e300, -1e300, -1e300, -1e300, -1e300};
            int any_flag = fl;
            for (int a = 0; a < na; a++) {
                outcome_t oa;
                sample_outcome(c, wi, map, Cs, alts_x[a], alts_y[a], zval, -1, &oa);
                outcome_t cand[3] = {oa, oa, oa};
                int nc = 1;
                if (oa.valid && (oa.inX || oa.inY)) {
                    int xi = nearest(alts_x[a]), yi = nearest(alts_y[a]);
                    double Di = map[(size_t)yi * wi->W + xi];
                    double thr = c->in.depth_domain == 0 ? Di / (1.0 + c->in.xy_eps) : Di * (1.0 + c->in.xy_eps);
                    if (fabs(zval - thr) <= mrel * Di) {
                        sample_outcome(c, wi, map, Cs, alts_x[a], alts_y[a], zval, 1, &cand[1]);
                        sample_outcome(c, wi, map, Cs, alts_x[a], alts_y[a], zval, 0, &cand[2]);
                        nc = 3;
                        any_flag = 1;
                    }
                }
                for (int ci = 0; ci < nc; ci++) {
                    double vals[5] = {cand[ci].valid, cand[ci].om, cand[ci].inX, cand[ci].G, cand[ci].inY};
                    for (int r = 0; r < 5; r++) {
                        if (vals[r] < l[r]) l[r] = vals[r];
                        if (vals[r] > h[r]) h[r] = vals[r];
                    }
                }
            }
            nflag += any_flag;
            nv_l += l[0]; sw_l += l[1]; nx_l += l[2]; sg_l += l[3]; ny_l += l[4];
            nv_h += h[0]; sw_h += h[1]; nx_h += h[2]; sg_h += h[3]; ny_h += h[4];
        }
        double S = nv > 0 ? sw / nv : 0.0;                                    /* Eq. 9 */
        double Vt = (nv > 0 && nx > 0) ? S * sg / nx : 0.0;                   /* Eq. 10 */
        double O = ny > 0 ? Oocc : 0.0;                                       /* Eq. 11 */
        /* interval bounds */
        double S_lo, S_hi, V_lo, V_hi, O_lo, O_hi;
        if (nv_h == 0) { S_lo = S_hi = 0; }
        else if (nv_l == 0) { S_lo = 0; S_hi = 1; }
        else { S_lo = sw_l / nv_h; S_hi = sw_h / nv_l; if (S_hi > 1) S_hi = 1; }
        if (nx_h == 0 || nv_h == 0) { V_lo = V_hi = 0; }
        else {
            double r_lo = (nx_l > 0) ? sg_l / nx_h : 0.0;
            double r_hi = (nx_l > 0) ? sg_h / nx_l : 1.0;
            if (r_hi > 1) r_hi = 1;
            V_lo = (nx_l > 0 && nv_l > 0) ? S_lo * r_lo : 0.0;
            V_hi = S_hi * r_hi;
        }
        O_lo = ny_l > 0 ? Oocc : 0.0;
        O_hi = ny_h > 0 ? Oocc : 0.0;
        if (Vt < V_lo) V_lo = Vt;
        if (Vt > V_hi) V_hi = Vt;
        if (S < S_lo) S_lo = S;
        if (S > S_hi) S_hi = S;
        o->S[k] = S; o->Vt[k] = Vt; o->O[k] = O;
        o->S_lo[k] = S_lo; o->S_hi[k] = S_hi; o->V_lo[k] = V_lo; o->V_hi[k] = V_hi; o->O_lo[k] = O_lo; o->O_hi[k] = O_hi;
        o->nvalid[k] = (int32_t)nv; o->nx[k] = (int32_t)nx; o->ny[k] = (int32_t)ny; o->nflag[k] = nflag;
        if (nflag) o->flag_energy = 1;
        ec += Vt + O;
        ec_lo += V_lo + O_lo;
        ec_hi += V_hi + O_hi;
    }
    double inv_n = w->nnb > 0 ? 1.0 / (double)w->nnb : 0.0;
    o->Ec = ec * inv_n;                                                        /* Eq. 8 */
    o->Ec_lo = ec_lo * inv_n;
    o->Ec_hi = ec_hi * inv_n;
    double Es = (c->in.term_mask & 1) ? o->Es : 1.0;
    int use_c = (c->in.term_mask & 2) != 0;
    o->E = (use_c ? o->Ec : 1.0) * Es;                                         /* Eq. 3 */
    o->E_lo = (use_c ? o->Ec_lo : 1.0) * Es;
    o->E_hi = (use_c ? o->Ec_hi : 1.0) * Es;
}

/* ------------------------------------------------------------------------ */
/* rasterisation: dense depth from superpixel planes                        */
/* ------------------------------------------------------------------------ */

static void rasterize_view(const orc_ctx *c, int v, const double *planes, double *map, double *depth)
{
    const orc_view *w = &c->views[v];
    for (int s = 0; s < w->S; s++) {
        const double *pl = &planes[4 * (size_t)(w->sp_base + s)];
        double g[3];
        int ok = w->cnt[s] > 0 && plane_g(w, pl[0], pl + 1, w->cen[2 * s], w->cen[2 * s + 1], g);
        for (int q = w->off[s]; q < w->off[s + 1]; q++) {
            int p = w->pix[q];
            double inv = ok ? g[0] * (p % w->W) + g[1] * (p / w->W) + g[2] : 0.0;
            int valid = ok && inv > 0 && isfinite(inv);
            if (map) map[p] = valid ? domain_value_of_inv(c, inv) : 0.0;
            if (depth) depth[p] = valid ? 1.0 / inv : 0.0;
        }
    }
}

void orc_rasterize(void *h, const double *planes, double *maps_out, double *depth_out)
{
    orc_ctx *c = h;
    size_t px = 0;
    for (int v = 0; v < c->V; v++) {
        size_t n = (size_t)c->views[v].W * c->views[v].H;
        rasterize_view(c, v, planes, maps_out ? maps_out + px : NULL, depth_out ? depth_out + px : NULL);
        px += n;
    }
}

static void set_state(orc_ctx *c, const double *planes)
{
    c->planes = planes;
    for (int v = 0; v < c->V; v++) rasterize_view(c, v, planes, c->maps[v], NULL);
}

/* ------------------------------------------------------------------------ */
/* work distribution over superpixels                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    orc_ctx *c;
    const int32_t *items;     /* global superpixel indices */
    int32_t n;
    int tid, nt;
    void (*fn)(orc_ctx *, int32_t, int32_t, void *);
    void *arg;
} job_t;

static void *job_run(void *p)
{
    job_t *j = p;
    for (int32_t i = j->tid; i < j->n; i += j->nt) j->fn(j->c, j->items[i], i, j->arg);
    return NULL;
}

static void for_items(orc_ctx *c, const int32_t *items, int32_t n, void (*fn)(orc_ctx *, int32_t, int32_t, void *), void *arg)
{
    int nt = c->in.threads > 0 ? c->in.threads : 1;
    if (nt > 256) nt = 256;
    if (nt == 1 || n < 2) {
        for (int32_t i = 0; i < n; i++) fn(c, items[i], i, arg);
        return;
    }
    pthread_t th[256];
    job_t jobs[256];
    for (int t = 0; t < nt; t++) {
        jobs[t] = (job_t){c, items, n, t, nt, fn, arg};
        pthread_create(&th[t], NULL, job_run, &jobs[t]);
    }
    for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
}

static void locate(const orc_ctx *c, int32_t gsp, int *v, int *s)
{
    int vv = 0;
    while (vv + 1 < c->V && c->views[vv + 1].sp_base <= gsp) vv++;
    *v = vv;
    *s = gsp - c->views[vv].sp_base;
}

/* ------------------------------------------------------------------------ */
/* plane sweep (Section III-B, Eq. 1-2)                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    double *planes_out;        /* [S_total*4] */
    int32_t *label_out;        /* per item */
    double *cost_out, *lo_out, *hi_out;   /* per item * L, may be NULL */
} sweep_arg;

static void sweep_normal(const orc_ctx *c, const orc_view *w, int s, double *n)
{
    if (c->in.sweep_frame == 0) { n[0] = 0; n[1] = 0; n[2] = -1; return; }
    double nw[3] = {0, 0, 1};
    matvec(w->R, nw, n);                              /* world z axis in camera frame */
    double p[3] = {w->cen[2 * s], w->cen[2 * s + 1], 1.0}, ray[3];
    matvec(w->Kinv, p, ray);
    if (dot3(n, ray) > 0) for (int r = 0; r < 3; r++) n[r] = -n[r];
}

static void sweep_one(orc_ctx *c, int32_t gsp, int32_t item, void *argp)
{
    sweep_arg *a = argp;
    int v, s;
    locate(c, gsp, &v, &s);
    const orc_view *w = &c->views[v];
    double *pl = &a->planes_out[4 * (size_t)gsp];
    if (w->cnt[s] == 0) {
        pl[0] = pl[1] = pl[2] = pl[3] = 0;
        if (a->label_out) a->label_out[item] = -1;
        return;
    }
    int L = c->in.L, best = -1;
    double best_cost = 0, best_d = 0, n[3];
    sweep_normal(c, w, s, n);
    for (int k = 0; k < L; k++) {
        double u = c->in.jitter ? orc_jitter_u(c->in.seed, c->in.lf_index, v, s, k) : 0.5;
        double z = 1.0 / c->in.d_max + ((double)k + u) * c->delta;       /* jittered inverse-depth level */
        double d = 1.0 / z, g[3], lo = INFINITY, hi = INFINITY;
        int flag = 0;
        double cost;
        if (plane_g(w, d, n, w->cen[2 * s], w->cen[2 * s + 1], g)) cost = tssd_cost(c, w, s, g, &flag, &lo, &hi);
        else cost = INFINITY;
        if (a->cost_out) a->cost_out[(size_t)item * L + k] = cost;
        if (a->lo_out) a->lo_out[(size_t)item * L + k] = lo;
        if (a->hi_out) a->hi_out[(size_t)item * L + k] = hi;
        if (best < 0 || cost < best_cost) { best = k; best_cost = cost; best_d = d; }   /* Eq. 2 */
    }
    pl[0] = best_d; pl[1] = n[0]; pl[2] = n[1]; pl[3] = n[2];
    if (a->label_out) a->label_out[item] = best;
}

/* items: global superpixel indices (NULL => all).  planes_out is the full
 * [S_total*4] array; only the listed superpixels are written. */
void orc_sweep(void *h, const int32_t *items, int32_t n_items, double *planes_out, int32_t *label_out,
               double *cost_out, double *lo_out, double *hi_out)
{
    orc_ctx *c = h;
    int32_t *all = NULL;
    if (!items) {
        all = malloc(sizeof(int32_t) * c->S_total);
        for (int i = 0; i < c->S_total; i++) all[i] = i;
        items = all;
        n_items = c->S_total;
    }
    sweep_arg a = {planes_out, label_out, cost_out, lo_out, hi_out};
    for_items(c, items, n_items, sweep_one, &a);
    free(all);
}

/* ------------------------------------------------------------------------ */
/* propagation + plane refinement (Section III-C, III-E)                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t iter;               /* 1-based */
    double *planes_out;         /* [S_total*4] */
    int32_t *choice_out;        /* per item * 2: propagation candidate, refinement triangle */
    double *energy_out;         /* per item * 2: E after propagation, E after refinement */
    int32_t *flag_out;          /* per item: 1 if a hypothesis was margin-flagged */
    double *cand_out;           /* per item * cand_cap * 3 (E, lo, hi), -inf if not evaluated */
    int32_t cand_cap;
    double *ref_out;            /* per item * 8 * 3 (E, lo, hi) of the refinement triangles */
} iter_arg;

static int grazing(const orc_view *w, const double *n, double cu, double cv, double mrel, int *flag)
{
    double p[3] = {cu, cv, 1.0}, ray[3];
    matvec(w->Kinv, p, ray);
    double rn = sqrt(dot3(ray, ray));
    double cs = fabs(dot3(n, ray)) / rn;
    if (fabs(cs - 0.1) <= mrel) *flag = 1;
    return cs < 0.1;
}

static void put3(double *dst, double E, double lo, double hi) { dst[0] = E; dst[1] = lo; dst[2] = hi; }

/* Refinement step (Section III-C, Fig. 3b): eight candidate normals, each the
 * normal of the triangle (own centroid point at depth dnew, centroid points of
 * two consecutive ring neighbours at their current depths).  Evaluates every
 * valid triangle; returns the first strictly better one (or -1). */
#define ORC_REF_MAX 32   /* refinement candidates: 8 triangles + up to 24 perturbation samples */

/* uniform [0,1) draw j of the perturbation variant for superpixel s of view v
 * at iteration I: SplitMix64 of a key of its own (seed xor "PERTURB1") */
static double perturb_u(uint64_t seed, int32_t lf, int32_t v, int32_t s, int32_t I, int32_t j)
{
    uint64_t key = ((((uint64_t)lf << 12) + (uint64_t)v) << 20) + (uint64_t)s;
    key = (key << 7) + (uint64_t)I;
    key = (key << 7) + (uint64_t)j;
    return (double)(orc_splitmix64((seed ^ 0x5045525455524231ULL) ^ key) >> 11) * (1.0 / 9007199254740992.0);
}

/* Refinement of superpixel s (Fig. 3b): the 8 ring-triangle normals at depth
 * dnew, then -- flagged variant, not in the paper -- perturbation_samples
 * random planes around (dnew, nbase) with a radius halving per iteration I;
 * the first strictly better candidate in this order wins. */
static int refine_step(const orc_ctx *c, const orc_view *w, int v, int s, double dnew, const double *nbase, int I,
                       double Ebase, double *keep, double *Eout, int *flag, double *ref_out)
{
    int gx = s % w->GW, gy = s / w->GW;
    double cu = w->cen[2 * s], cv = w->cen[2 * s + 1];
    double mrel = c->in.margin_rel;
    double p0[3] = {cu, cv, 1.0}, r0[3], P0[3];
    matvec(w->Kinv, p0, r0);
    for (int r = 0; r < 3; r++) P0[r] = dnew * r0[r];
    int nb_ok[8];
    double P[8][3];
    for (int dI = 0; dI < 8; dI++) {
        int x = gx + RING_DX[dI], y = gy + RING_DY[dI];
        nb_ok[dI] = 0;
        if (x < 0 || y < 0 || x >= w->GW || y >= w->GH) continue;
        int j = y * w->GW + x;
        if (w->cnt[j] == 0) continue;
        const double *pj = &c->planes[4 * (size_t)(w->sp_base + j)];
        if (!(pj[0] > 0)) continue;
        double pc[3] = {w->cen[2 * j], w->cen[2 * j + 1], 1.0}, rj[3];
        matvec(w->Kinv, pc, rj);
        for (int r = 0; r < 3; r++) P[dI][r] = pj[0] * rj[r];
        nb_ok[dI] = 1;
    }
    int choice = -1;
    double Ebest = Ebase;
    orc_terms t;
    for (int tI = 0; tI < 8; tI++) {
        if (ref_out) put3(ref_out + 3 * tI, -INFINITY, -INFINITY, -INFINITY);
        int a1 = tI, b1 = (tI + 1) % 8;
        if (!nb_ok[a1] || !nb_ok[b1]) continue;
        double e1[3], e2[3], n[3];
        for (int r = 0; r < 3; r++) { e1[r] = P[a1][r] - P0[r]; e2[r] = P[b1][r] - P0[r]; }
        cross3(e1, e2, n);
        double nn = sqrt(dot3(n, n));
        if (!(nn >= 1e-12 * sqrt(dot3(e1, e1)) * sqrt(dot3(e2, e2))) || nn == 0) continue;
        for (int r = 0; r < 3; r++) n[r] /= nn;
        if (dot3(n, P0) > 0) for (int r = 0; r < 3; r++) n[r] = -n[r];   /* face the camera */
        if (grazing(w, n, cu, cv, mrel, flag)) continue;
        double gt[3];
        if (!plane_g(w, dnew, n, cu, cv, gt)) continue;
        energy(c, w, s, gt, &t);
        if (t.flag_energy) *flag = 1;
        if (ref_out) put3(ref_out + 3 * tI, t.E, t.E_lo, t.E_hi);
        if (t.E > Ebest) {
            Ebest = t.E;
            choice = tI;
            keep[0] = dnew; keep[1] = n[0]; keep[2] = n[1]; keep[3] = n[2];
        }
    }
    const int K = c->in.perturb_samples;
    const double rad = ldexp(c->in.perturb_scale, 1 - I);
    for (int k = 0; k < K && 8 + k < ORC_REF_MAX; k++) {
        if (ref_out) put3(ref_out + 3 * (8 + k), -INFINITY, -INFINITY, -INFINITY);
        double u[4];
        for (int j = 0; j < 4; j++) u[j] = perturb_u(c->in.seed, c->in.lf_index, v, s, I, 4 * k + j);
        const double dp = dnew * (1.0 + rad * (2.0 * u[0] - 1.0));
        double n[3] = {nbase[0] + rad * (2.0 * u[1] - 1.0), nbase[1] + rad * (2.0 * u[2] - 1.0),
                       nbase[2] + rad * (2.0 * u[3] - 1.0)};
        const double nn = sqrt(dot3(n, n));
        if (!(nn > 0)) continue;
        for (int r = 0; r < 3; r++) n[r] /= nn;
        if (dot3(n, r0) > 0) for (int r = 0; r < 3; r++) n[r] = -n[r];      /* face the camera */
        if (fabs(dp - c->in.d_min) <= mrel * c->in.d_min || fabs(dp - c->in.d_max) <= mrel * c->in.d_max) *flag = 1;
        if (dp < c->in.d_min || dp > c->in.d_max) continue;
        if (grazing(w, n, cu, cv, mrel, flag)) continue;
        double gt[3];
        if (!plane_g(w, dp, n, cu, cv, gt)) continue;
        energy(c, w, s, gt, &t);
        if (t.flag_energy) *flag = 1;
        if (ref_out) put3(ref_out + 3 * (8 + k), t.E, t.E_lo, t.E_hi);
        if (t.E > Ebest) {
            Ebest = t.E;
            choice = 8 + k;
            keep[0] = dp; keep[1] = n[0]; keep[2] = n[1]; keep[3] = n[2];
        }
    }
    *Eout = Ebest;
    return choice;
}

static void iterate_one(orc_ctx *c, int32_t gsp, int32_t item, void *argp)
{
    iter_arg *a = argp;
    int v, s;
    locate(c, gsp, &v, &s);
    const orc_view *w = &c->views[v];
    const double *cur = &c->planes[4 * (size_t)gsp];
    double *out = &a->planes_out[4 * (size_t)gsp];
    int32_t ch0 = -1, ch1 = -1;
    double E0 = -INFINITY, E1 = -INFINITY;
    int flag = 0;
    double mrel = c->in.margin_rel;
    double *cand = a->cand_out ? a->cand_out + (size_t)item * a->cand_cap * 3 : NULL;
    double *refo = a->ref_out ? a->ref_out + (size_t)item * ORC_REF_MAX * 3 : NULL;
    if (cand) for (int m = 0; m < a->cand_cap; m++) put3(cand + 3 * m, -INFINITY, -INFINITY, -INFINITY);
    if (refo) for (int m = 0; m < ORC_REF_MAX; m++) put3(refo + 3 * m, -INFINITY, -INFINITY, -INFINITY);
    if (w->cnt[s] == 0) {
        out[0] = out[1] = out[2] = out[3] = 0;
        goto done;
    }
    double cu = w->cen[2 * s], cv = w->cen[2 * s + 1];
    double best[4] = {cur[0], cur[1], cur[2], cur[3]};
    double g[3];
    orc_terms t;
    ch0 = 0;
    if (plane_g(w, cur[0], cur + 1, cu, cv, g)) {
        energy(c, w, s, g, &t);
        E0 = t.E;
        flag |= t.flag_energy;
        if (cand && a->cand_cap > 0) put3(cand, t.E, t.E_lo, t.E_hi);
    }

    /* propagation step: planes of the kernel's superpixels (Eq. 4, Fig. 3a) */
    int32_t offs[2 * 4096];
    int I = a->iter + c->in.warm_iter_offset;
    int M = orc_kernel_offsets(w->ksize_init, w->ksteps_init, I, offs, 4096);
    int gx = s % w->GW, gy = s / w->GW;
    for (int m = 1; m < M; m++) {
        int x = gx + offs[2 * m], y = gy + offs[2 * m + 1];
        if (x < 0 || y < 0 || x >= w->GW || y >= w->GH) continue;
        int j = y * w->GW + x;
        if (w->cnt[j] == 0) continue;
        const double *pj = &c->planes[4 * (size_t)(w->sp_base + j)];
        double gj[3];
        if (!plane_g(w, pj[0], pj + 1, w->cen[2 * j], w->cen[2 * j + 1], gj)) continue;
        double ig = gj[0] * cu + gj[1] * cv + gj[2];          /* candidate plane at own centroid */
        if (!(ig > 0)) continue;
        double dhat = 1.0 / ig;                              /* d(d', n') of Section III-C */
        if (fabs(dhat - c->in.d_min) <= mrel * c->in.d_min || fabs(dhat - c->in.d_max) <= mrel * c->in.d_max) flag = 1;
        if (dhat < c->in.d_min || dhat > c->in.d_max) continue;
        if (grazing(w, pj + 1, cu, cv, mrel, &flag)) continue;
        energy(c, w, s, gj, &t);
        if (cand && m < a->cand_cap) put3(cand + 3 * m, t.E, t.E_lo, t.E_hi);
        flag |= t.flag_energy;
        if (t.E > E0) {                                      /* strict improvement */
            E0 = t.E;
            ch0 = m;
            best[0] = dhat; best[1] = pj[1]; best[2] = pj[2]; best[3] = pj[3];
        }
    }

    /* refinement step */
    E1 = E0;
    ch1 = -1;
    if (best[0] > 0 && E0 > -INFINITY) {
        double keep[4] = {best[0], best[1], best[2], best[3]};
        ch1 = refine_step(c, w, v, s, best[0], best + 1, I, E0, keep, &E1, &flag, refo);
        memcpy(best, keep, sizeof(keep));
    }
    memcpy(out, best, sizeof(best));
done:
    if (a->choice_out) { a->choice_out[2 * item] = ch0; a->choice_out[2 * item + 1] = ch1; }
    if (a->energy_out) { a->energy_out[2 * item] = E0; a->energy_out[2 * item + 1] = E1; }
    if (a->flag_out) a->flag_out[item] = flag;
}

/* One Jacobi iteration: every listed superpixel reads planes_in and the maps
 * rasterised from it, and writes its new plane into planes_out (full
 * [S_total*4] array; unlisted superpixels are copied through). */
void orc_iterate(void *h, int32_t iter, const double *planes_in, const int32_t *items, int32_t n_items,
                 double *planes_out, int32_t *choice_out, double *energy_out, int32_t *flag_out,
                 double *cand_out, int32_t cand_cap, double *ref_out)
{
    orc_ctx *c = h;
    set_state(c, planes_in);
    memcpy(planes_out, planes_in, sizeof(double) * 4 * (size_t)c->S_total);
    int32_t *all = NULL;
    if (!items) {
        all = malloc(sizeof(int32_t) * c->S_total);
        for (int i = 0; i < c->S_total; i++) all[i] = i;
        items = all;
        n_items = c->S_total;
    }
    iter_arg a = {iter, planes_out, choice_out, energy_out, flag_out, cand_out, cand_cap, ref_out};
    for_items(c, items, n_items, iterate_one, &a);
    free(all);
    c->planes = NULL;
}

/* Refinement candidates of one superpixel for a given post-propagation depth
 * (used to assess a divergent propagation choice).  out: 8*3 (E, lo, hi). */
int32_t orc_refine_candidates(void *h, const double *planes_state, int32_t gsp, double dnew, double nx, double ny,
                              double nz, int32_t iter, double *out)
{
    orc_ctx *c = h;
    set_state(c, planes_state);
    int v, s, flag = 0;
    locate(c, gsp, &v, &s);
    double keep[4] = {0, 0, 0, 0}, E;
    const double nb[3] = {nx, ny, nz};
    for (int m = 0; m < ORC_REF_MAX; m++) put3(out + 3 * m, -INFINITY, -INFINITY, -INFINITY);
    int r = refine_step(c, &c->views[v], v, s, dnew, nb, iter + c->in.warm_iter_offset, -INFINITY, keep, &E, &flag,
                        out);
    c->planes = NULL;
    (void)r;
    return flag;
}

/* ------------------------------------------------------------------------ */
/* per-hypothesis scoring                                                   */
/* ------------------------------------------------------------------------ */

typedef struct { int32_t view, sp; double d, nx, ny, nz; } orc_query;

typedef struct { const orc_query *q; orc_terms *out; } score_arg;

static void score_one(orc_ctx *c, int32_t unused, int32_t item, void *argp)
{
    (void)unused;
    score_arg *a = argp;
    const orc_query *q = &a->q[item];
    orc_terms *o = &a->out[item];
    memset(o, 0, sizeof(*o));
    const orc_view *w = &c->views[q->view];
    double n[3] = {q->nx, q->ny, q->nz}, g[3];
    if (w->cnt[q->sp] == 0 || !plane_g(w, q->d, n, w->cen[2 * q->sp], w->cen[2 * q->sp + 1], g)) {
        o->E = o->E_lo = o->E_hi = -INFINITY;
        return;
    }
    energy(c, w, q->sp, g, o);
    int f = 0;
    o->tssd = tssd_cost(c, w, q->sp, g, &f, &o->tssd_lo, &o->tssd_hi);
    o->flag_tssd = f;
}

void orc_score(void *h, const double *planes_state, const orc_query *q, int32_t nq, orc_terms *out)
{
    orc_ctx *c = h;
    set_state(c, planes_state);
    int32_t *idx = malloc(sizeof(int32_t) * (nq > 0 ? nq : 1));
    for (int i = 0; i < nq; i++) idx[i] = i;
    score_arg a = {q, out};
    for_items(c, idx, nq, score_one, &a);
    free(idx);
    c->planes = NULL;
}

int32_t orc_terms_size(void) { return (int32_t)sizeof(orc_terms); }
int32_t orc_query_size(void) { return (int32_t)sizeof(orc_query); }
int32_t orc_input_size(void) { return (int32_t)sizeof(orc_input); }
