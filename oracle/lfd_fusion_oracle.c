/*
 * FP64 CPU oracle of the stability-based depth fusion that ends the method of
 * Chuchvara, Barsi and Gotchev (arXiv 1812.06856), Section III-D.
 *
 * TEST INFRASTRUCTURE ONLY, like lfd_oracle.c: nothing in the product path may
 * include, link or call it, and it shares no code with the CUDA path.
 *
 * Each view in turn is the reference.  The pixels of every other view that
 * carry a depth are lifted to 3-D points and projected into the reference
 * camera; per reference pixel this gives one depth candidate per other view
 * (the nearest point of that view landing there) beside the reference's own
 * depth.  A candidate's stability is the number of other candidates that
 * agree with it minus the number that do not; the fused depth is the closest
 * candidate whose stability is not negative (0 when there is none).
 *
 * Readings of points Section III-D leaves open (shared with the CUDA path):
 *  - every other view is projected (not only the nearest ones);
 *  - a point lands on the nearest pixel floor(x + 0.5) of the reference, valid
 *    iff it is in front of the camera and 0 <= x <= W-1, 0 <= y <= H-1 before
 *    rounding (the window of the refinement step); per other view the point of
 *    smallest depth wins a pixel (z-buffer);
 *  - two depths agree when |z_a - z_c| <= tau * z_c, z_c the candidate whose
 *    stability is counted; tau is a parameter (default 0.01);
 *  - candidates are the reference's own depth when > 0 and one depth per
 *    other view where a point landed.
 *
 * Decisions within a margin of their threshold (the rounding boundary and
 * window edges of a projection, a z-buffer near-tie, an agreement test near
 * tau) flag the reference pixel; the FP32 GPU path may take either side there.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MARGIN_PX 1e-3     /* projected position within this of a rounding or window boundary */
#define MARGIN_REL 2e-5    /* relative margin of depth comparisons (z-buffer, agreement) */

static void mat3_inv(const double *A, double *B)
{
    const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    B[0] = c00 / det; B[3] = c01 / det; B[6] = c02 / det;
    B[1] = (A[2] * A[7] - A[1] * A[8]) / det; B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    B[2] = (A[1] * A[5] - A[2] * A[4]) / det; B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

static double frac_dist_half(double x)   /* distance of x to the nearest k + 0.5 */
{
    const double f = x - floor(x);
    return fabs(f - 0.5);
}

/*
 * V views; K, R, t: 9, 9, 3 doubles per view (x_cam = R X + t, pixel = K x / z);
 * W, H: sizes; depth: per view H*W doubles (0 = none); out: per view H*W
 * doubles; flags: per view H*W bytes (1 = a decision within its margin), may
 * be NULL.
 */
void orc_fuse(int32_t V, const double *K, const double *R, const double *t, const int32_t *W, const int32_t *H,
              const double *const *depth, double tau, double *const *out, uint8_t *const *flags)
{
    double *Kinv = (double *)malloc(sizeof(double) * 9 * V);
    for (int v = 0; v < V; v++) mat3_inv(K + 9 * v, Kinv + 9 * v);
    for (int r = 0; r < V; r++) {
        const int Wr = W[r], Hr = H[r];
        const size_t npx = (size_t)Wr * Hr;
        /* z-buffer per other view, and its flags */
        double *zb = (double *)malloc(sizeof(double) * npx * (V > 1 ? V - 1 : 1));
        uint8_t *fl = (uint8_t *)calloc(npx, 1);
        for (size_t k = 0; k < npx * (size_t)(V > 1 ? V - 1 : 1); k++) zb[k] = INFINITY;
        for (int i = 0, slot = 0; i < V; i++) {
            if (i == r) continue;
            double *z = zb + npx * (size_t)slot;
            slot++;
            const double *Ri = R + 9 * i, *ti = t + 3 * i, *Rr = R + 9 * r, *tr = t + 3 * r, *Kr = K + 9 * r;
            const double *Ki = Kinv + 9 * i;
            for (int y = 0; y < H[i]; y++)
                for (int x = 0; x < W[i]; x++) {
                    const double d = depth[i][(size_t)y * W[i] + x];
                    if (!(d > 0.0) || !isfinite(d)) continue;
                    /* camera-i point, world point, reference-camera point */
                    double ci[3], w[3], cr[3], pr[3];
                    for (int a = 0; a < 3; a++) ci[a] = d * (Ki[3 * a] * x + Ki[3 * a + 1] * y + Ki[3 * a + 2]);
                    for (int a = 0; a < 3; a++) {
                        const double s0 = ci[0] - ti[0], s1 = ci[1] - ti[1], s2 = ci[2] - ti[2];
                        w[a] = Ri[a] * s0 + Ri[3 + a] * s1 + Ri[6 + a] * s2;           /* R_i^T (c - t_i) */
                    }
                    for (int a = 0; a < 3; a++) cr[a] = Rr[3 * a] * w[0] + Rr[3 * a + 1] * w[1] + Rr[3 * a + 2] * w[2] + tr[a];
                    for (int a = 0; a < 3; a++) pr[a] = Kr[3 * a] * cr[0] + Kr[3 * a + 1] * cr[1] + Kr[3 * a + 2] * cr[2];
                    if (!(pr[2] > 0.0)) continue;
                    const double u = pr[0] / pr[2], vv = pr[1] / pr[2], zr = cr[2];
                    const int in = u >= 0.0 && u <= Wr - 1 && vv >= 0.0 && vv <= Hr - 1;
                    const int edge = fabs(u) < MARGIN_PX || fabs(u - (Wr - 1)) < MARGIN_PX || fabs(vv) < MARGIN_PX ||
                                     fabs(vv - (Hr - 1)) < MARGIN_PX;
                    const int rounding = frac_dist_half(u) < MARGIN_PX || frac_dist_half(vv) < MARGIN_PX;
                    const int qx = (int)floor(u + 0.5), qy = (int)floor(vv + 0.5);
                    if (edge || rounding) {
                        /* the point may land on q or, across an ambiguous rounding boundary,
                           on the neighbour on the other side of it; flag those pixels */
                        const int ax = frac_dist_half(u) < MARGIN_PX ? (u + 0.5 - qx < 0.5 ? qx - 1 : qx + 1) : qx;
                        const int ay = frac_dist_half(vv) < MARGIN_PX ? (vv + 0.5 - qy < 0.5 ? qy - 1 : qy + 1) : qy;
                        const int xs[2] = {qx, ax}, ys[2] = {qy, ay};
                        for (int b = 0; b < 2; b++)
                            for (int c = 0; c < 2; c++) {
                                const int px = xs[b], py = ys[c];
                                if (px >= 0 && py >= 0 && px < Wr && py < Hr) fl[(size_t)py * Wr + px] = 1;
                            }
                    }
                    if (!in) continue;
                    const size_t q = (size_t)qy * Wr + qx;
                    if (isfinite(z[q]) && fabs(zr - z[q]) <= MARGIN_REL * zr) fl[q] = 1;   /* z-buffer near-tie */
                    if (zr < z[q]) z[q] = zr;
                }
        }
        /* stability and choice per reference pixel */
        double *cand = (double *)malloc(sizeof(double) * (size_t)V);
        for (size_t q = 0; q < npx; q++) {
            int n = 0;
            const double own = depth[r][q];
            if (own > 0.0 && isfinite(own)) cand[n++] = own;
            for (int k = 0; k < V - 1; k++)
                if (isfinite(zb[npx * (size_t)k + q])) cand[n++] = zb[npx * (size_t)k + q];
            double best = 0.0;
            int have = 0;
            for (int a = 0; a < n; a++) {
                const double zc = cand[a];
                int stab = 0;
                for (int b = 0; b < n; b++) {
                    if (b == a) continue;
                    const double dz = fabs(cand[b] - zc), lim = tau * zc;
                    if (fabs(dz - lim) <= MARGIN_REL * zc) fl[q] = 1;
                    stab += dz <= lim ? 1 : -1;
                }
                if (stab >= 0 && (!have || zc < best)) {
                    best = zc;
                    have = 1;
                }
            }
            out[r][q] = have ? best : 0.0;
        }
        if (flags) memcpy(flags[r], fl, npx);
        free(cand);
        free(fl);
        free(zb);
    }
    free(Kinv);
}
