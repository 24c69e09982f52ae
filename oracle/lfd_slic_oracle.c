/*
 * FP64 CPU oracle of SLIC superpixels (Achanta et al., TPAMI 2012), the
 * segmentation step that precedes the method of Chuchvara, Barsi and Gotchev
 * (arXiv 1812.06856, Section III-A; the paper runs a GPU SLIC).
 *
 * TEST INFRASTRUCTURE ONLY, like lfd_oracle.c: nothing in the product path may
 * include, link or call it, and it shares no code with the CUDA path.
 *
 * Readings (shared with the CUDA path):
 *  - colour space CIELAB (sRGB companding, D65 white) of the RGB values in
 *    [0,1];
 *  - seeds: one per cell of the grid_w x grid_h grid whose boundaries are at
 *    round(k W / grid_w) (round half up), seed position the cell centre
 *    ((x0 + x1 - 1) / 2, (y0 + y1 - 1) / 2) and seed colour the colour of the
 *    pixel floor(centre + 0.5); no gradient perturbation;
 *  - assignment: a pixel in grid cell (cx, cy) compares the centres of the
 *    3x3 cells around its own (present ones) by
 *    D^2 = |lab - lab_c|^2 + (m / S)^2 |xy - xy_c|^2, S = sqrt(W H / (GW GH));
 *    the smallest D^2 wins, ties to the first in row-major cell order;
 *  - update: each centre becomes the mean (Lab and xy) of its pixels; a centre
 *    without pixels keeps its value;
 *  - a fixed number of iterations, label = cy * grid_w + cx of the winning
 *    centre; no connectivity post-processing.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Flag margin of an assignment, derived from the FP32 arithmetic an
 * implementation may use.  Its CIELAB conversion of a pixel (sRGB power,
 * matrix, cube root: a few ulp on f in [0, 1], times 116, 500 and 200 in
 * L, a, b) leaves each Lab vector within SLIC_LAB_EPS of this FP64 value
 * (about 3e-5 in L, 2.1e-4 in a, 8e-5 in b for 4-ulp power and 1-ulp cube
 * root; rounded up).  A distance D^2 = |Lab - Lab_c|^2 + w |xy - xy_c|^2
 * then moves by at most 2 |Lab - Lab_c| eps + eps^2 <= 2 sqrt(D^2) eps + eps^2,
 * and the FP32 rounding of the sum adds at most 8 u D^2 (u = 2^-24).  Two
 * candidates can swap only when their gap is below the sum of both bounds;
 * such pixels are flagged. */
#define SLIC_LAB_EPS 4e-4
#define SLIC_U 5.9604644775390625e-08

static int slic_near_tie(double best, double second)
{
    if (!isfinite(second)) return 0;
    const double e = SLIC_LAB_EPS;
    return (second - best) <= 2.0 * e * (sqrt(best) + sqrt(second)) + 2.0 * e * e + 8.0 * SLIC_U * (best + second);
}

static double srgb_to_linear(double c)
{
    return c <= 0.04045 ? c / 12.92 : pow((c + 0.055) / 1.055, 2.4);
}

static double lab_f(double t)
{
    const double e = 216.0 / 24389.0, k = 24389.0 / 27.0;
    return t > e ? cbrt(t) : (k * t + 16.0) / 116.0;
}

/* RGB in [0,1] -> CIELAB (D65) */
void orc_rgb_to_lab(const double *rgb, double *lab)
{
    const double r = srgb_to_linear(rgb[0]), g = srgb_to_linear(rgb[1]), b = srgb_to_linear(rgb[2]);
    const double X = (0.4124564 * r + 0.3575761 * g + 0.1804375 * b) / 0.95047;
    const double Y = (0.2126729 * r + 0.7151522 * g + 0.0721750 * b) / 1.00000;
    const double Z = (0.0193339 * r + 0.1191920 * g + 0.9503041 * b) / 1.08883;
    const double fx = lab_f(X), fy = lab_f(Y), fz = lab_f(Z);
    lab[0] = 116.0 * fy - 16.0;
    lab[1] = 500.0 * (fx - fy);
    lab[2] = 200.0 * (fy - fz);
}

static int round_half_up(double x) { return (int)floor(x + 0.5); }

static void cell_bounds(int W, int GW, int *bx)
{
    for (int k = 0; k <= GW; k++) bx[k] = round_half_up((double)k * W / GW);
}

/* initial centres: 5 doubles per cell {L, a, b, x, y} */
void orc_slic_seeds(int32_t W, int32_t H, const double *rgb, int32_t GW, int32_t GH, double *centres)
{
    int *bx = (int *)malloc(sizeof(int) * (GW + 1)), *by = (int *)malloc(sizeof(int) * (GH + 1));
    cell_bounds(W, GW, bx);
    cell_bounds(H, GH, by);
    for (int cy = 0; cy < GH; cy++)
        for (int cx = 0; cx < GW; cx++) {
            double *c = centres + 5 * (size_t)(cy * GW + cx);
            const double x = 0.5 * (bx[cx] + bx[cx + 1] - 1), y = 0.5 * (by[cy] + by[cy + 1] - 1);
            int px = round_half_up(x), py = round_half_up(y);
            if (px > W - 1) px = W - 1;
            if (py > H - 1) py = H - 1;
            orc_rgb_to_lab(rgb + 3 * ((size_t)py * W + px), c);
            c[3] = x;
            c[4] = y;
        }
    free(bx);
    free(by);
}

/* one assignment step from `centres`; flags (nullable): 1 where the two
 * smallest distances are a near tie (slic_near_tie) */
void orc_slic_assign(int32_t W, int32_t H, const double *rgb, int32_t GW, int32_t GH, const double *centres,
                     double m, int32_t *labels, uint8_t *flags)
{
    int *bx = (int *)malloc(sizeof(int) * (GW + 1)), *by = (int *)malloc(sizeof(int) * (GH + 1));
    cell_bounds(W, GW, bx);
    cell_bounds(H, GH, by);
    const double S = sqrt((double)W * H / ((double)GW * GH)), w = (m / S) * (m / S);
    int cy = 0;
    for (int y = 0; y < H; y++) {
        while (y >= by[cy + 1]) cy++;
        int cx = 0;
        for (int x = 0; x < W; x++) {
            while (x >= bx[cx + 1]) cx++;
            double lab[3];
            orc_rgb_to_lab(rgb + 3 * ((size_t)y * W + x), lab);
            double best = INFINITY, second = INFINITY;
            int arg = -1;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const int ny = cy + dy, nx = cx + dx;
                    if (nx < 0 || ny < 0 || nx >= GW || ny >= GH) continue;
                    const double *c = centres + 5 * (size_t)(ny * GW + nx);
                    const double dl = lab[0] - c[0], da = lab[1] - c[1], db = lab[2] - c[2];
                    const double ddx = x - c[3], ddy = y - c[4];
                    const double D = dl * dl + da * da + db * db + w * (ddx * ddx + ddy * ddy);
                    if (D < best) {
                        second = best;
                        best = D;
                        arg = ny * GW + nx;
                    } else if (D < second) {
                        second = D;
                    }
                }
            labels[(size_t)y * W + x] = arg;
            if (flags) flags[(size_t)y * W + x] = (uint8_t)slic_near_tie(best, second);
        }
    }
    free(bx);
    free(by);
}

/* one update step: centres_out = mean {L, a, b, x, y} of each label's pixels
 * (centres_in where a label has none) */
void orc_slic_update(int32_t W, int32_t H, const double *rgb, int32_t GW, int32_t GH, const int32_t *labels,
                     const double *centres_in, double *centres_out)
{
    const size_t S = (size_t)GW * GH;
    double *acc = (double *)calloc(6 * S, sizeof(double));
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            const int l = labels[(size_t)y * W + x];
            if (l < 0 || (size_t)l >= S) continue;
            double lab[3];
            orc_rgb_to_lab(rgb + 3 * ((size_t)y * W + x), lab);
            double *a = acc + 6 * (size_t)l;
            a[0] += lab[0]; a[1] += lab[1]; a[2] += lab[2]; a[3] += x; a[4] += y; a[5] += 1.0;
        }
    for (size_t c = 0; c < S; c++) {
        const double *a = acc + 6 * c;
        for (int k = 0; k < 5; k++) centres_out[5 * c + k] = a[5] > 0 ? a[k] / a[5] : centres_in[5 * c + k];
    }
    free(acc);
}

/* full SLIC: seeds, then `iterations` x (assign, update), then a last assignment */
void orc_slic(int32_t W, int32_t H, const double *rgb, int32_t GW, int32_t GH, double m, int32_t iterations,
              int32_t *labels, double *centres_out)
{
    const size_t S = (size_t)GW * GH;
    double *c = (double *)malloc(sizeof(double) * 5 * S), *c2 = (double *)malloc(sizeof(double) * 5 * S);
    orc_slic_seeds(W, H, rgb, GW, GH, c);
    for (int it = 0; it < iterations; it++) {
        orc_slic_assign(W, H, rgb, GW, GH, c, m, labels, NULL);
        orc_slic_update(W, H, rgb, GW, GH, labels, c, c2);
        double *t = c; c = c2; c2 = t;
    }
    orc_slic_assign(W, H, rgb, GW, GH, c, m, labels, NULL);
    if (centres_out) memcpy(centres_out, c, sizeof(double) * 5 * S);
    free(c);
    free(c2);
}
