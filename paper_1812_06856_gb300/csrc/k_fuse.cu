// Stability-based depth fusion (Section III-D), one light field at a time.
//
// Every pixel of every view that carries a depth is lifted to a 3-D point and
// projected into each other view of its light field (nearest pixel, the
// refinement step's validity window); per (reference view, source view) the
// point of smallest depth wins a reference pixel through an integer atomicMin
// on the float bits (positive floats order as integers, so the result does
// not depend on the order of the atomics).  Then every reference pixel
// counts, for each of its depth candidates (its own depth and one per other
// view), the candidates agreeing within tau (relative) minus those that do
// not, and keeps the closest candidate whose count is not negative.
//
// Layout: zbuf holds, per reference view r of the light field, (V_l - 1)
// planes of its pixel count (source slot = i, or i - 1 past r), +inf bits
// where no point landed.  The per-pair projection is x_r ~ d M (x, y, 1) + e
// with M = K_r R_r R_i^T K_i^-1 and e = K_r (t_r - R_r R_i^T t_i), composed in
// FP64 on the host and applied in FP32; row 3 of K is (0, 0, 1), so the third
// component is the camera-r depth.
#include "lfd_internal.cuh"

namespace lfd {

constexpr int FUSE_MAXC = 32;     // candidates held in registers; more are re-read

__global__ void k_fuse_clear(unsigned *zbuf, long long n)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) zbuf[k] = 0x7f800000u;     // +inf
}

// one thread per source pixel; blockIdx.y = source view within the light field
__global__ void __launch_bounds__(256) k_fuse_project(FuseArgs a)
{
    const int i = blockIdx.y;
    const int W = a.W[i], H = a.H[i];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= W * H) return;
    const float d = __ldg(a.depth_in[i] + p);
    if (!(d > 0.f) || !isfinite(d)) return;
    const float x = (float)(p % W), y = (float)(p / W);
    for (int r = 0; r < a.V; r++) {
        if (r == i) continue;
        const float *m = a.mats + 12 * (i * a.V + r);
        const float X = fmaf(d, fmaf(m[0], x, fmaf(m[1], y, m[2])), m[9]);
        const float Y = fmaf(d, fmaf(m[3], x, fmaf(m[4], y, m[5])), m[10]);
        const float Z = fmaf(d, fmaf(m[6], x, fmaf(m[7], y, m[8])), m[11]);
        if (!(Z > 0.f)) continue;
        const float rz = 1.0f / Z;
        const float u = X * rz, v = Y * rz;
        const int Wr = a.W[r], Hr = a.H[r];
        if (!(u >= 0.f && u <= (float)(Wr - 1) && v >= 0.f && v <= (float)(Hr - 1))) continue;
        const int qx = (int)floorf(u + 0.5f), qy = (int)floorf(v + 0.5f);
        const int slot = i < r ? i : i - 1;
        unsigned *z = a.zbuf + a.zoff[r] + (long long)slot * Wr * Hr;
        atomicMin(z + (long long)qy * Wr + qx, __float_as_uint(Z));
    }
}

// one thread per reference pixel; blockIdx.y = reference view within the light field
__global__ void __launch_bounds__(256) k_fuse_select(FuseArgs a)
{
    const int r = blockIdx.y;
    const int W = a.W[r], H = a.H[r];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= W * H) return;
    const long long np = (long long)W * H;
    const unsigned *z = a.zbuf + a.zoff[r] + q;
    float c[FUSE_MAXC];
    int n = 0;
    const float own = __ldg(a.depth_in[r] + q);
    if (own > 0.f && isfinite(own)) c[n++] = own;
    const int ns = a.V - 1;
    if (ns + 1 <= FUSE_MAXC) {
        for (int k = 0; k < ns; k++) {
            const float zk = __uint_as_float(__ldg(z + k * np));
            if (isfinite(zk)) c[n++] = zk;
        }
        float best = 0.f;
        bool have = false;
        for (int s = 0; s < n; s++) {
            const float zc = c[s], lim = a.tau * zc;
            int stab = 0;
            for (int b = 0; b < n; b++)
                if (b != s) stab += fabsf(c[b] - zc) <= lim ? 1 : -1;
            if (stab >= 0 && (!have || zc < best)) {
                best = zc;
                have = true;
            }
        }
        a.depth_out[r][q] = have ? best : 0.f;
        return;
    }
    // many views: candidates re-read from the z-buffer (own depth is index -1)
    float best = 0.f;
    bool have = false;
    for (int s = -1; s < ns; s++) {
        const float zc = s < 0 ? own : __uint_as_float(__ldg(z + s * np));
        if (!(zc > 0.f) || !isfinite(zc)) continue;
        const float lim = a.tau * zc;
        int stab = 0;
        for (int b = -1; b < ns; b++) {
            if (b == s) continue;
            const float zb = b < 0 ? own : __uint_as_float(__ldg(z + b * np));
            if (!(zb > 0.f) || !isfinite(zb)) continue;
            stab += fabsf(zb - zc) <= lim ? 1 : -1;
        }
        if (stab >= 0 && (!have || zc < best)) {
            best = zc;
            have = true;
        }
    }
    a.depth_out[r][q] = have ? best : 0.f;
}

cudaError_t launch_fuse(const FuseArgs &a, long long zbuf_words, int max_px, cudaStream_t st)
{
    k_fuse_clear<<<(unsigned)((zbuf_words + 255) / 256), 256, 0, st>>>(a.zbuf, zbuf_words);
    dim3 grid((max_px + 255) / 256, a.V);
    k_fuse_project<<<grid, 256, 0, st>>>(a);
    k_fuse_select<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace lfd
