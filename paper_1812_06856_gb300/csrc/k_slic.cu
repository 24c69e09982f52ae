// SLIC superpixels on the GPU (Achanta et al. 2012; the segmentation step the
// method runs before Section III-A), with the grid-indexed labels the rest of
// the path expects (label = cell_y * grid_w + cell_x of the winning centre).
//
// Colour space CIELAB (sRGB companding, D65 white); seeds at the centres of
// the grid cells (boundaries at round(k W / grid_w), half up); a pixel of cell
// (cx, cy) compares the centres of the 3x3 cells around its own by
// D^2 = |lab - lab_c|^2 + (m / S)^2 |xy - xy_c|^2, ties to the first cell in
// row-major order; a centre becomes the mean of its pixels (kept when it has
// none).  No connectivity post-processing: the superpixel builder accepts any
// label map.  Deterministic: the update sums each centre's window in a fixed
// order with a fixed reduction tree.
#include "lfd_internal.cuh"

namespace lfd {

__device__ __forceinline__ float srgb_linear(float c)
{
    return c <= 0.04045f ? c * (1.0f / 12.92f) : powf((c + 0.055f) * (1.0f / 1.055f), 2.4f);
}

__device__ __forceinline__ float lab_f(float t)
{
    return t > (216.0f / 24389.0f) ? cbrtf(t) : ((24389.0f / 27.0f) * t + 16.0f) * (1.0f / 116.0f);
}

__device__ __forceinline__ float3 rgb_to_lab(float r, float g, float b)
{
    r = srgb_linear(r); g = srgb_linear(g); b = srgb_linear(b);
    const float X = (0.4124564f * r + 0.3575761f * g + 0.1804375f * b) * (1.0f / 0.95047f);
    const float Y = 0.2126729f * r + 0.7151522f * g + 0.0721750f * b;
    const float Z = (0.0193339f * r + 0.1191920f * g + 0.9503041f * b) * (1.0f / 1.08883f);
    const float fx = lab_f(X), fy = lab_f(Y), fz = lab_f(Z);
    return make_float3(116.0f * fy - 16.0f, 500.0f * (fx - fy), 200.0f * (fy - fz));
}

__device__ __forceinline__ void texel_rgb(int fmt, const char *row, int x, float &r, float &g, float &b)
{
    if (fmt == LFD_RGBA8) {
        const uchar4 t = ((const uchar4 *)row)[x];
        r = t.x * (1.0f / 255.0f); g = t.y * (1.0f / 255.0f); b = t.z * (1.0f / 255.0f);
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

// boundary k of n cells over `size` pixels: round(k size / n), half up
__device__ __forceinline__ int cell_edge(int k, int size, int n)
{
    return (int)((2LL * k * size + n) / (2LL * n));
}

// cell containing pixel coordinate p
__device__ __forceinline__ int cell_of(int p, int size, int n)
{
    int k = (int)(((long long)p * n) / size);
    while (k > 0 && cell_edge(k, size, n) > p) k--;
    while (k < n - 1 && cell_edge(k + 1, size, n) <= p) k++;
    return k;
}

__global__ void __launch_bounds__(256) k_slic_lab(SlicView s)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.W * s.H) return;
    const int x = p % s.W, y = p / s.W;
    float r, g, b;
    texel_rgb(s.fmt, (const char *)s.img + (long long)y * s.pitch, x, r, g, b);
    const float3 l = rgb_to_lab(r, g, b);
    s.lab[p] = make_float4(l.x, l.y, l.z, 0.f);
}

__global__ void k_slic_seeds(SlicView s)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.GW * s.GH) return;
    const int cx = c % s.GW, cy = c / s.GW;
    const float x = 0.5f * (float)(cell_edge(cx, s.W, s.GW) + cell_edge(cx + 1, s.W, s.GW) - 1);
    const float y = 0.5f * (float)(cell_edge(cy, s.H, s.GH) + cell_edge(cy + 1, s.H, s.GH) - 1);
    const int px = min((int)floorf(x + 0.5f), s.W - 1), py = min((int)floorf(y + 0.5f), s.H - 1);
    const float4 l = s.lab[(long long)py * s.W + px];
    float *o = s.centres + 5 * (long long)c;
    o[0] = l.x; o[1] = l.y; o[2] = l.z; o[3] = x; o[4] = y;
}

__global__ void __launch_bounds__(256) k_slic_assign(SlicView s, const float *centres, float wxy)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.W * s.H) return;
    const int x = p % s.W, y = p / s.W;
    const int cx = cell_of(x, s.W, s.GW), cy = cell_of(y, s.H, s.GH);
    const float4 l = s.lab[p];
    float best = INFINITY;
    int arg = -1;
    for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
            const int nx = cx + dx, ny = cy + dy;
            if (nx < 0 || ny < 0 || nx >= s.GW || ny >= s.GH) continue;
            const float *c = centres + 5 * (long long)(ny * s.GW + nx);
            const float dl = l.x - c[0], da = l.y - c[1], db = l.z - c[2];
            const float ddx = (float)x - c[3], ddy = (float)y - c[4];
            const float D = fmaf(dl, dl, fmaf(da, da, db * db)) + wxy * fmaf(ddx, ddx, ddy * ddy);
            if (D < best) {
                best = D;
                arg = ny * s.GW + nx;
            }
        }
    s.labels[p] = arg;
}

// one warp per centre: the pixels of the 3x3 cells around its own that carry its label
__global__ void __launch_bounds__(128) k_slic_update(SlicView s, const float *cin, float *cout)
{
    const int c = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= s.GW * s.GH) return;
    const int cx = c % s.GW, cy = c / s.GW;
    const int x0 = cell_edge(max(cx - 1, 0), s.W, s.GW), x1 = cell_edge(min(cx + 2, s.GW), s.W, s.GW);
    const int y0 = cell_edge(max(cy - 1, 0), s.H, s.GH), y1 = cell_edge(min(cy + 2, s.GH), s.H, s.GH);
    const int ww = x1 - x0;
    const long long area = (long long)ww * (y1 - y0);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
    int n = 0;
    for (long long i = lane; i < area; i += 32) {
        const int x = x0 + (int)(i % ww), y = y0 + (int)(i / ww);
        const long long p = (long long)y * s.W + x;
        if (s.labels[p] != c) continue;
        const float4 l = s.lab[p];
        a0 += l.x; a1 += l.y; a2 += l.z; a3 += (float)x; a4 += (float)y;
        n++;
    }
    a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2); a3 = warp_sum(a3); a4 = warp_sum(a4);
    n = __reduce_add_sync(0xffffffffu, (unsigned)n);
    if (lane == 0) {
        float *o = cout + 5 * (long long)c;
        const float *i = cin + 5 * (long long)c;
        if (n > 0) {
            const float r = 1.0f / (float)n;
            o[0] = a0 * r; o[1] = a1 * r; o[2] = a2 * r; o[3] = a3 * r; o[4] = a4 * r;
        } else {
            for (int k = 0; k < 5; k++) o[k] = i[k];
        }
    }
}

cudaError_t launch_slic(const SlicView &s, const float *centres_in, int iterations, float m, float *centres_out,
                        cudaStream_t st)
{
    const int npx = s.W * s.H, S = s.GW * s.GH;
    const int pb = (npx + 255) / 256;
    k_slic_lab<<<pb, 256, 0, st>>>(s);
    float *a = s.centres, *b = s.centres2;
    if (centres_in) {
        cudaError_t e = cudaMemcpyAsync(a, centres_in, sizeof(float) * 5 * S, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    } else {
        k_slic_seeds<<<(S + 127) / 128, 128, 0, st>>>(s);
    }
    const double step = sqrt((double)npx / (double)S);
    const float wxy = (float)((m / step) * (m / step));
    for (int it = 0; it < iterations; it++) {
        k_slic_assign<<<pb, 256, 0, st>>>(s, a, wxy);
        k_slic_update<<<(S + 3) / 4, 128, 0, st>>>(s, a, b);
        float *t = a; a = b; b = t;
    }
    k_slic_assign<<<pb, 256, 0, st>>>(s, a, wxy);
    if (centres_out) {
        cudaError_t e = cudaMemcpyAsync(centres_out, a, sizeof(float) * 5 * S, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace lfd
