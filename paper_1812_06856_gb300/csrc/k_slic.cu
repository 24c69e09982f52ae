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
// label map.  Deterministic: the update's sums are integers (Lab in fixed
// point), so the order of their atomics does not matter.  Up to SLIC_BATCH
// views go through the same launches (blockIdx.y = view).
#include "lfd_slic.cuh"

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
// (32-bit unsigned: 2 k size + n < 2^32 for sizes up to LFD_MAX_DIM)
__device__ __forceinline__ int cell_edge(int k, int size, int n)
{
    return (int)((2u * (unsigned)k * (unsigned)size + (unsigned)n) / (2u * (unsigned)n));
}

__global__ void __launch_bounds__(256) k_slic_lab(const __grid_constant__ SlicBatch bt)
{
    const SlicView &s = bt.v[blockIdx.y];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.W * s.H) return;
    const int x = p % s.W, y = p / s.W;
    float r, g, b;
    texel_rgb(s.fmt, (const char *)s.img + (long long)y * s.pitch, x, r, g, b);
    const float3 l = rgb_to_lab(r, g, b);
    s.lab[p] = make_float4(l.x, l.y, l.z, 0.f);
}

__global__ void k_slic_seeds(const __grid_constant__ SlicBatch b)
{
    const SlicView &s = b.v[blockIdx.y];
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

// Fixed-point scale of the Lab sums: 2^18 (a power of two, so v * 2^18 is
// exact and the rounding error of one value is at most 2^-19), on values
// clamped to [-256, 256] (every sRGB colour is inside), so that a warp's sum
// fits 32 bits.  Integer sums are associative: the update does not depend on
// the order of the reductions and atomics.
constexpr float SLIC_FIX = 262144.0f;
constexpr float SLIC_LAB_MAX = 256.0f;

// One CTA per grid cell (cx, cy): its pixels pick the nearest of the 3x3
// cells' centres (ties to the first in row-major order) and, with `acc`,
// add {L, a, b} (fixed point), x, y and 1 to the winner's sums: per warp one
// REDUX per quantity and centre present, into the CTA's 9 bins in shared
// memory, then 9 x 6 64-bit atomics into acc.
constexpr int SLIC_ASSIGN_THREADS = 256;

__device__ __forceinline__ int slic_fix(float v)
{
    return __float2int_rn(fminf(fmaxf(v, -SLIC_LAB_MAX), SLIC_LAB_MAX) * SLIC_FIX);
}

__global__ void __launch_bounds__(SLIC_ASSIGN_THREADS) k_slic_assign(const __grid_constant__ SlicBatch b, int parity,
                                                                     bool accumulate)
{
    const SlicView &s = b.v[blockIdx.y];
    if ((int)blockIdx.x >= s.GW * s.GH) return;                // past this view's cells (whole CTA)
    const float *centres = parity ? s.centres2 : s.centres;
    unsigned long long *acc = accumulate ? s.acc : nullptr;
    const float wxy = b.wxy[blockIdx.y];
    __shared__ float cen[9][5];
    __shared__ int cid[9];
    __shared__ unsigned long long bin[9][6];
    const int lane = threadIdx.x & 31;
    const int cx = blockIdx.x % s.GW, cy = blockIdx.x / s.GW;
    if (threadIdx.x < 9) {
        const int nx = cx + threadIdx.x % 3 - 1, ny = cy + threadIdx.x / 3 - 1;
        const bool in = nx >= 0 && ny >= 0 && nx < s.GW && ny < s.GH;
        const int c = in ? ny * s.GW + nx : -1;
        cid[threadIdx.x] = c;
        for (int j = 0; j < 5; j++) cen[threadIdx.x][j] = in ? centres[5 * (long long)c + j] : 0.f;
    }
    if (threadIdx.x < 54) bin[threadIdx.x / 6][threadIdx.x % 6] = 0ull;
    __syncthreads();
    const int x0 = cell_edge(cx, s.W, s.GW), x1 = cell_edge(cx + 1, s.W, s.GW);
    const int y0 = cell_edge(cy, s.H, s.GH), y1 = cell_edge(cy + 1, s.H, s.GH);
    const int cw = x1 - x0, n = cw * (y1 - y0);
    for (int base = 0; base < n; base += SLIC_ASSIGN_THREADS) {
        if (base + (int)(threadIdx.x & ~31u) >= n) break;      // the whole warp is past the cell
        const int i = base + threadIdx.x;
        bool take = false;
        int k = 4, x = 0, y = 0;
        float4 l = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < n) {
            y = y0 + i / cw;
            x = x0 + i % cw;
            const long long p = (long long)y * s.W + x;
            l = __ldg(s.lab + p);
            float best = INFINITY;
            int kb = -1;
#pragma unroll
            for (int j = 0; j < 9; j++) {
                if (cid[j] < 0) continue;
                const float dl = l.x - cen[j][0], da = l.y - cen[j][1], db = l.z - cen[j][2];
                const float ddx = (float)x - cen[j][3], ddy = (float)y - cen[j][4];
                const float D = fmaf(dl, dl, fmaf(da, da, db * db)) + wxy * fmaf(ddx, ddx, ddy * ddy);
                if (D < best) {
                    best = D;
                    kb = j;
                }
            }
            take = kb >= 0;              // all distances NaN (non-finite colour): own cell, not counted
            if (take) k = kb;
            s.labels[p] = cid[k];
        }
        if (!acc) continue;
        const int qL = take ? slic_fix(l.x) : 0, qa = take ? slic_fix(l.y) : 0, qb = take ? slic_fix(l.z) : 0;
        unsigned present = __reduce_or_sync(0xffffffffu, take ? 1u << k : 0u);
        while (present) {
            const int j = __ffs(present) - 1;
            present &= present - 1;
            const bool me = take && k == j;
            const int sL = __reduce_add_sync(0xffffffffu, me ? qL : 0);
            const int sa = __reduce_add_sync(0xffffffffu, me ? qa : 0);
            const int sb = __reduce_add_sync(0xffffffffu, me ? qb : 0);
            const int sx = __reduce_add_sync(0xffffffffu, me ? x : 0);
            const int sy = __reduce_add_sync(0xffffffffu, me ? y : 0);
            const unsigned sc = __reduce_add_sync(0xffffffffu, me ? 1u : 0u);
            if (lane == 0) {
                atomicAdd(&bin[j][0], (unsigned long long)(long long)sL);
                atomicAdd(&bin[j][1], (unsigned long long)(long long)sa);
                atomicAdd(&bin[j][2], (unsigned long long)(long long)sb);
                atomicAdd(&bin[j][3], (unsigned long long)sx);
                atomicAdd(&bin[j][4], (unsigned long long)sy);
                atomicAdd(&bin[j][5], (unsigned long long)sc);
            }
        }
    }
    if (!acc) return;
    __syncthreads();
    if (threadIdx.x < 54) {
        const int j = threadIdx.x / 6, q = threadIdx.x % 6;
        if (cid[j] >= 0 && bin[j][5]) atomicAdd(acc + 6 * (long long)cid[j] + q, bin[j][q]);
    }
}

// centre c becomes the mean of its sums (kept when it has no pixel); the sums are cleared
__global__ void k_slic_finalize(const __grid_constant__ SlicBatch b, int parity)
{
    const SlicView &s = b.v[blockIdx.y];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.GW * s.GH) return;
    const float *cin = parity ? s.centres2 : s.centres;
    float *cout = parity ? s.centres : s.centres2;
    unsigned long long *acc = s.acc;
    unsigned long long *a = acc + 6 * (long long)c;
    const unsigned long long cnt = a[5];
    float *o = cout + 5 * (long long)c;
    if (cnt > 0) {
        const double r = 1.0 / (double)cnt;
        for (int j = 0; j < 3; j++) o[j] = (float)((double)(long long)a[j] * r * (1.0 / SLIC_FIX));
        o[3] = (float)((double)a[3] * r);
        o[4] = (float)((double)a[4] * r);
    } else {
        for (int j = 0; j < 5; j++) o[j] = cin[5 * (long long)c + j];
    }
    for (int j = 0; j < 6; j++) a[j] = 0ull;
}

cudaError_t launch_slic(const SlicBatch &b, const float *const *centres_in, int iterations,
                        float *const *centres_out, cudaStream_t st)
{
    const dim3 g_px((b.max_px + 255) / 256, b.n), g_cells((b.max_cells + 127) / 128, b.n), g_cta(b.max_cells, b.n);
    k_slic_lab<<<g_px, 256, 0, st>>>(b);
    bool seeds = false;
    for (int v = 0; v < b.n; v++) {
        const SlicView &s = b.v[v];
        const size_t S = (size_t)s.GW * s.GH;
        cudaError_t e = cudaSuccess;
        if (centres_in && centres_in[v])
            e = cudaMemcpyAsync(s.centres, centres_in[v], sizeof(float) * 5 * S, cudaMemcpyDeviceToDevice, st);
        else
            seeds = true;
        if (e == cudaSuccess && iterations > 0) e = cudaMemsetAsync(s.acc, 0, sizeof(unsigned long long) * 6 * S, st);
        if (e != cudaSuccess) return e;
    }
    if (seeds) {
        // views with given centres keep them: seed only the others
        SlicBatch bs = b;
        int k = 0;
        for (int v = 0; v < b.n; v++)
            if (!(centres_in && centres_in[v])) bs.v[k++] = b.v[v];
        bs.n = k;
        k_slic_seeds<<<dim3((b.max_cells + 127) / 128, k), 128, 0, st>>>(bs);
    }
    for (int it = 0; it < iterations; it++) {
        k_slic_assign<<<g_cta, SLIC_ASSIGN_THREADS, 0, st>>>(b, it & 1, true);
        k_slic_finalize<<<g_cells, 128, 0, st>>>(b, it & 1);
    }
    const int parity = iterations & 1;
    k_slic_assign<<<g_cta, SLIC_ASSIGN_THREADS, 0, st>>>(b, parity, false);
    for (int v = 0; v < b.n && centres_out; v++) {
        if (!centres_out[v]) continue;
        const SlicView &s = b.v[v];
        cudaError_t e = cudaMemcpyAsync(centres_out[v], parity ? s.centres2 : s.centres,
                                        sizeof(float) * 5 * (size_t)s.GW * s.GH, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace lfd
