// Bilinear sampling and truncated SSD (Eq. 1) on the per-pixel quad textures.
// Shared by the sweep kernel and the per-hypothesis score kernel.
#pragma once
#include "lfd_internal.cuh"

namespace lfd {

// colour of one texel of the quad in the sampler's units (RGBA8: 0..255)
template <int FMT>
struct Quad;

// RGBA8 views are sampled from a coefficient-form texture: per pixel and
// channel c(x+fx, y+fy) = a + fx bx + fy by + fx fy bxy with a = c00,
// bx = c10 - c00, by = c01 - c00, bxy = c11 - c10 - c01 + c00.  All four are
// integers of at most 11 bits, hence exact as IEEE halves: 12 halves = 24 B
// per pixel, stored as a 16-B record (a.rgb, bx.rgb, by.rg) and an 8-B record
// (by.b, bxy.rgb).  Values are in byte units (0..255).
__device__ __forceinline__ float2 h2f(unsigned u);

struct Coef8 {
    float a[3], bx[3], by[3], bxy[3];
    __device__ __forceinline__ void load(const void *tex, long long idx, long long npx)
    {
        const uint4 q = __ldg((const uint4 *)tex + idx);
        const uint2 e = __ldg((const uint2 *)((const uint4 *)tex + npx) + idx);
        float2 t;
        t = h2f(q.x); a[0] = t.x; a[1] = t.y;
        t = h2f(q.y); a[2] = t.x; bx[0] = t.y;
        t = h2f(q.z); bx[1] = t.x; bx[2] = t.y;
        t = h2f(q.w); by[0] = t.x; by[1] = t.y;
        t = h2f(e.x); by[2] = t.x; bxy[0] = t.y;
        t = h2f(e.y); bxy[1] = t.x; bxy[2] = t.y;
    }
};

__device__ __forceinline__ float2 h2f(unsigned u)
{
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    return __half22float2(h);
}

__device__ __forceinline__ float2 bf2f(unsigned u)
{
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&u);
    return __bfloat1622float2(h);
}

template <>
struct Quad<LFD_RGBA_F16> {
    float r[4], g[4], b[4];
    __device__ __forceinline__ void load(const void *tex, long long idx)
    {
        const uint4 *q = (const uint4 *)tex + 2 * idx;
        const uint4 a = __ldg(q), c = __ldg(q + 1);
        float2 t;
        t = h2f(a.x); r[0] = t.x; g[0] = t.y; b[0] = h2f(a.y).x;
        t = h2f(a.z); r[1] = t.x; g[1] = t.y; b[1] = h2f(a.w).x;
        t = h2f(c.x); r[2] = t.x; g[2] = t.y; b[2] = h2f(c.y).x;
        t = h2f(c.z); r[3] = t.x; g[3] = t.y; b[3] = h2f(c.w).x;
    }
};

template <>
struct Quad<LFD_RGBA_BF16> {
    float r[4], g[4], b[4];
    __device__ __forceinline__ void load(const void *tex, long long idx)
    {
        const uint4 *q = (const uint4 *)tex + 2 * idx;
        const uint4 a = __ldg(q), c = __ldg(q + 1);
        float2 t;
        t = bf2f(a.x); r[0] = t.x; g[0] = t.y; b[0] = bf2f(a.y).x;
        t = bf2f(a.z); r[1] = t.x; g[1] = t.y; b[1] = bf2f(a.w).x;
        t = bf2f(c.x); r[2] = t.x; g[2] = t.y; b[2] = bf2f(c.y).x;
        t = bf2f(c.z); r[3] = t.x; g[3] = t.y; b[3] = bf2f(c.w).x;
    }
};

template <>
struct Quad<LFD_RGBA_F32> {
    float r[4], g[4], b[4];
    __device__ __forceinline__ void load(const void *tex, long long idx)
    {
        const float4 *q = (const float4 *)tex + 3 * idx;
        const float4 a = __ldg(q), c = __ldg(q + 1), d = __ldg(q + 2);
        r[0] = a.x; g[0] = a.y; b[0] = a.z; r[1] = a.w;
        g[1] = c.x; b[1] = c.y; r[2] = c.z; g[2] = c.w;
        b[2] = d.x; r[3] = d.y; g[3] = d.z; b[3] = d.w;
    }
};

// colour of pixel (x,y) itself (texel t00 of its quad); npx = pixels of the view
template <int FMT>
__device__ __forceinline__ float3 texel_colour(const void *tex, long long idx, long long npx)
{
    if constexpr (FMT == LFD_RGBA8) {
        const uint4 q = __ldg((const uint4 *)tex + idx);
        const float2 t0 = h2f(q.x), t1 = h2f(q.y);
        return make_float3(t0.x, t0.y, t1.x);
    } else {
        Quad<FMT> q;
        q.load(tex, idx);
        return make_float3(q.r[0], q.g[0], q.b[0]);
    }
}

// Truncated SSD of Eq. 1 between the reference colour `ref` and view i sampled
// bilinearly at the homogeneous point (X, Y, Wz); T when the point is behind
// camera i (Wz <= 0) or off the image's texture area -1/2 <= x < Wi - 1/2,
// -1/2 <= y < Hi - 1/2 (its nearest pixel is not a pixel of view i).  Inside,
// the coordinates are clamped to the outermost pixel centres (clamp to edge).
template <int FMT>
__device__ __forceinline__ float tssd_sample(const void *tex, int Wi, int Hi, float X, float Y, float Wz, float3 ref,
                                             float T)
{
    const float rw = rcp_approx(Wz);
    const float xr = X * rw, yr = Y * rw;
    const bool ok = (Wz > 0.f) && (xr >= -0.5f) && (xr < (float)Wi - 0.5f) && (yr >= -0.5f) &&
                    (yr < (float)Hi - 0.5f);
    if (!ok) return T;
    const float x = fminf(fmaxf(xr, 0.f), (float)(Wi - 1)), y = fminf(fmaxf(yr, 0.f), (float)(Hi - 1));
    const float xf = floorf(x), yf = floorf(y);
    const float fx = x - xf, fy = y - yf;
    const long long idx = (long long)(int)yf * Wi + (int)xf;
    float dr, dg, db;
    if constexpr (FMT == LFD_RGBA8) {
        Coef8 q;
        q.load(tex, idx, (long long)Wi * Hi);
        const float fxy = fx * fy;
        dr = ref.x - fmaf(fxy, q.bxy[0], fmaf(fy, q.by[0], fmaf(fx, q.bx[0], q.a[0])));
        dg = ref.y - fmaf(fxy, q.bxy[1], fmaf(fy, q.by[1], fmaf(fx, q.bx[1], q.a[1])));
        db = ref.z - fmaf(fxy, q.bxy[2], fmaf(fy, q.by[2], fmaf(fx, q.bx[2], q.a[2])));
    } else {
        Quad<FMT> q;
        q.load(tex, idx);
        const float r0 = fmaf(fx, q.r[1] - q.r[0], q.r[0]), r1 = fmaf(fx, q.r[3] - q.r[2], q.r[2]);
        const float g0 = fmaf(fx, q.g[1] - q.g[0], q.g[0]), g1 = fmaf(fx, q.g[3] - q.g[2], q.g[2]);
        const float b0 = fmaf(fx, q.b[1] - q.b[0], q.b[0]), b1 = fmaf(fx, q.b[3] - q.b[2], q.b[2]);
        dr = ref.x - fmaf(fy, r1 - r0, r0);
        dg = ref.y - fmaf(fy, g1 - g0, g0);
        db = ref.z - fmaf(fy, b1 - b0, b0);
    }
    const float ssd = fmaf(dr, dr, fmaf(dg, dg, db * db));
    return fminf(ssd, T);
}

}  // namespace lfd
