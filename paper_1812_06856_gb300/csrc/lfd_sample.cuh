// Bilinear sampling and truncated SSD (Eq. 1) on the per-pixel quad textures.
// Shared by the sweep kernel and the per-hypothesis score kernel.
#pragma once
#include "lfd_internal.cuh"

namespace lfd {

// colour of one texel of the quad in the sampler's units (RGBA8: 0..255)
template <int FMT>
struct Quad;

template <>
struct Quad<LFD_RGBA8> {
    float r[4], g[4], b[4];   // t00, t10, t01, t11
    __device__ __forceinline__ void load(const void *tex, long long idx)
    {
        const uint4 q = __ldg((const uint4 *)tex + idx);
        r[0] = u8_to_f<0>(q.x); g[0] = u8_to_f<1>(q.x); b[0] = u8_to_f<2>(q.x);
        r[1] = u8_to_f<0>(q.y); g[1] = u8_to_f<1>(q.y); b[1] = u8_to_f<2>(q.y);
        r[2] = u8_to_f<0>(q.z); g[2] = u8_to_f<1>(q.z); b[2] = u8_to_f<2>(q.z);
        r[3] = u8_to_f<0>(q.w); g[3] = u8_to_f<1>(q.w); b[3] = u8_to_f<2>(q.w);
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

// colour of pixel (x,y) itself (texel t00 of its quad)
template <int FMT>
__device__ __forceinline__ float3 texel_colour(const void *tex, long long idx)
{
    Quad<FMT> q;
    q.load(tex, idx);
    return make_float3(q.r[0], q.g[0], q.b[0]);
}

// Truncated SSD of Eq. 1 between the reference colour `ref` and view i sampled
// bilinearly at the homogeneous point (X, Y, Wz); T when the point is behind
// camera i (Wz <= 0) or outside 0 <= x <= Wi-1, 0 <= y <= Hi-1.
template <int FMT>
__device__ __forceinline__ float tssd_sample(const void *tex, int Wi, int Hi, float X, float Y, float Wz, float3 ref,
                                             float T)
{
    const float rw = rcp_approx(Wz);
    const float x = X * rw, y = Y * rw;
    const bool ok = (Wz > 0.f) && (x >= 0.f) && (x <= (float)(Wi - 1)) && (y >= 0.f) && (y <= (float)(Hi - 1));
    if (!ok) return T;
    const float xf = floorf(x), yf = floorf(y);
    const float fx = x - xf, fy = y - yf;
    Quad<FMT> q;
    q.load(tex, (long long)(int)yf * Wi + (int)xf);
    const float r0 = fmaf(fx, q.r[1] - q.r[0], q.r[0]), r1 = fmaf(fx, q.r[3] - q.r[2], q.r[2]);
    const float g0 = fmaf(fx, q.g[1] - q.g[0], q.g[0]), g1 = fmaf(fx, q.g[3] - q.g[2], q.g[2]);
    const float b0 = fmaf(fx, q.b[1] - q.b[0], q.b[0]), b1 = fmaf(fx, q.b[3] - q.b[2], q.b[2]);
    const float dr = ref.x - fmaf(fy, r1 - r0, r0);
    const float dg = ref.y - fmaf(fy, g1 - g0, g0);
    const float db = ref.z - fmaf(fy, b1 - b0, b0);
    const float ssd = fmaf(dr, dr, fmaf(dg, dg, db * db));
    return fminf(ssd, T);
}

}  // namespace lfd
