// Bilinear sampling and truncated SSD (Eq. 1) on the per-pixel quad textures.
// Shared by the sweep kernel and the per-hypothesis score kernel.
#pragma once
#include "lfd_internal.cuh"

namespace lfd {

// colour of one texel of the quad in the sampler's units (RGBA8: 0..255)
template <int FMT>
struct Quad;

// The sampling texture's storage format: RGBA8 views keep their texels as
// IEEE halves (integers 0..255 are exact), laid out as the FP16 texture;
// values are in byte units (0..255).
template <int FMT>
__host__ __device__ constexpr int tex_fmt() { return FMT == LFD_RGBA8 ? LFD_RGBA_F16 : FMT; }

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

// The 2x2 texels of a float quad (k = 0 (x,y), 1 (x+1,y), 2 (x,y+1),
// 3 (x+1,y+1)): rg[k] = (red, green) of texel k, and the blues as the
// column pairs b02 = (b0, b2), b13 = (b1, b3), each a pair for the packed
// arithmetic (the x lerp of both rows of blue is one packed lerp).
// FP16/BF16 entries: a 16-B record of the four red/green pairs and an 8-B
// record of the two blue pairs, the second array starting after npx 16-B
// records.
template <>
struct Quad<LFD_RGBA_F16> {
    float2 rg[4];
    float2 b02, b13;
    __device__ __forceinline__ void load(const void *tex, long long idx, long long npx)
    {
        const uint4 a = __ldg((const uint4 *)tex + idx);
        const uint2 e = __ldg((const uint2 *)((const uint4 *)tex + npx) + idx);
        rg[0] = h2f(a.x); rg[1] = h2f(a.y); rg[2] = h2f(a.z); rg[3] = h2f(a.w);
        b02 = h2f(e.x);
        b13 = h2f(e.y);
    }
};

template <>
struct Quad<LFD_RGBA_BF16> {
    float2 rg[4];
    float2 b02, b13;
    __device__ __forceinline__ void load(const void *tex, long long idx, long long npx)
    {
        const uint4 a = __ldg((const uint4 *)tex + idx);
        const uint2 e = __ldg((const uint2 *)((const uint4 *)tex + npx) + idx);
        rg[0] = bf2f(a.x); rg[1] = bf2f(a.y); rg[2] = bf2f(a.z); rg[3] = bf2f(a.w);
        b02 = bf2f(e.x);
        b13 = bf2f(e.y);
    }
};

template <>
struct Quad<LFD_RGBA_F32> {
    float2 rg[4];
    float2 b02, b13;
    __device__ __forceinline__ void load(const void *tex, long long idx, long long)
    {
        const float4 *q = (const float4 *)tex + 3 * idx;
        const float4 a = __ldg(q), c = __ldg(q + 1), d = __ldg(q + 2);
        rg[0] = make_float2(a.x, a.y);
        rg[1] = make_float2(a.w, c.x);
        rg[2] = make_float2(c.z, c.w);
        rg[3] = make_float2(d.y, d.z);
        b02 = make_float2(a.z, d.x);
        b13 = make_float2(c.y, d.w);
    }
};

// (float(lo(w)) - a.x, float(hi(w)) - a.y) for a word w of two FP16 or BF16
// values: Blackwell's mixed-precision subtraction takes the 16-bit operand
// as it is (the conversion is exact, one rounding as FSUB of the converted
// values), which saves converting the second texel of each lerp.
template <int FMT>
__device__ __forceinline__ float2 msub2(unsigned w, float2 a)
{
    float2 d;
    if constexpr (FMT == LFD_RGBA_F16)
        asm("{\n\t.reg .f16 l, h;\n\tmov.b32 {l, h}, %2;\n\tsub.rn.f32.f16 %0, l, %3;\n\t"
            "sub.rn.f32.f16 %1, h, %4;\n\t}"
            : "=f"(d.x), "=f"(d.y) : "r"(w), "f"(a.x), "f"(a.y));
    else
        asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tsub.rn.f32.bf16 %0, l, %3;\n\t"
            "sub.rn.f32.bf16 %1, h, %4;\n\t}"
            : "=f"(d.x), "=f"(d.y) : "r"(w), "f"(a.x), "f"(a.y));
    return d;
}

// float(lo(w)) - a for a word w holding a FP16 or BF16 value in its low half
template <int FMT>
__device__ __forceinline__ float msub1(unsigned w, float a)
{
    float d;
    if constexpr (FMT == LFD_RGBA_F16)
        asm("{\n\t.reg .f16 l, h;\n\tmov.b32 {l, h}, %1;\n\tsub.rn.f32.f16 %0, l, %2;\n\t}"
            : "=f"(d) : "r"(w), "f"(a));
    else
        asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\tsub.rn.f32.bf16 %0, l, %2;\n\t}"
            : "=f"(d) : "r"(w), "f"(a));
    return d;
}

// (lo, hi) packed as the texture's 16-bit format (exact for its own texel values)
template <int FMT>
__device__ __forceinline__ unsigned pack2(float lo, float hi)
{
    if constexpr (FMT == LFD_RGBA_F16) {
        __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<unsigned *>(&h);
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<unsigned *>(&h);
    }
}

template <int FMT>
__device__ __forceinline__ float2 cvt2(unsigned w)
{
    if constexpr (FMT == LFD_RGBA_F16) return h2f(w);
    else return bf2f(w);
}

// entry of pixel (x, y) in a view's sampling texture (a border of one quad
// on the left and top, (W + 1) x (H + 1) entries; see k_quads)
__device__ __forceinline__ long long quad_index(int x, int y, int W)
{
    return (long long)(y + 1) * (W + 1) + (x + 1);
}

__device__ __forceinline__ long long quad_entries(int W, int H) { return (long long)(W + 1) * (H + 1); }

// colour of pixel (x,y) itself (texel t00 of its quad)
template <int FMT>
__device__ __forceinline__ float3 texel_colour(const void *tex, int x, int y, int W, int H)
{
    const long long idx = quad_index(x, y, W), npx = quad_entries(W, H);
    Quad<tex_fmt<FMT>()> q;
    q.load(tex, idx, npx);
    return make_float3(q.rg[0].x, q.rg[0].y, q.b02.x);
}

// Truncated SSD of Eq. 1 between the reference colour `ref` and the bilinear
// sample of the quad at entry idx of view i's texture (the 2 x 2 texels from
// pixel (x0, y0), idx = quad_index(x0, y0, Wi)) at fractions (fx, fy) in
// [0, 1); npx = quad_entries(Wi, Hi).
template <int FMT>
__device__ __forceinline__ float tssd_quad(const void *tex, long long idx, long long npx, float fx, float fy,
                                           float3 ref, float T)
{
    constexpr int TF = tex_fmt<FMT>();
    if constexpr (TF == LFD_RGBA_F16 || TF == LFD_RGBA_BF16) {
        // the record's words as they are: the first texel of each x lerp
        // converted, the second entering through the mixed-precision
        // subtraction; the same values as the Quad form below
        const uint4 a = __ldg((const uint4 *)tex + idx);
        const uint2 e = __ldg((const uint2 *)((const uint4 *)tex + npx) + idx);
        const float2 FX = dup2(fx);
        const float2 r0 = cvt2<TF>(a.x), r2 = cvt2<TF>(a.z), b02 = cvt2<TF>(e.x);
        const float2 top = ffma2(FX, msub2<TF>(a.y, r0), r0);
        const float2 bot = ffma2(FX, msub2<TF>(a.w, r2), r2);
        const float2 rg = ffma2(dup2(fy), fsub2(bot, top), top);
        const float2 bb = ffma2(FX, msub2<TF>(e.y, b02), b02);        // (top, bottom) blue
        const float2 d = fsub2(make_float2(ref.x, ref.y), rg);
        const float2 d2 = fmul2(d, d);
        const float db = ref.z - fmaf(fy, bb.y - bb.x, bb.x);
        return fminf(fmaf(db, db, d2.x + d2.y), T);
    } else {
        // red/green of a row and blue of both rows as packed pairs: the same
        // lerps as scalar code in fewer issue slots
        Quad<FMT> q;
        q.load(tex, idx, npx);
        const float2 FX = dup2(fx);
        const float2 top = ffma2(FX, fsub2(q.rg[1], q.rg[0]), q.rg[0]);
        const float2 bot = ffma2(FX, fsub2(q.rg[3], q.rg[2]), q.rg[2]);
        const float2 rg = ffma2(dup2(fy), fsub2(bot, top), top);
        const float2 bb = ffma2(FX, fsub2(q.b13, q.b02), q.b02);       // (top, bottom) blue
        const float2 d = fsub2(make_float2(ref.x, ref.y), rg);
        const float2 d2 = fmul2(d, d);
        const float db = ref.z - fmaf(fy, bb.y - bb.x, bb.x);
        return fminf(fmaf(db, db, d2.x + d2.y), T);
    }
}

// tssd_quad for a 16-bit texture with the reference colour given in the
// texture's own format (ref_rg: red|green, ref_b: blue in the low half):
// the reference enters the differences through the mixed-precision
// subtraction, the same values as tssd_quad on the converted colour.
template <int FMT>
__device__ __forceinline__ float tssd_quad_href(const void *tex, long long idx, long long npx, float fx, float fy,
                                                unsigned ref_rg, unsigned ref_b, float T)
{
    constexpr int TF = tex_fmt<FMT>();
    static_assert(TF == LFD_RGBA_F16 || TF == LFD_RGBA_BF16, "16-bit textures only");
    const uint4 a = __ldg((const uint4 *)tex + idx);
    const uint2 e = __ldg((const uint2 *)((const uint4 *)tex + npx) + idx);
    const float2 FX = dup2(fx);
    const float2 r0 = cvt2<TF>(a.x), r2 = cvt2<TF>(a.z), b02 = cvt2<TF>(e.x);
    const float2 top = ffma2(FX, msub2<TF>(a.y, r0), r0);
    const float2 bot = ffma2(FX, msub2<TF>(a.w, r2), r2);
    const float2 rg = ffma2(dup2(fy), fsub2(bot, top), top);
    const float2 bb = ffma2(FX, msub2<TF>(e.y, b02), b02);        // (top, bottom) blue
    const float2 d = msub2<TF>(ref_rg, rg);
    const float2 d2 = fmul2(d, d);
    const float db = msub1<TF>(ref_b, fmaf(fy, bb.y - bb.x, bb.x));
    return fminf(fmaf(db, db, d2.x + d2.y), T);
}

// Truncated SSD of Eq. 1 between the reference colour `ref` and view i sampled
// bilinearly at the homogeneous point (X, Y, Wz); T when the point is behind
// camera i (Wz <= 0) or off the image's texture area -1/2 <= x < Wi - 1/2,
// -1/2 <= y < Hi - 1/2 (its nearest pixel is not a pixel of view i).  Inside,
// the texture's border quads give clamp-to-edge (see k_quads).
// tssd_at: the same at the dehomogenised point (x, y) of a point in front of
// camera i.
template <int FMT>
__device__ __forceinline__ float tssd_at(const void *tex, int Wi, int Hi, float x, float y, float3 ref, float T)
{
    const bool ok = (x >= -0.5f) && (x < (float)Wi - 0.5f) && (y >= -0.5f) && (y < (float)Hi - 0.5f);
    if (!ok) return T;
    const float xf = floorf(x), yf = floorf(y);          // -1 .. W-1, -1 .. H-1
    return tssd_quad<FMT>(tex, quad_index((int)xf, (int)yf, Wi), quad_entries(Wi, Hi), x - xf, y - yf, ref, T);
}

template <int FMT>
__device__ __forceinline__ float tssd_sample(const void *tex, int Wi, int Hi, float X, float Y, float Wz, float3 ref,
                                             float T)
{
    const float rw = rcp_approx(Wz);
    if (!(Wz > 0.f)) return T;
    return tssd_at<FMT>(tex, Wi, Hi, X * rw, Y * rw, ref, T);
}

}  // namespace lfd
