// C ABI of liblfdepth: context, validation, workspace, host logic and the
// enqueueing of the hot-path kernels (include/lfdepth.h documents every call).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lfd_internal.cuh"

using namespace lfd;

namespace {

// ---------------------------------------------------------------------------
// host logic: neighbour views and propagation-kernel radii
// ---------------------------------------------------------------------------

void camera_centre(const lfd_camera &c, double C[3])
{
    // C = -R^T t
    for (int k = 0; k < 3; k++) C[k] = -(c.R[k] * c.t[0] + c.R[3 + k] * c.t[1] + c.R[6 + k] * c.t[2]);
}

// N(v): the k nearest camera centres, nearer first; a later view displaces the
// current choice only when it is nearer by more than a relative 1e-9, so equal
// distances keep the lower index.
void neighbour_views(const lfd_camera *cams, int V, int k, std::vector<int> &out)
{
    out.assign((size_t)V * LFD_MAXN, -1);
    std::vector<double> C((size_t)V * 3);
    for (int v = 0; v < V; v++) camera_centre(cams[v], &C[3 * v]);
    std::vector<double> dist(V);
    std::vector<char> taken(V);
    for (int v = 0; v < V; v++) {
        for (int i = 0; i < V; i++) {
            const double dx = C[3 * i] - C[3 * v], dy = C[3 * i + 1] - C[3 * v + 1], dz = C[3 * i + 2] - C[3 * v + 2];
            dist[i] = std::sqrt(dx * dx + dy * dy + dz * dz);
            taken[i] = (i == v);
        }
        for (int r = 0; r < k; r++) {
            int pick = -1;
            for (int i = 0; i < V; i++) {
                if (taken[i]) continue;
                if (pick < 0 || dist[i] < dist[pick] * (1.0 - 1e-9)) pick = i;
            }
            taken[pick] = 1;
            out[(size_t)v * LFD_MAXN + r] = pick;
        }
    }
}

// Distinct ray radii of iteration I (Eq. 4): r_k = max(1, floor(k Size_I /
// Steps_I + 0.5)) is non-decreasing in k, so the cells of a repeated radius or
// of radius 1 (the immediate ring) are repeats; the kernel is the ring plus
// 8 cells for each distinct radius > 1, in increasing order.
int kernel_radii(int size_init, int steps_init, int I, int *radii, int cap)
{
    if (size_init < 1 || I < 1) return 0;
    const double size_I = (double)size_init / (double)I;
    const int steps_I = std::max(1, steps_init / I);
    int n = 0, last = 1;
    for (int k = 1; k <= steps_I; k++) {
        const int r = std::max(1, (int)std::floor((double)k * size_I / (double)steps_I + 0.5));
        if (r > last) {
            if (n < cap && radii) radii[n] = r;
            n++;
            last = r;
        }
    }
    return n;
}

const int RDX[8] = {1, 1, 0, -1, -1, -1, 0, 1};
const int RDY[8] = {0, -1, -1, -1, 0, 1, 1, 1};

int texel_bytes(int fmt)
{
    switch (fmt) {
    case LFD_RGBA8: return 4;
    case LFD_RGBA_F16: case LFD_RGBA_BF16: return 8;
    case LFD_RGBA_F32: return 16;
    default: return 0;
    }
}

int quad_bytes(int fmt)
{
    switch (fmt) {
    case LFD_RGBA8: return 24;
    case LFD_RGBA_F16: case LFD_RGBA_BF16: return 32;
    case LFD_RGBA_F32: return 48;
    default: return 0;
    }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Arena {
    char *base = nullptr;
    size_t cap = 0, used = 0;
    void *take(size_t bytes)
    {
        used = align_up(used, 256);
        void *p = base + used;
        used += bytes;
        return p;
    }
};

struct Layout {
    int V = 0;
    std::vector<int> W, H, GW, GH, S, sp_base;
    std::vector<long long> px_base;
    int S_total = 0;
    long long px_total = 0;
    int max_px = 0;
};

}  // namespace

struct lfd_ctx {
    int device = 0;
    uint64_t budget = 0;
    std::string err;
    bool bound = false;
    lfd_params p{};
    Consts c{};
    Layout L;
    std::vector<lfd_camera> cams;
    std::vector<int> nbr;
    int nnb = 0;
    int fmt = 0;
    // workspace
    Arena ws;
    Workspace w{};
    ViewDev *d_views = nullptr;
    PairDev *d_pairs = nullptr;
    int *d_sp_view = nullptr, *d_sp_off = nullptr, *d_sp_cnt = nullptr;
    unsigned *d_sp_pix = nullptr;
    int2 *d_sp_ref = nullptr;
    double2 *d_sp_cen = nullptr;
    float4 *d_sp_col = nullptr;
    double4_32a *d_sp_g = nullptr;
    float4 *d_sp_rc = nullptr;
    int4 *d_bbox = nullptr;
    short *d_radii = nullptr;
    int *d_radii_cnt = nullptr;
    DevCounters *d_ctr = nullptr;
    float4 *d_planesA = nullptr, *d_planesB = nullptr;
    int *d_label = nullptr, *d_choice = nullptr;
    float *d_energy = nullptr;
    std::vector<void *> quads;
    std::vector<float4 *> maps;
    // on-demand buffers
    float *d_cost = nullptr;
    size_t cost_cap = 0;
    void *d_stage_in = nullptr;      // host-path views + labels
    size_t stage_in_cap = 0;
    float *d_stage_depth = nullptr;
    size_t stage_depth_cap = 0;
    lfd_query *d_q = nullptr;
    float *d_qout = nullptr;
    int q_cap = 0;
    // tracing: event pairs around launches, per stage
    bool prof = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_used;
    std::vector<cudaEvent_t> prof_free;
    long long launches[LFD_STAGES] = {0, 0, 0, 0};
    // pinned upload staging
    void *h_stage = nullptr;
    size_t h_stage_cap = 0;
    cudaEvent_t ev_stage = nullptr;
};

namespace {

lfd_status fail(lfd_ctx *ctx, lfd_status s, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return s;
}

#define LFD_CUDA(call)                                                                                        \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess)                                                                                \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? LFD_ERR_OOM : LFD_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                                   \
    } while (0)

lfd_status check_params(lfd_ctx *ctx, const lfd_params *p)
{
    if (!p) return fail(ctx, LFD_ERR_INVALID_ARG, "params is NULL");
    if (!(p->d_min > 0) || !(p->d_max > p->d_min) || !std::isfinite(p->d_max))
        return fail(ctx, LFD_ERR_INVALID_ARG, "depth range needs 0 < d_min < d_max (got %g, %g)", p->d_min, p->d_max);
    if (p->num_labels < 1 || p->num_labels > LFD_MAX_LABELS)
        return fail(ctx, LFD_ERR_INVALID_ARG, "num_labels %d outside 1..%d", p->num_labels, LFD_MAX_LABELS);
    if (p->iterations < 0 || p->iterations + p->warm_iter_offset > LFD_MAX_ITER_INDEX || p->warm_iter_offset < 0)
        return fail(ctx, LFD_ERR_INVALID_ARG, "iterations %d + warm offset %d outside 0..%d", p->iterations,
                    p->warm_iter_offset, LFD_MAX_ITER_INDEX);
    if (!(p->T > 0) || !(p->alpha > 0) || p->sigma < 0 || !(p->eta >= 0) || !(p->kernel_step_sp > 0) ||
        !(p->xy_eps >= 0))
        return fail(ctx, LFD_ERR_INVALID_ARG, "T, alpha, kernel_step_sp must be > 0; sigma, eta, xy_eps >= 0");
    if (p->max_neighbor_views < 0 || p->max_neighbor_views > LFD_MAXN)
        return fail(ctx, LFD_ERR_INVALID_ARG, "max_neighbor_views %d outside 0..%d", p->max_neighbor_views, LFD_MAXN);
    if (p->depth_domain != 0 && p->depth_domain != 1) return fail(ctx, LFD_ERR_INVALID_ARG, "depth_domain must be 0 or 1");
    if (p->sweep_frame != 0 && p->sweep_frame != 1) return fail(ctx, LFD_ERR_INVALID_ARG, "sweep_frame must be 0 or 1");
    if (p->kernel_size_init < 0) return fail(ctx, LFD_ERR_INVALID_ARG, "kernel_size_init must be >= 0");
    return LFD_OK;
}

lfd_status check_lightfield(lfd_ctx *ctx, const lfd_lightfield *lf, bool host_mem)
{
    if (!lf) return fail(ctx, LFD_ERR_INVALID_ARG, "light field is NULL");
    if (lf->num_views < 2 || lf->num_views > LFD_MAX_VIEWS)
        return fail(ctx, LFD_ERR_INVALID_ARG, "num_views %d outside 2..%d", lf->num_views, LFD_MAX_VIEWS);
    if (texel_bytes(lf->fmt) == 0) return fail(ctx, LFD_ERR_INVALID_ARG, "unknown pixel format %d", lf->fmt);
    if (!lf->cams || !lf->views || !lf->labels || !lf->grid_w || !lf->grid_h)
        return fail(ctx, LFD_ERR_INVALID_ARG, "NULL array in the light field");
    const int tb = texel_bytes(lf->fmt);
    long long px_total = 0;
    for (int v = 0; v < lf->num_views; v++) {
        const lfd_camera &c = lf->cams[v];
        if (c.width < 1 || c.height < 1 || c.width > LFD_MAX_DIM || c.height > LFD_MAX_DIM)
            return fail(ctx, LFD_ERR_INVALID_ARG, "view %d: size %dx%d outside 1..%d", v, c.width, c.height, LFD_MAX_DIM);
        if (c.K[3] != 0 || c.K[6] != 0 || c.K[7] != 0 || c.K[8] != 1 || !(c.K[0] != 0) || !(c.K[4] != 0) ||
            !std::isfinite(c.K[0] * c.K[4]))
            return fail(ctx, LFD_ERR_INVALID_ARG, "view %d: K must be pinhole [[fx,s,cx],[0,fy,cy],[0,0,1]] with fx,fy != 0", v);
        for (int k = 0; k < 9; k++)
            if (!std::isfinite(c.R[k]) || !std::isfinite(c.K[k])) return fail(ctx, LFD_ERR_INVALID_ARG, "view %d: non-finite camera", v);
        for (int k = 0; k < 3; k++)
            if (!std::isfinite(c.t[k])) return fail(ctx, LFD_ERR_INVALID_ARG, "view %d: non-finite camera", v);
        if (lf->grid_w[v] < 1 || lf->grid_h[v] < 1 || (long long)lf->grid_w[v] * lf->grid_h[v] > (1 << 22))
            return fail(ctx, LFD_ERR_INVALID_ARG, "view %d: superpixel grid %dx%d invalid", v, lf->grid_w[v], lf->grid_h[v]);
        if (!lf->views[v] || !lf->labels[v]) return fail(ctx, LFD_ERR_INVALID_ARG, "view %d: NULL image or label map", v);
        const long long pitch = (lf->view_pitch_bytes && lf->view_pitch_bytes[v]) ? lf->view_pitch_bytes[v]
                                                                                   : (long long)c.width * tb;
        if (pitch < (long long)c.width * tb || pitch % tb)
            return fail(ctx, LFD_ERR_INVALID_ARG, "view %d: pitch %lld too small or not a multiple of %d", v, pitch, tb);
        if (!host_mem && (((uintptr_t)lf->views[v] % tb) || ((uintptr_t)lf->labels[v] % 4)))
            return fail(ctx, LFD_ERR_INVALID_ARG, "view %d: image or label pointer misaligned", v);
        px_total += (long long)c.width * c.height;
    }
    if (px_total >= (1LL << 31)) return fail(ctx, LFD_ERR_INVALID_ARG, "more than 2^31 pixels in one light field");
    return LFD_OK;
}

void inv_pinhole(const double K[9], double Ki[9])
{
    const double fx = K[0], s = K[1], cx = K[2], fy = K[4], cy = K[5];
    Ki[0] = 1.0 / fx; Ki[1] = -s / (fx * fy); Ki[2] = (s * cy - cx * fy) / (fx * fy);
    Ki[3] = 0.0; Ki[4] = 1.0 / fy; Ki[5] = -cy / fy;
    Ki[6] = 0.0; Ki[7] = 0.0; Ki[8] = 1.0;
}

void mat_mul(const double A[9], const double B[9], double C[9])
{
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}

Consts make_consts(const lfd_params &p, int V, int fmt)
{
    Consts c{};
    c.V = V;
    c.L = p.num_labels;
    c.fmt = fmt;
    c.domain = p.depth_domain;
    c.jitter = p.jitter;
    c.term_mask = (int)p.term_mask;
    c.sweep_frame = p.sweep_frame;
    c.lf_index = p.lf_index;
    c.seed = p.seed;
    c.d_min = p.d_min;
    c.d_max = p.d_max;
    c.inv_dmin = 1.0 / p.d_min;
    c.inv_dmax = 1.0 / p.d_max;
    c.delta = (1.0 / p.d_min - 1.0 / p.d_max) / (double)p.num_labels;
    const double unit = fmt == LFD_RGBA8 ? 255.0 : 1.0;
    c.T = (float)(p.T * unit * unit);
    c.col_scale = (float)(1.0 / unit);
    const double log2e = 1.4426950408889634;
    c.k_col = (float)(log2e / (2.0 * p.alpha * p.alpha));
    double sigma = p.sigma;
    if (!(sigma > 0)) sigma = p.depth_domain == 0 ? 2.0 * c.delta : 2.0 * (p.d_max - p.d_min) / p.num_labels;
    c.k_sig = (float)(log2e / (2.0 * sigma * sigma));
    c.eta = (float)p.eta;
    c.xy_lo = (float)(1.0 / (1.0 + p.xy_eps));
    c.xy_hi = (float)(1.0 + p.xy_eps);
    return c;
}

lfd_status ensure_pinned(lfd_ctx *ctx, size_t bytes)
{
    if (ctx->ev_stage) LFD_CUDA(cudaEventSynchronize(ctx->ev_stage));   // previous upload has left the buffer
    if (ctx->h_stage_cap >= bytes) return LFD_OK;
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->h_stage_cap = 0;
    LFD_CUDA(cudaMallocHost(&ctx->h_stage, bytes));
    ctx->h_stage_cap = bytes;
    return LFD_OK;
}

lfd_status ensure_dev(lfd_ctx *ctx, void **ptr, size_t *cap, size_t bytes)
{
    if (*cap >= bytes) return LFD_OK;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    LFD_CUDA(cudaMalloc(ptr, bytes));
    *cap = bytes;
    return LFD_OK;
}

lfd_status set_device(lfd_ctx *ctx)
{
    LFD_CUDA(cudaSetDevice(ctx->device));
    return LFD_OK;
}

// -- tracing -----------------------------------------------------------------
cudaEvent_t prof_event(lfd_ctx *ctx)
{
    if (!ctx->prof_free.empty()) {
        cudaEvent_t e = ctx->prof_free.back();
        ctx->prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Runs `launch` (returns cudaError_t) bracketed by events when tracing.
template <typename F>
cudaError_t traced(lfd_ctx *ctx, int stage, cudaStream_t st, F launch)
{
    ctx->launches[stage]++;
    if (!ctx->prof) return launch();
    cudaEvent_t a = prof_event(ctx), b = prof_event(ctx);
    if (!a || !b) return launch();
    cudaEventRecord(a, st);
    cudaError_t e = launch();
    cudaEventRecord(b, st);
    ctx->prof_used.push_back({stage, {a, b}});
    return e;
}

// -- layout + workspace allocation -------------------------------------------
lfd_status plan_workspace(lfd_ctx *ctx, const lfd_lightfield *lf)
{
    Layout L;
    L.V = lf->num_views;
    for (int v = 0; v < L.V; v++) {
        const lfd_camera &c = lf->cams[v];
        L.W.push_back(c.width);
        L.H.push_back(c.height);
        L.GW.push_back(lf->grid_w[v]);
        L.GH.push_back(lf->grid_h[v]);
        L.S.push_back(lf->grid_w[v] * lf->grid_h[v]);
        L.sp_base.push_back(L.S_total);
        L.px_base.push_back(L.px_total);
        L.S_total += L.S.back();
        L.px_total += (long long)c.width * c.height;
        L.max_px = std::max(L.max_px, c.width * c.height);
    }
    const int V = L.V;
    const size_t S = L.S_total, P = (size_t)L.px_total;
    const int qb = quad_bytes(lf->fmt);
    size_t need = 0;
    auto add = [&](size_t b) { need = align_up(need, 256) + b; };
    add(sizeof(ViewDev) * V);
    add(sizeof(PairDev) * V * LFD_MAXN);
    add(2 * (size_t)V * (LFD_MAX_ITER_INDEX + 1) * LFD_MAX_RADII);
    add(4 * (size_t)V * (LFD_MAX_ITER_INDEX + 1));
    add(4 * S); add(4 * (S + 1)); add(4 * S); add(4 * P);
    add(8 * S); add(16 * S); add(16 * S); add(32 * S); add(16 * S); add(16 * S);
    add(sizeof(DevCounters));
    add(16 * S); add(16 * S); add(4 * S); add(8 * S); add(8 * S);
    for (int v = 0; v < V; v++) add((size_t)qb * L.W[v] * L.H[v]);
    for (int v = 0; v < V; v++) add((size_t)16 * L.W[v] * L.H[v]);
    need += 256;
    if (ctx->budget && need > ctx->budget)
        return fail(ctx, LFD_ERR_BUDGET, "workspace needs %zu bytes, budget is %llu", need,
                    (unsigned long long)ctx->budget);
    if (ctx->ws.cap < need) {
        if (ctx->ws.base) {
            LFD_CUDA(cudaDeviceSynchronize());
            cudaFree(ctx->ws.base);
        }
        ctx->ws.base = nullptr;
        ctx->ws.cap = 0;
        void *b = nullptr;
        cudaError_t e = cudaMalloc(&b, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, LFD_ERR_OOM, "cudaMalloc(%zu) failed: %s", need, cudaGetErrorString(e));
        }
        ctx->ws.base = (char *)b;
        ctx->ws.cap = need;
    }
    Arena &a = ctx->ws;
    a.used = 0;
    // host-built records first and contiguous: one upload from the pinned staging
    ctx->d_views = (ViewDev *)a.take(sizeof(ViewDev) * V);
    ctx->d_pairs = (PairDev *)a.take(sizeof(PairDev) * V * LFD_MAXN);
    ctx->d_radii = (short *)a.take(2 * (size_t)V * (LFD_MAX_ITER_INDEX + 1) * LFD_MAX_RADII);
    ctx->d_radii_cnt = (int *)a.take(4 * (size_t)V * (LFD_MAX_ITER_INDEX + 1));
    ctx->d_sp_view = (int *)a.take(4 * S);
    ctx->d_sp_off = (int *)a.take(4 * (S + 1));
    ctx->d_sp_cnt = (int *)a.take(4 * S);
    ctx->d_sp_pix = (unsigned *)a.take(4 * P);
    ctx->d_sp_ref = (int2 *)a.take(8 * S);
    ctx->d_sp_cen = (double2 *)a.take(16 * S);
    ctx->d_sp_col = (float4 *)a.take(16 * S);
    ctx->d_sp_g = (double4_32a *)a.take(32 * S);
    ctx->d_sp_rc = (float4 *)a.take(16 * S);
    ctx->d_bbox = (int4 *)a.take(16 * S);
    ctx->d_ctr = (DevCounters *)a.take(sizeof(DevCounters));
    ctx->d_planesA = (float4 *)a.take(16 * S);
    ctx->d_planesB = (float4 *)a.take(16 * S);
    ctx->d_label = (int *)a.take(4 * S);
    ctx->d_choice = (int *)a.take(8 * S);
    ctx->d_energy = (float *)a.take(8 * S);
    ctx->quads.assign(V, nullptr);
    ctx->maps.assign(V, nullptr);
    for (int v = 0; v < V; v++) ctx->quads[v] = a.take((size_t)qb * L.W[v] * L.H[v]);
    for (int v = 0; v < V; v++) ctx->maps[v] = (float4 *)a.take((size_t)16 * L.W[v] * L.H[v]);
    ctx->L = L;
    Workspace &w = ctx->w;
    w.views = ctx->d_views;
    w.pairs = ctx->d_pairs;
    w.sp_view = ctx->d_sp_view;
    w.sp_off = ctx->d_sp_off;
    w.sp_cnt = ctx->d_sp_cnt;
    w.sp_pix = ctx->d_sp_pix;
    w.sp_ref = ctx->d_sp_ref;
    w.sp_cen = ctx->d_sp_cen;
    w.sp_col = ctx->d_sp_col;
    w.sp_g = ctx->d_sp_g;
    w.sp_rc = ctx->d_sp_rc;
    w.radii = ctx->d_radii;
    w.radii_cnt = ctx->d_radii_cnt;
    w.ctr = ctx->d_ctr;
    w.S_total = L.S_total;
    w.px_total = L.px_total;
    return LFD_OK;
}

__global__ void k_fill_sp_view(int *sp_view, int base, int S, int v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S) sp_view[base + i] = v;
}

lfd_status set_input_impl(lfd_ctx *ctx, const lfd_lightfield *lf, const lfd_params *p, cudaStream_t st)
{
    lfd_status s;
    if ((s = check_params(ctx, p)) != LFD_OK) return s;
    if ((s = check_lightfield(ctx, lf, false)) != LFD_OK) return s;
    if ((s = plan_workspace(ctx, lf)) != LFD_OK) return s;
    const Layout &L = ctx->L;
    const int V = L.V;
    ctx->p = *p;
    ctx->fmt = lf->fmt;
    ctx->cams.assign(lf->cams, lf->cams + V);
    ctx->nnb = std::min(V - 1, p->max_neighbor_views > 0 ? p->max_neighbor_views : LFD_MAXN);
    neighbour_views(lf->cams, V, ctx->nnb, ctx->nbr);
    ctx->c = make_consts(*p, V, lf->fmt);

    // host records -> pinned staging -> device
    const size_t bytes_views = sizeof(ViewDev) * V, bytes_pairs = sizeof(PairDev) * V * LFD_MAXN;
    const size_t bytes_radii = 2 * (size_t)V * (LFD_MAX_ITER_INDEX + 1) * LFD_MAX_RADII;
    const size_t bytes_rcnt = 4 * (size_t)V * (LFD_MAX_ITER_INDEX + 1);
    const size_t o_pairs = align_up(bytes_views, 256), o_radii = align_up(o_pairs + bytes_pairs, 256),
                 o_rcnt = align_up(o_radii + bytes_radii, 256), total = o_rcnt + bytes_rcnt;
    if ((s = ensure_pinned(ctx, total)) != LFD_OK) return s;
    char *h = (char *)ctx->h_stage;
    memset(h, 0, total);
    ViewDev *hv = (ViewDev *)h;
    PairDev *hp = (PairDev *)(h + o_pairs);
    short *hr = (short *)(h + o_radii);
    int *hrc = (int *)(h + o_rcnt);
    std::vector<std::vector<double>> Kinv(V, std::vector<double>(9));
    for (int v = 0; v < V; v++) inv_pinhole(lf->cams[v].K, Kinv[v].data());
    for (int v = 0; v < V; v++) {
        const lfd_camera &cv = lf->cams[v];
        ViewDev &d = hv[v];
        d.W = L.W[v]; d.H = L.H[v]; d.GW = L.GW[v]; d.GH = L.GH[v];
        d.S = L.S[v]; d.sp_base = L.sp_base[v]; d.px_base = L.px_base[v];
        d.nnb = ctx->nnb;
        memcpy(d.Kinv, Kinv[v].data(), sizeof(d.Kinv));
        for (int k = 0; k < 3; k++) d.wz[k] = cv.R[3 * k + 2];
        d.labels = lf->labels[v];
        d.quad = ctx->quads[v];
        d.map = ctx->maps[v];
        // propagation kernel: Size_init in cells (Section IV-A: smallest image dimension by default)
        const double pitch = std::sqrt((double)d.W * d.H / ((double)d.GW * d.GH));
        const int size_px = p->kernel_size_init > 0 ? p->kernel_size_init : std::min(d.W, d.H);
        d.ksize_init = (int)std::floor((double)size_px / pitch);
        d.ksteps_init = (int)std::floor((double)d.ksize_init / p->kernel_step_sp + 0.5);
        for (int I = 0; I <= LFD_MAX_ITER_INDEX; I++) {
            const int n = kernel_radii(d.ksize_init, d.ksteps_init, I, nullptr, 0);
            if (n > LFD_MAX_RADII)
                return fail(ctx, LFD_ERR_INVALID_ARG, "propagation kernel of iteration %d has %d radii (max %d); "
                            "raise kernel_step_sp", I, n, LFD_MAX_RADII);
            int rr[LFD_MAX_RADII];
            kernel_radii(d.ksize_init, d.ksteps_init, I, rr, LFD_MAX_RADII);
            hrc[v * (LFD_MAX_ITER_INDEX + 1) + I] = n;
            for (int k = 0; k < n; k++) hr[((size_t)v * (LFD_MAX_ITER_INDEX + 1) + I) * LFD_MAX_RADII + k] = (short)rr[k];
        }
        for (int k = 0; k < ctx->nnb; k++) {
            const int i = ctx->nbr[(size_t)v * LFD_MAXN + k];
            const lfd_camera &ci = lf->cams[i];
            // R_rel = R_i R_v^T, t_rel = t_i - R_rel t_v, P = K_i R_rel K_v^-1, q = K_i t_rel
            double Rrel[9], tmp[9], P[9];
            for (int r = 0; r < 3; r++)
                for (int cc = 0; cc < 3; cc++)
                    Rrel[3 * r + cc] = ci.R[3 * r] * cv.R[3 * cc] + ci.R[3 * r + 1] * cv.R[3 * cc + 1] +
                                       ci.R[3 * r + 2] * cv.R[3 * cc + 2];
            double trel[3];
            for (int r = 0; r < 3; r++)
                trel[r] = ci.t[r] - (Rrel[3 * r] * cv.t[0] + Rrel[3 * r + 1] * cv.t[1] + Rrel[3 * r + 2] * cv.t[2]);
            mat_mul(ci.K, Rrel, tmp);
            mat_mul(tmp, Kinv[v].data(), P);
            PairDev &pd = hp[v * LFD_MAXN + k];
            pd.i = i;
            pd.Wi = L.W[i];
            pd.Hi = L.H[i];
            for (int r = 0; r < 9; r++) {
                pd.P[r] = P[r];
                pd.Pf[r] = (float)P[r];
            }
            for (int r = 0; r < 3; r++) {
                pd.q[r] = ci.K[3 * r] * trel[0] + ci.K[3 * r + 1] * trel[1] + ci.K[3 * r + 2] * trel[2];
                pd.qf[r] = (float)pd.q[r];
            }
            pd.quad_i = ctx->quads[i];
            pd.map_i = ctx->maps[i];
        }
    }
    if ((char *)ctx->d_pairs - (char *)ctx->d_views != (ptrdiff_t)o_pairs ||
        (char *)ctx->d_radii - (char *)ctx->d_views != (ptrdiff_t)o_radii ||
        (char *)ctx->d_radii_cnt - (char *)ctx->d_views != (ptrdiff_t)o_rcnt)
        return fail(ctx, LFD_ERR_STATE, "internal: workspace record layout mismatch");
    LFD_CUDA(cudaMemcpyAsync(ctx->d_views, h, total, cudaMemcpyHostToDevice, st));
    LFD_CUDA(cudaEventRecord(ctx->ev_stage, st));
    LFD_CUDA(cudaMemsetAsync(ctx->d_ctr, 0, sizeof(DevCounters), st));
    for (int v = 0; v < V; v++) {
        LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st, [&] {
            k_fill_sp_view<<<(L.S[v] + 255) / 256, 256, 0, st>>>(ctx->d_sp_view, L.sp_base[v], L.S[v], v);
            return cudaGetLastError();
        }));
    }

    ViewPtrs img;
    memset(&img, 0, sizeof(img));
    const int tb = texel_bytes(lf->fmt);
    for (int v = 0; v < V; v++) {
        img.p[v] = lf->views[v];
        img.pitch[v] = (lf->view_pitch_bytes && lf->view_pitch_bytes[v]) ? lf->view_pitch_bytes[v] : (long long)L.W[v] * tb;
    }
    LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st, [&] {
        return launch_sp_count(ctx->w, V, L.max_px, ctx->d_sp_cnt, ctx->d_bbox, st);
    }));
    LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st,
                    [&] { return launch_sp_scan(ctx->w, V, ctx->d_sp_cnt, ctx->d_sp_off, st); }));
    LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st, [&] {
        return launch_sp_collect(ctx->w, ctx->c, img, ctx->d_bbox, ctx->d_sp_cnt, ctx->d_sp_pix, ctx->d_sp_cen,
                                 ctx->d_sp_ref, ctx->d_sp_col, st);
    }));
    LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st, [&] { return launch_sp_minw(ctx->w, ctx->c, ctx->d_sp_col, st); }));
    LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st,
                    [&] { return launch_quads(ctx->w, V, L.max_px, lf->fmt, img, st); }));
    ctx->bound = true;
    return LFD_OK;
}

lfd_status need_bound(lfd_ctx *ctx)
{
    if (!ctx) return LFD_ERR_INVALID_ARG;
    if (!ctx->bound) return fail(ctx, LFD_ERR_STATE, "no light field bound: call lfd_set_input first");
    return LFD_OK;
}

lfd_status gather_planes(lfd_ctx *ctx, const float *const *src, float4 *dst, cudaStream_t st)
{
    if (!src) return fail(ctx, LFD_ERR_INVALID_ARG, "planes array is NULL");
    for (int v = 0; v < ctx->L.V; v++) {
        if (!src[v]) return fail(ctx, LFD_ERR_INVALID_ARG, "planes of view %d is NULL", v);
        LFD_CUDA(cudaMemcpyAsync(dst + ctx->L.sp_base[v], src[v], 16 * (size_t)ctx->L.S[v], cudaMemcpyDeviceToDevice, st));
    }
    return LFD_OK;
}

template <typename T>
lfd_status scatter(lfd_ctx *ctx, const T *src, T *const *dst, size_t per_sp, cudaStream_t st,
                   cudaMemcpyKind kind = cudaMemcpyDeviceToDevice)
{
    if (!dst) return LFD_OK;
    for (int v = 0; v < ctx->L.V; v++) {
        if (!dst[v]) continue;
        LFD_CUDA(cudaMemcpyAsync(dst[v], src + (size_t)ctx->L.sp_base[v] * per_sp, sizeof(T) * per_sp * ctx->L.S[v],
                                 kind, st));
    }
    return LFD_OK;
}

lfd_status rasterize_state(lfd_ctx *ctx, const float4 *planes, const OutPtrs *depth, cudaStream_t st)
{
    LFD_CUDA(traced(ctx, LFD_STAGE_RASTER, st,
                    [&] { return launch_plane_prep(ctx->w, ctx->c, planes, ctx->d_sp_g, ctx->d_sp_rc, st); }));
    LFD_CUDA(traced(ctx, LFD_STAGE_RASTER, st, [&] { return launch_rasterize(ctx->w, ctx->c, depth, st); }));
    return LFD_OK;
}

lfd_status iterate_flat(lfd_ctx *ctx, int iter, const float4 *in, float4 *out, int *choice, float *energy, cudaStream_t st)
{
    lfd_status s;
    if ((s = rasterize_state(ctx, in, nullptr, st)) != LFD_OK) return s;
    LFD_CUDA(traced(ctx, LFD_STAGE_PROPAGATE, st, [&] {
        return launch_propagate(ctx->w, ctx->c, iter + ctx->p.warm_iter_offset, in, out, choice, energy, st);
    }));
    return LFD_OK;
}

lfd_status estimate_impl(lfd_ctx *ctx, const lfd_lightfield *lf, const lfd_params *p, const float *const *warm,
                         float *const *planes_out, const OutPtrs *depth, cudaStream_t st, bool planes_to_host)
{
    lfd_status s;
    if ((s = set_input_impl(ctx, lf, p, st)) != LFD_OK) return s;
    if (warm) {
        if ((s = gather_planes(ctx, warm, ctx->d_planesA, st)) != LFD_OK) return s;
    } else {
        LFD_CUDA(traced(ctx, LFD_STAGE_SWEEP, st,
                        [&] { return launch_sweep(ctx->w, ctx->c, ctx->d_planesA, ctx->d_label, nullptr, st); }));
    }
    float4 *a = ctx->d_planesA, *b = ctx->d_planesB;
    for (int it = 1; it <= p->iterations; it++) {
        if ((s = iterate_flat(ctx, it, a, b, nullptr, nullptr, st)) != LFD_OK) return s;
        std::swap(a, b);
    }
    if ((s = rasterize_state(ctx, a, depth, st)) != LFD_OK) return s;
    if (planes_out) {
        if ((s = scatter<float>(ctx, (const float *)a, planes_out, 4, st,
                                planes_to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice)) != LFD_OK)
            return s;
    }
    return LFD_OK;
}

}  // namespace

// ===========================================================================
// exported C ABI
// ===========================================================================

extern "C" {

int32_t lfd_version(void) { return LFD_VERSION; }

void lfd_struct_sizes(int32_t *out)
{
    if (!out) return;
    out[0] = (int32_t)sizeof(lfd_camera);
    out[1] = (int32_t)sizeof(lfd_lightfield);
    out[2] = (int32_t)sizeof(lfd_params);
    out[3] = (int32_t)sizeof(lfd_query);
}

const char *lfd_status_string(lfd_status s)
{
    switch (s) {
    case LFD_OK: return "ok";
    case LFD_ERR_INVALID_ARG: return "invalid argument";
    case LFD_ERR_CUDA: return "CUDA error";
    case LFD_ERR_OOM: return "out of memory";
    case LFD_ERR_BUDGET: return "HBM budget exceeded";
    case LFD_ERR_TIMEOUT: return "timeout";
    case LFD_ERR_DEVICE_CHECK: return "device-side input check failed";
    case LFD_ERR_BUSY: return "busy";
    case LFD_ERR_STATE: return "wrong call order";
    default: return "unknown status";
    }
}

void lfd_params_default(lfd_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->d_min = 1.0;
    p->d_max = 10.0;
    p->num_labels = 64;
    p->iterations = 5;
    p->T = 0.04;
    p->sigma = 0.0;
    p->alpha = 0.1;
    p->eta = 0.5;
    p->kernel_size_init = 0;
    p->kernel_step_sp = 5.0;
    p->max_neighbor_views = 0;
    p->depth_domain = 0;
    p->jitter = 1;
    p->term_mask = 7;
    p->sweep_frame = 0;
    p->seed = 0x5EED;
    p->lf_index = 0;
    p->xy_eps = 0.0;
    p->warm_iter_offset = 0;
}

lfd_status lfd_create(lfd_ctx **out, int32_t device, uint64_t hbm_budget_bytes)
{
    if (!out) return LFD_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return LFD_ERR_INVALID_ARG;
    }
    lfd_ctx *ctx = new (std::nothrow) lfd_ctx();
    if (!ctx) return LFD_ERR_OOM;
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    if (cudaSetDevice(device) != cudaSuccess || cudaEventCreateWithFlags(&ctx->ev_stage, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return LFD_ERR_CUDA;
    }
    *out = ctx;
    return LFD_OK;
}

lfd_status lfd_destroy(lfd_ctx *ctx)
{
    if (!ctx) return LFD_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->ws.base) cudaFree(ctx->ws.base);
    if (ctx->d_cost) cudaFree(ctx->d_cost);
    if (ctx->d_stage_in) cudaFree(ctx->d_stage_in);
    if (ctx->d_stage_depth) cudaFree(ctx->d_stage_depth);
    if (ctx->d_q) cudaFree(ctx->d_q);
    if (ctx->d_qout) cudaFree(ctx->d_qout);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->ev_stage) cudaEventDestroy(ctx->ev_stage);
    for (auto &u : ctx->prof_used) {
        cudaEventDestroy(u.second.first);
        cudaEventDestroy(u.second.second);
    }
    for (cudaEvent_t e : ctx->prof_free) cudaEventDestroy(e);
    delete ctx;
    return LFD_OK;
}

const char *lfd_last_error(const lfd_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

lfd_status lfd_set_input(lfd_ctx *ctx, const lfd_lightfield *lf, const lfd_params *p, void *stream)
{
    if (!ctx) return LFD_ERR_INVALID_ARG;
    ctx->err.clear();
    lfd_status s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    ctx->bound = false;
    return set_input_impl(ctx, lf, p, (cudaStream_t)stream);
}

lfd_status lfd_num_superpixels(const lfd_ctx *ctx, int32_t view, int32_t *out)
{
    if (!ctx || !out) return LFD_ERR_INVALID_ARG;
    if (!ctx->bound) return LFD_ERR_STATE;
    if (view < 0 || view >= ctx->L.V) return LFD_ERR_INVALID_ARG;
    *out = ctx->L.S[view];
    return LFD_OK;
}

lfd_status lfd_plane_sweep(lfd_ctx *ctx, float *const *planes_out, int32_t *const *label_out, float *const *cost_out,
                           void *stream)
{
    lfd_status s;
    if ((s = need_bound(ctx)) != LFD_OK) return s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    if (!planes_out) return fail(ctx, LFD_ERR_INVALID_ARG, "planes_out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    float *cost = nullptr;
    if (cost_out) {
        const size_t need = sizeof(float) * (size_t)ctx->L.S_total * ctx->p.num_labels;
        if ((s = ensure_dev(ctx, (void **)&ctx->d_cost, &ctx->cost_cap, need)) != LFD_OK) return s;
        cost = ctx->d_cost;
    }
    LFD_CUDA(traced(ctx, LFD_STAGE_SWEEP, st,
                    [&] { return launch_sweep(ctx->w, ctx->c, ctx->d_planesA, ctx->d_label, cost, st); }));
    if ((s = scatter<float>(ctx, (const float *)ctx->d_planesA, planes_out, 4, st)) != LFD_OK) return s;
    if ((s = scatter<int32_t>(ctx, ctx->d_label, label_out, 1, st)) != LFD_OK) return s;
    if (cost_out && (s = scatter<float>(ctx, cost, cost_out, ctx->p.num_labels, st)) != LFD_OK) return s;
    return LFD_OK;
}

lfd_status lfd_rasterize(lfd_ctx *ctx, const float *const *planes, float *const *depth_out, void *stream)
{
    lfd_status s;
    if ((s = need_bound(ctx)) != LFD_OK) return s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = gather_planes(ctx, planes, ctx->d_planesA, st)) != LFD_OK) return s;
    OutPtrs dp;
    memset(&dp, 0, sizeof(dp));
    if (depth_out)
        for (int v = 0; v < ctx->L.V; v++) dp.p[v] = depth_out[v];
    return rasterize_state(ctx, ctx->d_planesA, depth_out ? &dp : nullptr, st);
}

lfd_status lfd_iterate(lfd_ctx *ctx, int32_t iter, const float *const *planes_in, float *const *planes_out,
                       int32_t *const *choice_out, float *const *energy_out, void *stream)
{
    lfd_status s;
    if ((s = need_bound(ctx)) != LFD_OK) return s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    if (iter < 1 || iter + ctx->p.warm_iter_offset > LFD_MAX_ITER_INDEX)
        return fail(ctx, LFD_ERR_INVALID_ARG, "iteration index %d outside 1..%d", iter,
                    LFD_MAX_ITER_INDEX - ctx->p.warm_iter_offset);
    if (!planes_out) return fail(ctx, LFD_ERR_INVALID_ARG, "planes_out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = gather_planes(ctx, planes_in, ctx->d_planesA, st)) != LFD_OK) return s;
    if ((s = iterate_flat(ctx, iter, ctx->d_planesA, ctx->d_planesB, choice_out ? ctx->d_choice : nullptr,
                          energy_out ? ctx->d_energy : nullptr, st)) != LFD_OK)
        return s;
    if ((s = scatter<float>(ctx, (const float *)ctx->d_planesB, planes_out, 4, st)) != LFD_OK) return s;
    if ((s = scatter<int32_t>(ctx, ctx->d_choice, choice_out, 2, st)) != LFD_OK) return s;
    if ((s = scatter<float>(ctx, ctx->d_energy, energy_out, 2, st)) != LFD_OK) return s;
    return LFD_OK;
}

lfd_status lfd_estimate(lfd_ctx *ctx, const lfd_lightfield *lf, const lfd_params *p, const float *const *warm_planes,
                        float *const *planes_out, float *const *depth_out, void *stream)
{
    if (!ctx) return LFD_ERR_INVALID_ARG;
    ctx->err.clear();
    lfd_status s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    if (!planes_out) return fail(ctx, LFD_ERR_INVALID_ARG, "planes_out is NULL");
    OutPtrs dp;
    memset(&dp, 0, sizeof(dp));
    if (depth_out && lf && lf->num_views <= LFD_MAX_VIEWS)
        for (int v = 0; v < lf->num_views; v++) dp.p[v] = depth_out[v];
    return estimate_impl(ctx, lf, p, warm_planes, planes_out, depth_out ? &dp : nullptr, (cudaStream_t)stream, false);
}

lfd_status lfd_estimate_host(lfd_ctx *ctx, const lfd_lightfield *lf_host, const lfd_params *p,
                             float *const *planes_out_host, float *const *depth_out_host, void *stream)
{
    if (!ctx) return LFD_ERR_INVALID_ARG;
    ctx->err.clear();
    lfd_status s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    if ((s = check_params(ctx, p)) != LFD_OK) return s;
    if ((s = check_lightfield(ctx, lf_host, true)) != LFD_OK) return s;
    if (!planes_out_host) return fail(ctx, LFD_ERR_INVALID_ARG, "planes_out_host is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const int V = lf_host->num_views, tb = texel_bytes(lf_host->fmt);
    size_t need_in = 0, need_depth = 0;
    std::vector<size_t> o_img(V), o_lab(V), o_dep(V);
    for (int v = 0; v < V; v++) {
        const size_t npx = (size_t)lf_host->cams[v].width * lf_host->cams[v].height;
        o_img[v] = need_in = align_up(need_in, 256);
        need_in += npx * tb;
        o_lab[v] = need_in = align_up(need_in, 256);
        need_in += npx * 4;
        o_dep[v] = need_depth;
        need_depth += npx;
    }
    if ((s = ensure_dev(ctx, &ctx->d_stage_in, &ctx->stage_in_cap, need_in)) != LFD_OK) return s;
    if (depth_out_host &&
        (s = ensure_dev(ctx, (void **)&ctx->d_stage_depth, &ctx->stage_depth_cap, need_depth * 4)) != LFD_OK)
        return s;
    std::vector<const void *> dv(V);
    std::vector<const int32_t *> dl(V);
    std::vector<int64_t> pitch(V);
    for (int v = 0; v < V; v++) {
        const int Wv = lf_host->cams[v].width, Hv = lf_host->cams[v].height;
        const size_t row = (size_t)Wv * tb;
        const long long hp = (lf_host->view_pitch_bytes && lf_host->view_pitch_bytes[v]) ? lf_host->view_pitch_bytes[v]
                                                                                         : (long long)row;
        char *dimg = (char *)ctx->d_stage_in + o_img[v];
        LFD_CUDA(cudaMemcpy2DAsync(dimg, row, lf_host->views[v], hp, row, Hv, cudaMemcpyHostToDevice, st));
        int32_t *dlab = (int32_t *)((char *)ctx->d_stage_in + o_lab[v]);
        LFD_CUDA(cudaMemcpyAsync(dlab, lf_host->labels[v], (size_t)Wv * Hv * 4, cudaMemcpyHostToDevice, st));
        dv[v] = dimg;
        dl[v] = dlab;
        pitch[v] = (int64_t)row;
    }
    lfd_lightfield lfd = *lf_host;
    lfd.views = dv.data();
    lfd.labels = dl.data();
    lfd.view_pitch_bytes = pitch.data();
    OutPtrs dp;
    memset(&dp, 0, sizeof(dp));
    if (depth_out_host)
        for (int v = 0; v < V; v++) dp.p[v] = ctx->d_stage_depth + o_dep[v];
    if ((s = estimate_impl(ctx, &lfd, p, nullptr, planes_out_host, depth_out_host ? &dp : nullptr, st, true)) != LFD_OK)
        return s;
    if (depth_out_host)
        for (int v = 0; v < V; v++)
            if (depth_out_host[v])
                LFD_CUDA(cudaMemcpyAsync(depth_out_host[v], dp.p[v],
                                         4 * (size_t)lf_host->cams[v].width * lf_host->cams[v].height,
                                         cudaMemcpyDeviceToHost, st));
    return LFD_OK;
}

lfd_status lfd_synchronize(lfd_ctx *ctx, void *stream)
{
    if (!ctx) return LFD_ERR_INVALID_ARG;
    lfd_status s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    LFD_CUDA(cudaStreamSynchronize(st));
    if (!ctx->bound || !ctx->d_ctr) return LFD_OK;
    DevCounters h;
    LFD_CUDA(cudaMemcpy(&h, ctx->d_ctr, sizeof(h), cudaMemcpyDeviceToHost));
    if (h.status) {
        const int st_bits = h.status;
        LFD_CUDA(cudaMemset(&ctx->d_ctr->status, 0, sizeof(int)));
        if (st_bits & DEV_ERR_LABEL)
            return fail(ctx, LFD_ERR_DEVICE_CHECK, "label outside [0, grid_w*grid_h) in view %d at pixel %d", h.bad_view,
                        h.bad_index);
        return fail(ctx, LFD_ERR_DEVICE_CHECK, "superpixel pixel count mismatch in view %d superpixel %d", h.bad_view,
                    h.bad_index);
    }
    return LFD_OK;
}

lfd_status lfd_counters(lfd_ctx *ctx, uint64_t *hypotheses, uint64_t *samples, void *stream)
{
    lfd_status s;
    if ((s = need_bound(ctx)) != LFD_OK) return s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    LFD_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    DevCounters h;
    LFD_CUDA(cudaMemcpy(&h, ctx->d_ctr, sizeof(h), cudaMemcpyDeviceToHost));
    if (hypotheses) *hypotheses = h.hyp;
    if (samples) *samples = h.samples;
    return LFD_OK;
}

lfd_status lfd_score(lfd_ctx *ctx, const float *const *state_planes, int32_t nq, const lfd_query *queries, float *out,
                     void *stream)
{
    lfd_status s;
    if ((s = need_bound(ctx)) != LFD_OK) return s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    if (nq < 0 || (nq > 0 && (!queries || !out))) return fail(ctx, LFD_ERR_INVALID_ARG, "bad query arguments");
    for (int i = 0; i < nq; i++)
        if (queries[i].view < 0 || queries[i].view >= ctx->L.V || queries[i].sp < 0 ||
            queries[i].sp >= ctx->L.S[queries[i].view])
            return fail(ctx, LFD_ERR_INVALID_ARG, "query %d names view %d superpixel %d outside the light field", i,
                        queries[i].view, queries[i].sp);
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = gather_planes(ctx, state_planes, ctx->d_planesA, st)) != LFD_OK) return s;
    if ((s = rasterize_state(ctx, ctx->d_planesA, nullptr, st)) != LFD_OK) return s;
    if (nq == 0) return LFD_OK;
    if (nq > ctx->q_cap) {
        if (ctx->d_q) cudaFree(ctx->d_q);
        if (ctx->d_qout) cudaFree(ctx->d_qout);
        ctx->d_q = nullptr;
        ctx->d_qout = nullptr;
        ctx->q_cap = 0;
        LFD_CUDA(cudaMalloc(&ctx->d_q, sizeof(lfd_query) * nq));
        LFD_CUDA(cudaMalloc(&ctx->d_qout, sizeof(float) * LFD_TERMS_STRIDE * (size_t)nq));
        ctx->q_cap = nq;
    }
    LFD_CUDA(cudaMemcpyAsync(ctx->d_q, queries, sizeof(lfd_query) * nq, cudaMemcpyHostToDevice, st));
    LFD_CUDA(launch_score(ctx->w, ctx->c, ctx->d_planesA, nq, ctx->d_q, ctx->d_qout, st));
    LFD_CUDA(cudaMemcpyAsync(out, ctx->d_qout, sizeof(float) * LFD_TERMS_STRIDE * (size_t)nq, cudaMemcpyDeviceToHost, st));
    LFD_CUDA(cudaStreamSynchronize(st));
    return LFD_OK;
}

lfd_status lfd_get_superpixels(lfd_ctx *ctx, int32_t view, int32_t *offsets, int32_t *pixels, float *stats,
                               int32_t *neighbours, void *stream)
{
    lfd_status s;
    if ((s = need_bound(ctx)) != LFD_OK) return s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    if (view < 0 || view >= ctx->L.V) return fail(ctx, LFD_ERR_INVALID_ARG, "view %d outside the light field", view);
    cudaStream_t st = (cudaStream_t)stream;
    LFD_CUDA(cudaStreamSynchronize(st));
    const int S = ctx->L.S[view], base = ctx->L.sp_base[view];
    const long long pxb = ctx->L.px_base[view];
    const int npx = ctx->L.W[view] * ctx->L.H[view];
    std::vector<int> off(S + 1);
    LFD_CUDA(cudaMemcpy(off.data(), ctx->d_sp_off + base, 4 * (size_t)(S + 1), cudaMemcpyDeviceToHost));
    if (offsets)
        for (int i = 0; i <= S; i++) offsets[i] = (int)(off[i] - pxb);
    if (pixels) {
        std::vector<unsigned> pk(npx);
        LFD_CUDA(cudaMemcpy(pk.data(), ctx->d_sp_pix + pxb, 4 * (size_t)npx, cudaMemcpyDeviceToHost));
        for (int i = 0; i < npx; i++) pixels[i] = (int)(pk[i] >> 16) * ctx->L.W[view] + (int)(pk[i] & 0xffff);
    }
    if (stats) {
        std::vector<double2> cen(S);
        std::vector<float4> col(S);
        std::vector<int> cnt(S);
        LFD_CUDA(cudaMemcpy(cen.data(), ctx->d_sp_cen + base, 16 * (size_t)S, cudaMemcpyDeviceToHost));
        LFD_CUDA(cudaMemcpy(col.data(), ctx->d_sp_col + base, 16 * (size_t)S, cudaMemcpyDeviceToHost));
        LFD_CUDA(cudaMemcpy(cnt.data(), ctx->d_sp_cnt + base, 4 * (size_t)S, cudaMemcpyDeviceToHost));
        for (int i = 0; i < S; i++) {
            float *r = stats + 8 * (size_t)i;
            r[0] = (float)cen[i].x; r[1] = (float)cen[i].y;
            r[2] = col[i].x; r[3] = col[i].y; r[4] = col[i].z; r[5] = col[i].w;
            r[6] = (float)cnt[i]; r[7] = 0.f;
        }
    }
    if (neighbours)
        for (int k = 0; k < LFD_MAXN; k++) neighbours[k] = ctx->nbr[(size_t)view * LFD_MAXN + k];
    return LFD_OK;
}

lfd_status lfd_profile_enable(lfd_ctx *ctx, int32_t enable)
{
    if (!ctx) return LFD_ERR_INVALID_ARG;
    ctx->prof = enable != 0;
    return LFD_OK;
}

lfd_status lfd_profile_read(lfd_ctx *ctx, double *ms_out, int64_t *launches_out)
{
    if (!ctx) return LFD_ERR_INVALID_ARG;
    lfd_status s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    double ms[LFD_STAGES] = {0, 0, 0, 0};
    for (auto &u : ctx->prof_used) {
        LFD_CUDA(cudaEventSynchronize(u.second.second));
        float t = 0.f;
        LFD_CUDA(cudaEventElapsedTime(&t, u.second.first, u.second.second));
        ms[u.first] += t;
        ctx->prof_free.push_back(u.second.first);
        ctx->prof_free.push_back(u.second.second);
    }
    ctx->prof_used.clear();
    for (int k = 0; k < LFD_STAGES; k++) {
        if (ms_out) ms_out[k] = ms[k];
        if (launches_out) launches_out[k] = ctx->launches[k];
        ctx->launches[k] = 0;
    }
    return LFD_OK;
}

lfd_status lfd_neighbor_views(const lfd_camera *cams, int32_t V, int32_t max_k, int32_t *out, int32_t *k_out)
{
    if (!cams || !out || V < 2 || V > LFD_MAX_VIEWS || max_k < 0 || max_k > LFD_MAXN) return LFD_ERR_INVALID_ARG;
    const int k = std::min(V - 1, max_k > 0 ? max_k : LFD_MAXN);
    std::vector<int> nb;
    neighbour_views(cams, V, k, nb);
    for (size_t i = 0; i < nb.size(); i++) out[i] = nb[i];
    if (k_out) *k_out = k;
    return LFD_OK;
}

int32_t lfd_kernel_offsets(int32_t size_init, int32_t steps_init, int32_t I, int32_t *dxdy, int32_t cap)
{
    const int nr = kernel_radii(size_init, steps_init, I, nullptr, 0);
    const int n = 9 + 8 * nr;
    if (!dxdy || n > cap) return n;
    std::vector<int> rr(std::max(nr, 1));
    kernel_radii(size_init, steps_init, I, rr.data(), nr);
    dxdy[0] = 0;
    dxdy[1] = 0;
    for (int d = 0; d < 8; d++) {
        dxdy[2 + 2 * d] = RDX[d];
        dxdy[3 + 2 * d] = RDY[d];
    }
    for (int k = 0; k < nr; k++)
        for (int d = 0; d < 8; d++) {
            dxdy[18 + 16 * k + 2 * d] = RDX[d] * rr[k];
            dxdy[19 + 16 * k + 2 * d] = RDY[d] * rr[k];
        }
    return n;
}

}  // extern "C"
