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
#include "lfd_slic.cuh"

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
    case LFD_RGBA_F16: case LFD_RGBA_BF16: return 24;
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

// Pinned host staging for uploads that must not block the caller: a ring of
// buffers, each reused only once the upload that last read it has finished,
// so a caller can queue several frames on a busy stream without waiting.
struct PinnedRing {
    static constexpr int N = 4;
    void *p[N] = {};
    size_t cap[N] = {};
    cudaEvent_t ev[N] = {};
    int cur = 0;
    cudaError_t init()
    {
        for (cudaEvent_t &e : ev) {
            const cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    }
    // advance to the next buffer, grown to `bytes`, after its last upload
    cudaError_t next(size_t bytes)
    {
        cur = (cur + 1) % N;
        cudaError_t r = cudaEventSynchronize(ev[cur]);
        if (r != cudaSuccess) return r;
        if (cap[cur] >= bytes) return cudaSuccess;
        if (p[cur]) cudaFreeHost(p[cur]);
        p[cur] = nullptr;
        cap[cur] = 0;
        r = cudaMallocHost(&p[cur], bytes);
        if (r == cudaSuccess) cap[cur] = bytes;
        return r;
    }
    void *buf() const { return p[cur]; }
    cudaEvent_t event() const { return ev[cur]; }
    void release()
    {
        for (int i = 0; i < N; i++) {
            if (ev[i]) cudaEventSynchronize(ev[i]);
            if (p[i]) cudaFreeHost(p[i]);
            if (ev[i]) cudaEventDestroy(ev[i]);
            p[i] = nullptr;
            ev[i] = nullptr;
        }
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
struct LfInfo {
    int first_view, V;
    lfd_params p;
};

struct lfd_ctx {
    int device = 0;
    int num_sms = 0;
    uint64_t budget = 0;
    std::string err;
    bool bound = false;
    Consts c{};
    Layout L;
    std::vector<LfInfo> lfs;
    std::vector<int> nbr;          // [V_total * 8] global view indices
    int fmt = 0;
    LaunchCfg lc{256, 1, 8, 1, 0, 32, ORDER_BANDS, 0};
    int max_pair_form = 2;         // largest homography specialisation allowed (lfd_set_pair_forms)
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
    int *d_order = nullptr, *d_order_sweep = nullptr, *d_hist = nullptr, *d_queue = nullptr;
    float **d_depth_ptrs = nullptr;
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
    long long launches[LFD_STAGES] = {};
    // pinned upload staging (records) and depth-pointer table
    PinnedRing stage;                // view/pair/radii records
    PinnedRing dtab;                 // depth-output pointer tables
    PinnedRing ftab;                 // fusion tables
    std::vector<lfd_camera> cams;    // cameras of the bound views (global order)
    void *d_slic = nullptr;          // SLIC scratch (CIELAB image, centres)
    size_t slic_cap = 0;
    unsigned *d_zbuf = nullptr;      // fusion z-buffers (one light field at a time)
    size_t zbuf_cap = 0;
    void *d_ftab = nullptr;
    size_t ftab_cap = 0;
    // CUDA graph of a batched frame and the pinned depth table it reads
    cudaGraphExec_t gexec = nullptr;
    uint64_t gsig = 0;
    long long glaunches[LFD_STAGES] = {};
    float **h_bdepth = nullptr;
    int h_bdepth_cap = 0;
    cudaEvent_t ev_bdepth = nullptr;
    uint64_t tuned_sig = 0;
    // sweep launches: superpixels of label-count class c at order_sweep[cls_base[c] ..+ cls_count[c])
    int cls_base[NSCLASS] = {}, cls_count[NSCLASS] = {};
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
    if (p->perturb_samples < 0 || p->perturb_samples > LFD_MAX_PERTURB || !(p->perturb_scale >= 0) ||
        !std::isfinite(p->perturb_scale))
        return fail(ctx, LFD_ERR_INVALID_ARG, "perturb_samples must be 0..%d and perturb_scale >= 0", LFD_MAX_PERTURB);
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
    }
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

// parameters of one light field into its view records
void view_params(ViewDev &d, const lfd_params &p, int fmt, int lf)
{
    d.lf = lf;
    d.L = p.num_labels;
    d.jitter = p.jitter;
    d.lf_index = p.lf_index;
    d.term_mask = (int)p.term_mask;
    d.iters = p.iterations;
    d.warm_off = p.warm_iter_offset;
    d.seed = p.seed;
    d.inv_dmin = 1.0 / p.d_min;
    d.inv_dmax = 1.0 / p.d_max;
    d.delta = (1.0 / p.d_min - 1.0 / p.d_max) / (double)p.num_labels;
    const double unit = fmt == LFD_RGBA8 ? 255.0 : 1.0;
    d.T = (float)(p.T * unit * unit);
    const double log2e = 1.4426950408889634;
    d.k_col = (float)(log2e / (2.0 * p.alpha * p.alpha));
    double sigma = p.sigma;
    if (!(sigma > 0)) sigma = p.depth_domain == 0 ? 2.0 * d.delta : 2.0 * (p.d_max - p.d_min) / p.num_labels;
    d.k_sig = (float)(log2e / (2.0 * sigma * sigma));
    d.col_gain = (float)std::sqrt((double)d.k_col);
    d.dep_gain = (float)std::sqrt((double)d.k_sig);
    d.eta = (float)p.eta;
    d.xy_lo = (float)(1.0 / (1.0 + p.xy_eps));
    d.xy_hi = (float)(1.0 + p.xy_eps);
    d.perturb_k = p.perturb_samples;
    d.perturb_scale = p.perturb_scale;
    d.sclass = 3 * label_class(p.num_labels);   // the pair form is added once the pairs are known
}

lfd_status ensure_pinned(lfd_ctx *ctx, size_t bytes)
{
    LFD_CUDA(ctx->stage.next(bytes));
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
cudaError_t traced(lfd_ctx *ctx, int stage, cudaStream_t st, F launch, int kernels = 1)
{
    ctx->launches[stage] += kernels;    // kernels the launch function enqueues
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
constexpr int ORDER_KEYS_HOST = ORDER_KEYS;   // keys of the work orders' counting sort

// Sizes of the bound views in call order (global numbering).
lfd_status make_layout(lfd_ctx *ctx, int n, const lfd_lightfield *lfs, Layout &L)
{
    L = Layout();
    for (int l = 0; l < n; l++)
        for (int v = 0; v < lfs[l].num_views; v++) {
            const lfd_camera &c = lfs[l].cams[v];
            L.W.push_back(c.width);
            L.H.push_back(c.height);
            L.GW.push_back(lfs[l].grid_w[v]);
            L.GH.push_back(lfs[l].grid_h[v]);
            L.S.push_back(lfs[l].grid_w[v] * lfs[l].grid_h[v]);
            L.sp_base.push_back(L.S_total);
            L.px_base.push_back(L.px_total);
            if ((long long)L.S_total + L.S.back() >= (1LL << 30))
                return fail(ctx, LFD_ERR_INVALID_ARG, "more than 2^30 superpixels in one call");
            L.S_total += L.S.back();
            L.px_total += (long long)c.width * c.height;
            L.max_px = std::max(L.max_px, c.width * c.height);
            L.V++;
        }
    if (L.px_total >= (1LL << 31)) return fail(ctx, LFD_ERR_INVALID_ARG, "more than 2^31 pixels in one call");
    return LFD_OK;
}

// Device workspace of a layout, in bytes (the arena carved by plan_workspace).
size_t workspace_need(const Layout &L, int fmt)
{
    const int V = L.V;
    const size_t S = L.S_total, P = (size_t)L.px_total;
    const int qb = quad_bytes(fmt);
    size_t need = 0;
    auto add = [&](size_t b) { need = align_up(need, 256) + b; };
    add(sizeof(ViewDev) * V);
    add(sizeof(PairDev) * V * LFD_MAXN);
    add(2 * (size_t)V * (LFD_MAX_ITER_INDEX + 1) * LFD_MAX_RADII);
    add(4 * (size_t)V * (LFD_MAX_ITER_INDEX + 1));
    add(4 * S); add(4 * (S + 1)); add(4 * S); add(4 * P);
    add(8 * S); add(16 * S); add(16 * S); add(32 * S); add(16 * S); add(16 * S);
    add(sizeof(DevCounters));
    add(4 * S); add(4 * S); add(4 * ORDER_KEYS_HOST); add(64); add(sizeof(float *) * V);
    add(16 * S); add(16 * S); add(4 * S); add(8 * S); add(8 * S);
    for (int v = 0; v < V; v++) add((size_t)qb * (L.W[v] + 1) * (L.H[v] + 1));
    for (int v = 0; v < V; v++) add((size_t)16 * L.W[v] * L.H[v]);
    return need + 256;
}

lfd_status plan_workspace(lfd_ctx *ctx, int n, const lfd_lightfield *lfs)
{
    Layout L;
    lfd_status s;
    if ((s = make_layout(ctx, n, lfs, L)) != LFD_OK) return s;
    const int V = L.V;
    const size_t S = L.S_total, P = (size_t)L.px_total;
    const int qb = quad_bytes(lfs[0].fmt);
    const size_t need = workspace_need(L, lfs[0].fmt);
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
        if (ctx->gexec) {                       // a captured graph points into the old arena
            cudaGraphExecDestroy(ctx->gexec);
            ctx->gexec = nullptr;
            ctx->gsig = 0;
        }
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
    ctx->d_order = (int *)a.take(4 * S);
    ctx->d_order_sweep = (int *)a.take(4 * S);
    ctx->d_hist = (int *)a.take(4 * ORDER_KEYS_HOST);
    ctx->d_queue = (int *)a.take(4 * QUEUE_INTS);
    ctx->d_depth_ptrs = (float **)a.take(sizeof(float *) * V);
    ctx->d_planesA = (float4 *)a.take(16 * S);
    ctx->d_planesB = (float4 *)a.take(16 * S);
    ctx->d_label = (int *)a.take(4 * S);
    ctx->d_choice = (int *)a.take(8 * S);
    ctx->d_energy = (float *)a.take(8 * S);
    ctx->quads.assign(V, nullptr);
    ctx->maps.assign(V, nullptr);
    for (int v = 0; v < V; v++) ctx->quads[v] = a.take((size_t)qb * (L.W[v] + 1) * (L.H[v] + 1));
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
    w.order = ctx->d_order;
    w.order_sweep = ctx->d_order_sweep;
    w.queue = ctx->d_queue;
    w.S_total = L.S_total;
    w.px_total = L.px_total;
    return LFD_OK;
}

__global__ void k_fill_sp_view(int *sp_view, int base, int S, int v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S) sp_view[base + i] = v;
}

// Host half of binding n light fields: validation, workspace, records staged in
// pinned memory.  Nothing is enqueued.
lfd_status plan_input(lfd_ctx *ctx, int n, const lfd_lightfield *lfs, const lfd_params *ps, bool host_mem)
{
    lfd_status s;
    if (n < 1 || !lfs || !ps) return fail(ctx, LFD_ERR_INVALID_ARG, "need at least one light field and its parameters");
    for (int l = 0; l < n; l++) {
        if ((s = check_params(ctx, &ps[l])) != LFD_OK) return s;
        if ((s = check_lightfield(ctx, &lfs[l], host_mem)) != LFD_OK) return s;
        if (lfs[l].fmt != lfs[0].fmt || ps[l].depth_domain != ps[0].depth_domain ||
            ps[l].sweep_frame != ps[0].sweep_frame)
            return fail(ctx, LFD_ERR_INVALID_ARG, "light fields of one call must share pixel format, depth domain "
                                                  "and sweep frame (light field %d differs)", l);
    }
    if ((s = plan_workspace(ctx, n, lfs)) != LFD_OK) return s;
    const Layout &L = ctx->L;
    const int V = L.V;
    ctx->fmt = lfs[0].fmt;
    ctx->lfs.clear();
    ctx->cams.clear();
    for (int l = 0; l < n; l++) ctx->cams.insert(ctx->cams.end(), lfs[l].cams, lfs[l].cams + lfs[l].num_views);
    ctx->nbr.assign((size_t)V * LFD_MAXN, -1);
    Consts c{};
    c.V = V;
    c.L = ps[0].num_labels;
    c.fmt = lfs[0].fmt;
    c.domain = ps[0].depth_domain;
    c.sweep_frame = ps[0].sweep_frame;
    c.col_scale = (float)(lfs[0].fmt == LFD_RGBA8 ? 1.0 / 255.0 : 1.0);
    ctx->c = c;

    const size_t bytes_views = sizeof(ViewDev) * V, bytes_pairs = sizeof(PairDev) * V * LFD_MAXN;
    const size_t bytes_radii = 2 * (size_t)V * (LFD_MAX_ITER_INDEX + 1) * LFD_MAX_RADII;
    const size_t bytes_rcnt = 4 * (size_t)V * (LFD_MAX_ITER_INDEX + 1);
    const size_t o_pairs = align_up(bytes_views, 256), o_radii = align_up(o_pairs + bytes_pairs, 256),
                 o_rcnt = align_up(o_radii + bytes_radii, 256), total = o_rcnt + bytes_rcnt;
    if ((char *)ctx->d_pairs - (char *)ctx->d_views != (ptrdiff_t)o_pairs ||
        (char *)ctx->d_radii - (char *)ctx->d_views != (ptrdiff_t)o_radii ||
        (char *)ctx->d_radii_cnt - (char *)ctx->d_views != (ptrdiff_t)o_rcnt)
        return fail(ctx, LFD_ERR_STATE, "internal: workspace record layout mismatch");
    if ((s = ensure_pinned(ctx, total)) != LFD_OK) return s;
    char *h = (char *)ctx->stage.buf();
    memset(h, 0, total);
    ViewDev *hv = (ViewDev *)h;
    PairDev *hp = (PairDev *)(h + o_pairs);
    short *hr = (short *)(h + o_radii);
    int *hrc = (int *)(h + o_rcnt);
    const int tb = texel_bytes(lfs[0].fmt);
    int gv = 0;
    for (int l = 0; l < n; l++) {
        const lfd_lightfield &lf = lfs[l];
        const lfd_params &p = ps[l];
        ctx->lfs.push_back({gv, lf.num_views, p});
        const int nnb = std::min(lf.num_views - 1, p.max_neighbor_views > 0 ? p.max_neighbor_views : LFD_MAXN);
        std::vector<int> nb;
        neighbour_views(lf.cams, lf.num_views, nnb, nb);
        std::vector<std::vector<double>> Kinv(lf.num_views, std::vector<double>(9));
        for (int v = 0; v < lf.num_views; v++) inv_pinhole(lf.cams[v].K, Kinv[v].data());
        for (int v = 0; v < lf.num_views; v++, gv++) {
            const lfd_camera &cv = lf.cams[v];
            ViewDev &d = hv[gv];
            d.W = L.W[gv]; d.H = L.H[gv]; d.GW = L.GW[gv]; d.GH = L.GH[gv];
            d.S = L.S[gv]; d.sp_base = L.sp_base[gv]; d.px_base = L.px_base[gv];
            d.nnb = nnb;
            memcpy(d.Kinv, Kinv[v].data(), sizeof(d.Kinv));
            for (int k = 0; k < 3; k++) d.wz[k] = cv.R[3 * k + 2];
            d.labels = lf.labels[v];
            d.img = lf.views[v];
            d.pitch = (lf.view_pitch_bytes && lf.view_pitch_bytes[v]) ? lf.view_pitch_bytes[v] : (long long)d.W * tb;
            d.quad = ctx->quads[gv];
            d.map = ctx->maps[gv];
            view_params(d, p, lf.fmt, l);
            d.lv = v;
            // propagation kernel: Size_init in cells (Section IV-A: smallest image dimension by default)
            const double pitch = std::sqrt((double)d.W * d.H / ((double)d.GW * d.GH));
            const int size_px = p.kernel_size_init > 0 ? p.kernel_size_init : std::min(d.W, d.H);
            d.ksize_init = (int)std::floor((double)size_px / pitch);
            d.ksteps_init = (int)std::floor((double)d.ksize_init / p.kernel_step_sp + 0.5);
            for (int I = 0; I <= LFD_MAX_ITER_INDEX; I++) {
                const int nr = kernel_radii(d.ksize_init, d.ksteps_init, I, nullptr, 0);
                if (nr > LFD_MAX_RADII)
                    return fail(ctx, LFD_ERR_INVALID_ARG, "propagation kernel of iteration %d has %d radii (max %d); "
                                "raise kernel_step_sp", I, nr, LFD_MAX_RADII);
                int rr[LFD_MAX_RADII];
                kernel_radii(d.ksize_init, d.ksteps_init, I, rr, LFD_MAX_RADII);
                hrc[gv * (LFD_MAX_ITER_INDEX + 1) + I] = nr;
                for (int k = 0; k < nr; k++)
                    hr[((size_t)gv * (LFD_MAX_ITER_INDEX + 1) + I) * LFD_MAX_RADII + k] = (short)rr[k];
            }
            for (int k = 0; k < nnb; k++) {
                const int i = nb[(size_t)v * LFD_MAXN + k];
                const int gi = ctx->lfs[l].first_view + i;
                ctx->nbr[(size_t)gv * LFD_MAXN + k] = gi;
                const lfd_camera &ci = lf.cams[i];
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
                PairDev &pd = hp[gv * LFD_MAXN + k];
                pd.i = gi;
                pd.Wi = L.W[gi];
                pd.Hi = L.H[gi];
                for (int r = 0; r < 9; r++) {
                    pd.P[r] = P[r];
                    pd.Pf[r] = (float)P[r];
                }
                for (int r = 0; r < 3; r++) {
                    pd.q[r] = ci.K[3 * r] * trel[0] + ci.K[3 * r + 1] * trel[1] + ci.K[3 * r + 2] * trel[2];
                    pd.qf[r] = (float)pd.q[r];
                }
                pd.quad_i = ctx->quads[gi];
                pd.map_i = ctx->maps[gi];
            }
        }
    }
    // affine pairs: P row 3 = (0, 0, P22) and q_z = 0, so A(g) = P + q g^T keeps
    // row 3 = (0, 0, P22) for every plane g (cameras with parallel optical axes
    // and equal z in the reference frame, e.g. planar arrays)
    // translation pairs: affine with P's upper 2 x 2 block = P22 I to within
    // 1e-12 relative (rectified cameras with equal intrinsics): a pixel offset
    // du < 2^16 then moves by less than 1e-7 px against the exact homography
    // The propagation takes one form for the whole input, the sweep one per
    // view (its sweep class), so that a batch of mixed rigs sweeps each view
    // with the form of its own pairs.
    int affine = 1, shift = 1;
    for (int v = 0; v < V; v++) {
        int aff_v = 1, shift_v = 1;
        for (int k = 0; k < LFD_MAXN; k++) {
            if (ctx->nbr[(size_t)v * LFD_MAXN + k] < 0) continue;
            const PairDev &pd = hp[v * LFD_MAXN + k];
            if (pd.P[6] != 0.0 || pd.P[7] != 0.0 || pd.q[2] != 0.0) aff_v = 0;
            const double e = 1e-12 * std::fabs(pd.P[8]);
            if (!(pd.P[8] > 0.0) || std::fabs(pd.P[0] - pd.P[8]) > e || std::fabs(pd.P[4] - pd.P[8]) > e ||
                std::fabs(pd.P[1]) > e || std::fabs(pd.P[3]) > e)
                shift_v = 0;
        }
        const int pf = std::min(aff_v ? (shift_v ? 2 : 1) : 0, ctx->max_pair_form);
        hv[v].sclass += ctx->c.sweep_frame ? 0 : pf;     // world-frame sweeps: general form
        affine &= aff_v;
        shift &= shift_v;
    }
    ctx->c.affine = affine && ctx->max_pair_form >= 1;
    ctx->c.shift = affine && shift && ctx->max_pair_form >= 2;
    // the sweep order is partitioned by sweep class, classes ascending
    for (int k = 0; k < NSCLASS; k++) ctx->cls_count[k] = 0;
    for (int v = 0; v < V; v++) ctx->cls_count[hv[v].sclass] += L.S[v];
    for (int k = 0, b = 0; k < NSCLASS; k++) {
        ctx->cls_base[k] = b;
        b += ctx->cls_count[k];
    }
    return LFD_OK;
}

// Work orders of the persistent launches (k_superpixels.cu): the sweep's by
// size class and row band, then partitioned by label-count class when the
// bound light fields have several (d_order serves as the scratch of that
// pass before it receives the propagation's order).
lfd_status build_orders(lfd_ctx *ctx, cudaStream_t st)
{
    const int bands = ctx->lc.order_bands;
    int classes = 0;
    for (int k = 0; k < NSCLASS; k++) classes += ctx->cls_count[k] > 0;
    if (classes > 1) {
        LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st, [&] {
            return launch_sp_order(ctx->w, ctx->d_order, ctx->d_hist, 1, bands, nullptr, st);
        }, 2));
        LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st, [&] {
            return launch_sp_order(ctx->w, ctx->d_order_sweep, ctx->d_hist, 2, bands, ctx->d_order, st);
        }, 2));
    } else {
        LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st, [&] {
            return launch_sp_order(ctx->w, ctx->d_order_sweep, ctx->d_hist, 1, bands, nullptr, st);
        }, 2));
    }
    LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st, [&] {
        return launch_sp_order(ctx->w, ctx->d_order, ctx->d_hist, 0, bands, nullptr, st);
    }, 2));
    return LFD_OK;
}

// Device half: upload the staged records and build superpixels, textures and
// the cost order.  Capturable (no allocation, no synchronisation).
lfd_status enqueue_input(lfd_ctx *ctx, cudaStream_t st, bool record_event)
{
    const Layout &L = ctx->L;
    const int V = L.V;
    const size_t total = (char *)(ctx->d_radii_cnt + (size_t)V * (LFD_MAX_ITER_INDEX + 1)) - (char *)ctx->d_views;
    LFD_CUDA(cudaMemcpyAsync(ctx->d_views, ctx->stage.buf(), total, cudaMemcpyHostToDevice, st));
    if (record_event) LFD_CUDA(cudaEventRecord(ctx->stage.event(), st));
    LFD_CUDA(cudaMemsetAsync(ctx->d_ctr, 0, sizeof(DevCounters), st));
    for (int v = 0; v < V; v++) {
        LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st, [&] {
            k_fill_sp_view<<<(L.S[v] + 255) / 256, 256, 0, st>>>(ctx->d_sp_view, L.sp_base[v], L.S[v], v);
            return cudaGetLastError();
        }));
    }
    LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st, [&] {
        return launch_sp_count(ctx->w, V, L.max_px, ctx->d_sp_cnt, ctx->d_bbox, st);
    }, 2));
    LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st,
                    [&] { return launch_sp_scan(ctx->w, V, ctx->d_sp_cnt, ctx->d_sp_off, st); }));
    LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st, [&] {
        return launch_sp_collect(ctx->w, ctx->c, ctx->d_bbox, ctx->d_sp_cnt, ctx->d_sp_pix, ctx->d_sp_cen,
                                 ctx->d_sp_ref, ctx->d_sp_col, st);
    }));
    LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st, [&] { return launch_sp_minw(ctx->w, ctx->c, ctx->d_sp_col, st); }));
    int max_quads = 0;
    for (int v = 0; v < V; v++) max_quads = std::max(max_quads, (L.W[v] + 1) * (L.H[v] + 1));
    LFD_CUDA(traced(ctx, LFD_STAGE_SUPERPIXELS, st, [&] { return launch_quads(ctx->w, V, max_quads, ctx->fmt, st); }));
    // work orders: propagation by descending slot class, the sweep by descending
    // power-of-two size class, index order inside a class
    const lfd_status so = build_orders(ctx, st);
    if (so != LFD_OK) return so;
    return LFD_OK;
}

lfd_status set_input_multi(lfd_ctx *ctx, int n, const lfd_lightfield *lfs, const lfd_params *ps, cudaStream_t st)
{
    lfd_status s;
    ctx->bound = false;
    if (ctx->gexec) {               // the staging a captured graph reads is about to change
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
        ctx->gsig = 0;
    }
    if ((s = plan_input(ctx, n, lfs, ps, false)) != LFD_OK) return s;
    if ((s = enqueue_input(ctx, st, true)) != LFD_OK) return s;
    ctx->bound = true;
    return LFD_OK;
}

lfd_status need_bound(lfd_ctx *ctx)
{
    if (!ctx) return LFD_ERR_INVALID_ARG;
    if (!ctx->bound) return fail(ctx, LFD_ERR_STATE, "no light field bound: call lfd_set_input first");
    return LFD_OK;
}

lfd_status gather_planes(lfd_ctx *ctx, const float *const *src, float4 *dst, cudaStream_t st, bool allow_null = false)
{
    if (!src) return fail(ctx, LFD_ERR_INVALID_ARG, "planes array is NULL");
    for (int v = 0; v < ctx->L.V; v++) {
        if (!src[v]) {
            if (allow_null) continue;
            return fail(ctx, LFD_ERR_INVALID_ARG, "planes of view %d is NULL", v);
        }
        LFD_CUDA(cudaMemcpyAsync(dst + ctx->L.sp_base[v], src[v], 16 * (size_t)ctx->L.S[v], cudaMemcpyDeviceToDevice, st));
    }
    return LFD_OK;
}

template <typename T>
lfd_status scatter(lfd_ctx *ctx, const T *src, T *const *dst, size_t per_sp, cudaStream_t st,
                   cudaMemcpyKind kind = cudaMemcpyDeviceToDevice, int first_view = 0, int nviews = -1)
{
    if (!dst) return LFD_OK;
    if (nviews < 0) nviews = ctx->L.V;
    for (int k = 0; k < nviews; k++) {
        const int v = first_view + k;
        if (!dst[k]) continue;
        LFD_CUDA(cudaMemcpyAsync(dst[k], src + (size_t)ctx->L.sp_base[v] * per_sp, sizeof(T) * per_sp * ctx->L.S[v],
                                 kind, st));
    }
    return LFD_OK;
}

// Upload a per-view table of depth-output pointers (NULL entries allowed).
lfd_status upload_depth_ptrs(lfd_ctx *ctx, float *const *per_view, cudaStream_t st, float ***dev_out)
{
    *dev_out = nullptr;
    if (!per_view) return LFD_OK;
    const int V = ctx->L.V;
    LFD_CUDA(ctx->dtab.next(sizeof(float *) * V));
    float **h = (float **)ctx->dtab.buf();
    for (int v = 0; v < V; v++) h[v] = per_view[v];
    LFD_CUDA(cudaMemcpyAsync(ctx->d_depth_ptrs, h, sizeof(float *) * V, cudaMemcpyHostToDevice, st));
    LFD_CUDA(cudaEventRecord(ctx->dtab.event(), st));
    *dev_out = ctx->d_depth_ptrs;
    return LFD_OK;
}

lfd_status rasterize_state(lfd_ctx *ctx, const float4 *planes, float *const *depth_dev, cudaStream_t st)
{
    LFD_CUDA(traced(ctx, LFD_STAGE_RASTER, st,
                    [&] { return launch_plane_prep(ctx->w, ctx->c, planes, ctx->d_sp_g, ctx->d_sp_rc, st); }));
    LFD_CUDA(traced(ctx, LFD_STAGE_RASTER, st, [&] { return launch_rasterize(ctx->w, ctx->c, depth_dev, st); }));
    return LFD_OK;
}

// One sweep launch per sweep class present (label-count class x pair form),
// CTAs as wide as the class's label count (at most lc.sweep_threads).
lfd_status run_sweep(lfd_ctx *ctx, float *cost, cudaStream_t st)
{
    if (ctx->lc.sweep_persistent) LFD_CUDA(cudaMemsetAsync(ctx->d_queue, 0, 4 * QUEUE_INTS, st));
    for (int k = 0; k < NSCLASS; k++) {
        if (!ctx->cls_count[k]) continue;
        const int threads = std::min(LCLASS_THREADS[k / 3], ctx->lc.sweep_threads);
        Consts c = ctx->c;                   // the class's pair form
        c.affine = k % 3 >= 1;
        c.shift = k % 3 == 2;
        LFD_CUDA(traced(ctx, LFD_STAGE_SWEEP, st, [&] {
            return launch_sweep(ctx->w, c, ctx->lc, threads, ctx->cls_base[k], ctx->cls_count[k], 4 + k,
                                ctx->d_planesA, ctx->d_label, cost, st);
        }));
    }
    return LFD_OK;
}

// One iteration over every bound view.  In a frame (`frame`), a view whose
// light field has already run its own iteration count passes its plane through.
lfd_status iterate_flat(lfd_ctx *ctx, int iter, const float4 *in, float4 *out, int *choice, float *energy,
                        cudaStream_t st, bool frame = false)
{
    lfd_status s;
    if ((s = rasterize_state(ctx, in, nullptr, st)) != LFD_OK) return s;
    if (ctx->lc.prop_persistent) LFD_CUDA(cudaMemsetAsync(ctx->d_queue, 0, 4 * QUEUE_INTS, st));
    Consts c = ctx->c;
    c.batch_iters = frame ? 1 : 0;
    LFD_CUDA(traced(ctx, LFD_STAGE_PROPAGATE, st, [&] {
        return launch_propagate(ctx->w, c, ctx->lc, iter, in, out, choice, energy, st);
    }));
    return LFD_OK;
}

int max_iterations(const lfd_ctx *ctx)
{
    int m = 0;
    for (const LfInfo &l : ctx->lfs) m = std::max(m, l.p.iterations);
    return m;
}

// The device work of one frame after the inputs are bound: sweep (or warm
// planes), all iterations, final rasterisation, planes out.  warm: NULL (every
// view cold) or one planes pointer per bound view, NULL for a cold view (the
// sweep leaves out the views marked sweep_skip, whose planes are gathered
// after it).  Capturable.
lfd_status enqueue_frame(lfd_ctx *ctx, const float *const *warm, float *const *const *planes_out,
                         float *const *depth_dev, cudaStream_t st, cudaMemcpyKind out_kind)
{
    lfd_status s;
    bool all_warm = warm != nullptr;
    if (warm)
        for (int v = 0; v < ctx->L.V; v++) all_warm = all_warm && warm[v] != nullptr;
    if (!all_warm)
        if ((s = run_sweep(ctx, nullptr, st)) != LFD_OK) return s;
    if (warm)
        if ((s = gather_planes(ctx, warm, ctx->d_planesA, st, true)) != LFD_OK) return s;
    float4 *a = ctx->d_planesA, *b = ctx->d_planesB;
    const int iters = max_iterations(ctx);
    for (int it = 1; it <= iters; it++) {
        if ((s = iterate_flat(ctx, it, a, b, nullptr, nullptr, st, true)) != LFD_OK) return s;
        std::swap(a, b);
    }
    if ((s = rasterize_state(ctx, a, depth_dev, st)) != LFD_OK) return s;
    if (planes_out)
        for (size_t l = 0; l < ctx->lfs.size(); l++)
            if ((s = scatter<float>(ctx, (const float *)a, planes_out[l], 4, st, out_kind, ctx->lfs[l].first_view,
                                    ctx->lfs[l].V)) != LFD_OK)
                return s;
    return LFD_OK;
}

// Launch-shape autotuner: times each sweep and propagate variant on the bound
// input (one warm-up run, then the median of three) and keeps the fastest.
// Axes: sweep threads 128/256 x grid/persistent x row bands 1/16 of the
// sweep's work order; propagation CTAs per SM 7/8 x grid/persistent
// warps/cooperative CTAs x candidates per pass 16/32 x row bands 1/16
// (timed on the first and the last iteration of the input).
// Results do not depend on the shape (per-superpixel work is the same).
lfd_status autotune(lfd_ctx *ctx, cudaStream_t st)
{
    const bool prof = ctx->prof;
    ctx->prof = false;
    cudaEvent_t e0, e1;
    LFD_CUDA(cudaEventCreate(&e0));
    LFD_CUDA(cudaEventCreate(&e1));
    auto time_it = [&](auto &&fn, float &ms) -> lfd_status {
        lfd_status s;
        float t[3];
        if ((s = fn()) != LFD_OK) return s;
        for (int r = 0; r < 3; r++) {
            LFD_CUDA(cudaEventRecord(e0, st));
            if ((s = fn()) != LFD_OK) return s;
            LFD_CUDA(cudaEventRecord(e1, st));
            LFD_CUDA(cudaEventSynchronize(e1));
            LFD_CUDA(cudaEventElapsedTime(&t[r], e0, e1));
        }
        std::sort(t, t + 3);
        ms = t[1];
        return LFD_OK;
    };
    auto order = [&](int mode, int bands) -> lfd_status {    // mode 0: propagation, 1: sweep orders
        const int keep = ctx->lc.order_bands;
        ctx->lc.order_bands = bands;
        lfd_status so = build_orders(ctx, st);
        ctx->lc.order_bands = keep;
        (void)mode;
        return so;
    };
    lfd_status s;
    LaunchCfg best = ctx->lc;
    float best_ms = 1e30f;
    const int th[2] = {128, 256}, bands[2] = {1, ORDER_BANDS};
    int sweep_bands = ORDER_BANDS, prop_bands = ORDER_BANDS;
    for (int bi = 0; bi < 2; bi++) {
        if ((s = order(1, bands[bi])) != LFD_OK) return s;
        for (int pi = 0; pi < 2; pi++)
            for (int ti = 0; ti < 2; ti++) {
                ctx->lc.sweep_threads = th[ti];
                ctx->lc.sweep_persistent = pi;
                float ms = 0;
                if ((s = time_it([&] { return run_sweep(ctx, nullptr, st); }, ms)) != LFD_OK) return s;
                if (ms < best_ms) {
                    best_ms = ms;
                    best.sweep_threads = th[ti];
                    best.sweep_persistent = pi;
                    sweep_bands = bands[bi];
                }
            }
    }
    ctx->lc.sweep_threads = best.sweep_threads;
    ctx->lc.sweep_persistent = best.sweep_persistent;
    if ((s = order(1, sweep_bands)) != LFD_OK) return s;
    if ((s = run_sweep(ctx, nullptr, st)) != LFD_OK) return s;
    if ((s = rasterize_state(ctx, ctx->d_planesA, nullptr, st)) != LFD_OK) return s;
    best_ms = 1e30f;
    const int pb[2] = {7, 8}, cb[2] = {16, 32};
    int it_last = 1;
    for (const LfInfo &l : ctx->lfs) it_last = std::max(it_last, l.p.iterations);
    for (int bi = 0; bi < 2; bi++) {
        if ((s = order(0, bands[bi])) != LFD_OK) return s;
        for (int pi = 0; pi < 3; pi++)        // grid, persistent warps, cooperative CTAs
            for (int ki = 0; ki < 2; ki++)
                for (int ci = 0; ci < 2; ci++) {
                    ctx->lc.prop_blocks = pb[ki];
                    ctx->lc.prop_persistent = pi > 0;
                    ctx->lc.prop_coop = pi == 2;
                    ctx->lc.prop_batch = cb[ci];
                    float ms = 0;
                    // the first and the last iteration: the candidate count falls with the
                    // iteration index, and a shape can win on the first and lose on the rest
                    auto fn = [&]() -> lfd_status {
                        for (int it : {1, it_last}) {
                            if (ctx->lc.prop_persistent) LFD_CUDA(cudaMemsetAsync(ctx->d_queue, 0, 4 * QUEUE_INTS, st));
                            LFD_CUDA(launch_propagate(ctx->w, ctx->c, ctx->lc, it, ctx->d_planesA, ctx->d_planesB,
                                                      nullptr, nullptr, st));
                            if (it_last == 1) break;
                        }
                        return LFD_OK;
                    };
                    if ((s = time_it(fn, ms)) != LFD_OK) return s;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best.prop_blocks = pb[ki];
                        best.prop_persistent = pi > 0;
                        best.prop_coop = pi == 2;
                        best.prop_batch = cb[ci];
                        prop_bands = bands[bi];
                    }
                }
    }
    // one band count serves both orders (enqueue_input builds both with it):
    // the propagation's choice, the larger share of a frame's time
    best.order_bands = prop_bands;
    ctx->lc = best;
    if ((s = order(0, prop_bands)) != LFD_OK) return s;
    if ((s = order(1, prop_bands)) != LFD_OK) return s;
    (void)sweep_bands;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->prof = prof;
    return LFD_OK;
}

uint64_t mix64(uint64_t h, uint64_t v)
{
    h ^= v + 0x9E3779B97F4A7C15ULL + (h << 6) + (h >> 2);
    return h;
}

uint64_t hash_bytes(uint64_t h, const void *p, size_t n)
{
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < n; i++) h = mix64(h, b[i]);
    return h;
}

// signature of a batched call: every pointer, size, camera and parameter
uint64_t batch_signature(int n, const lfd_lightfield *lfs, const lfd_params *ps, float *const *const *planes_out,
                         float *const *const *depth_out, const lfd_batch_options *opt)
{
    uint64_t h = mix64(0x1234, (uint64_t)n);
    for (int l = 0; l < n; l++) {
        const lfd_lightfield &lf = lfs[l];
        h = mix64(h, (uint64_t)lf.num_views);
        h = mix64(h, (uint64_t)lf.fmt);
        h = hash_bytes(h, &ps[l], sizeof(lfd_params));
        for (int v = 0; v < lf.num_views; v++) {
            h = hash_bytes(h, &lf.cams[v], sizeof(lfd_camera));
            h = mix64(h, (uint64_t)(uintptr_t)lf.views[v]);
            h = mix64(h, (uint64_t)(uintptr_t)lf.labels[v]);
            h = mix64(h, (uint64_t)(lf.view_pitch_bytes ? lf.view_pitch_bytes[v] : 0));
            h = mix64(h, (uint64_t)lf.grid_w[v] * 65536u + (uint64_t)lf.grid_h[v]);
            h = mix64(h, (uint64_t)(uintptr_t)(planes_out && planes_out[l] ? planes_out[l][v] : nullptr));
            h = mix64(h, (uint64_t)(uintptr_t)(depth_out && depth_out[l] ? depth_out[l][v] : nullptr));
        }
    }
    h = hash_bytes(h, opt, sizeof(*opt));
    return h | 1;
}

}  // namespace

namespace {

void drop_graph(lfd_ctx *ctx)
{
    if (!ctx->gexec) return;
    cudaEventSynchronize(ctx->stage.event());   // the last replay has finished
    cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
    ctx->gsig = 0;
}

lfd_status apply_options(lfd_ctx *ctx, const lfd_batch_options &o)
{
    if ((o.sweep_threads != 0 && o.sweep_threads != 128 && o.sweep_threads != 256) ||
        (o.prop_blocks != 0 && o.prop_blocks != 7 && o.prop_blocks != 8) || (o.sweep_persistent & ~1) ||
        (o.prop_persistent & ~1) || (o.autotune & ~1) || (o.graph & ~1) ||
        (o.prop_batch != 0 && o.prop_batch != 16 && o.prop_batch != 32) ||
        (o.order_bands != 0 && o.order_bands != 1 && o.order_bands != ORDER_BANDS) || (o.prop_coop & ~1))
        return fail(ctx, LFD_ERR_INVALID_ARG, "batch options: sweep_threads 0/128/256, prop_blocks 0/7/8, "
                                              "prop_batch 0/16/32, order_bands 0/1/16, flags 0/1");
    if (o.autotune) return LFD_OK;
    ctx->lc.sweep_threads = o.sweep_threads ? o.sweep_threads : 256;
    ctx->lc.sweep_persistent = o.sweep_persistent;
    ctx->lc.prop_blocks = o.prop_blocks ? o.prop_blocks : 8;
    ctx->lc.prop_persistent = o.prop_persistent;
    ctx->lc.prop_batch = o.prop_batch ? o.prop_batch : 32;
    ctx->lc.order_bands = o.order_bands ? o.order_bands : ORDER_BANDS;
    ctx->lc.prop_coop = o.prop_coop;
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
    out[4] = (int32_t)sizeof(lfd_batch_options);
    out[5] = (int32_t)sizeof(lfd_result);
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
    p->perturb_samples = 0;
    p->perturb_scale = 0.05;
}

void lfd_batch_options_default(lfd_batch_options *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->sweep_threads = 256;
    o->sweep_persistent = 1;
    o->prop_blocks = 8;
    o->prop_persistent = 1;
    o->prop_batch = 32;
    o->order_bands = ORDER_BANDS;
    o->prop_coop = 0;
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
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        ctx->stage.init() != cudaSuccess || ctx->dtab.init() != cudaSuccess || ctx->ftab.init() != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_bdepth, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ctx->stage.release();
        ctx->dtab.release();
        ctx->ftab.release();
        if (ctx->ev_bdepth) cudaEventDestroy(ctx->ev_bdepth);
        delete ctx;
        return LFD_ERR_CUDA;
    }
    ctx->lc.num_sms = ctx->num_sms;
    *out = ctx;
    return LFD_OK;
}

lfd_status lfd_destroy(lfd_ctx *ctx)
{
    if (!ctx) return LFD_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->ws.base) cudaFree(ctx->ws.base);
    if (ctx->d_cost) cudaFree(ctx->d_cost);
    if (ctx->d_stage_in) cudaFree(ctx->d_stage_in);
    if (ctx->d_stage_depth) cudaFree(ctx->d_stage_depth);
    if (ctx->d_q) cudaFree(ctx->d_q);
    if (ctx->d_qout) cudaFree(ctx->d_qout);
    ctx->stage.release();
    ctx->dtab.release();
    ctx->ftab.release();
    if (ctx->d_zbuf) cudaFree(ctx->d_zbuf);
    if (ctx->d_slic) cudaFree(ctx->d_slic);
    if (ctx->d_ftab) cudaFree(ctx->d_ftab);
    if (ctx->h_bdepth) cudaFreeHost(ctx->h_bdepth);
    if (ctx->ev_bdepth) cudaEventDestroy(ctx->ev_bdepth);
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
    if (!lf || !p) return fail(ctx, LFD_ERR_INVALID_ARG, "light field or params is NULL");
    return set_input_multi(ctx, 1, lf, p, (cudaStream_t)stream);
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
        for (const LfInfo &l : ctx->lfs)
            if (l.p.num_labels != ctx->c.L)
                return fail(ctx, LFD_ERR_INVALID_ARG, "cost_out needs one label count across the bound light fields");
        const size_t need = sizeof(float) * (size_t)ctx->L.S_total * ctx->c.L;
        if ((s = ensure_dev(ctx, (void **)&ctx->d_cost, &ctx->cost_cap, need)) != LFD_OK) return s;
        cost = ctx->d_cost;
    }
    if ((s = run_sweep(ctx, cost, st)) != LFD_OK) return s;
    if ((s = scatter<float>(ctx, (const float *)ctx->d_planesA, planes_out, 4, st)) != LFD_OK) return s;
    if ((s = scatter<int32_t>(ctx, ctx->d_label, label_out, 1, st)) != LFD_OK) return s;
    if (cost_out && (s = scatter<float>(ctx, cost, cost_out, ctx->c.L, st)) != LFD_OK) return s;
    return LFD_OK;
}

lfd_status lfd_rasterize(lfd_ctx *ctx, const float *const *planes, float *const *depth_out, void *stream)
{
    lfd_status s;
    if ((s = need_bound(ctx)) != LFD_OK) return s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = gather_planes(ctx, planes, ctx->d_planesA, st)) != LFD_OK) return s;
    float **dp = nullptr;
    if ((s = upload_depth_ptrs(ctx, depth_out, st, &dp)) != LFD_OK) return s;
    return rasterize_state(ctx, ctx->d_planesA, dp, st);
}

lfd_status lfd_iterate(lfd_ctx *ctx, int32_t iter, const float *const *planes_in, float *const *planes_out,
                       int32_t *const *choice_out, float *const *energy_out, void *stream)
{
    lfd_status s;
    if ((s = need_bound(ctx)) != LFD_OK) return s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    int warm = 0;
    for (const LfInfo &l : ctx->lfs) warm = std::max(warm, l.p.warm_iter_offset);
    if (iter < 1 || iter + warm > LFD_MAX_ITER_INDEX)
        return fail(ctx, LFD_ERR_INVALID_ARG, "iteration index %d outside 1..%d", iter, LFD_MAX_ITER_INDEX - warm);
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
    if (!lf || !p) return fail(ctx, LFD_ERR_INVALID_ARG, "light field or params is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = set_input_multi(ctx, 1, lf, p, st)) != LFD_OK) return s;
    float **dp = nullptr;
    if ((s = upload_depth_ptrs(ctx, depth_out, st, &dp)) != LFD_OK) return s;
    float *const *po[1] = {planes_out};
    return enqueue_frame(ctx, warm_planes, po, dp, st, cudaMemcpyDeviceToDevice);
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
    drop_graph(ctx);
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
    std::vector<float *> dptr(V, nullptr);
    if (depth_out_host)
        for (int v = 0; v < V; v++) dptr[v] = ctx->d_stage_depth + o_dep[v];
    if ((s = set_input_multi(ctx, 1, &lfd, p, st)) != LFD_OK) return s;
    float **dp = nullptr;
    if ((s = upload_depth_ptrs(ctx, depth_out_host ? dptr.data() : nullptr, st, &dp)) != LFD_OK) return s;
    float *const *po[1] = {planes_out_host};
    if ((s = enqueue_frame(ctx, nullptr, po, dp, st, cudaMemcpyDeviceToHost)) != LFD_OK) return s;
    if (depth_out_host)
        for (int v = 0; v < V; v++)
            if (depth_out_host[v])
                LFD_CUDA(cudaMemcpyAsync(depth_out_host[v], dptr[v],
                                         4 * (size_t)lf_host->cams[v].width * lf_host->cams[v].height,
                                         cudaMemcpyDeviceToHost, st));
    return LFD_OK;
}

}  // extern "C"

namespace {

// lfd_estimate_batch and lfd_estimate_batch_warm: warm = NULL (every light
// field cold) or per light field NULL / its views' warm planes
lfd_status estimate_batch_impl(lfd_ctx *ctx, int32_t n, const lfd_lightfield *lfs, const lfd_params *params,
                               const float *const *const *warm, float *const *const *planes_out,
                               float *const *const *depth_out, const lfd_batch_options *options, void *stream)
{
    if (!ctx) return LFD_ERR_INVALID_ARG;
    ctx->err.clear();
    lfd_status s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    lfd_batch_options o;
    lfd_batch_options_default(&o);
    if (options) o = *options;
    if ((s = apply_options(ctx, o)) != LFD_OK) return s;
    if (n < 1 || !lfs || !params) return fail(ctx, LFD_ERR_INVALID_ARG, "need n >= 1 light fields and parameters");
    if (!planes_out) return fail(ctx, LFD_ERR_INVALID_ARG, "planes_out is NULL");
    for (int l = 0; l < n; l++)
        if (!planes_out[l]) return fail(ctx, LFD_ERR_INVALID_ARG, "planes_out[%d] is NULL", l);
    cudaStream_t st = (cudaStream_t)stream;
    if (o.graph && !st) return fail(ctx, LFD_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    for (int l = 0; l < n; l++)
        if (!lfs[l].num_views || lfs[l].num_views > LFD_MAX_VIEWS || !lfs[l].cams || !lfs[l].views || !lfs[l].labels ||
            !lfs[l].grid_w || !lfs[l].grid_h)
            return fail(ctx, LFD_ERR_INVALID_ARG, "light field %d is incomplete", l);
    bool any_warm = false;
    if (warm)
        for (int l = 0; l < n; l++)
            if (warm[l]) {
                any_warm = true;
                for (int v = 0; v < lfs[l].num_views; v++)
                    if (!warm[l][v]) return fail(ctx, LFD_ERR_INVALID_ARG, "warm planes of light field %d view %d "
                                                 "are NULL", l, v);
            }
    if (any_warm && o.graph) return fail(ctx, LFD_ERR_INVALID_ARG, "warm-started batches are not graph-captured");
    const uint64_t sig = batch_signature(n, lfs, params, planes_out, depth_out, &o);

    if (o.graph && ctx->gexec && ctx->gsig == sig && ctx->bound) {     // replay
        if (ctx->ev_bdepth) LFD_CUDA(cudaEventSynchronize(ctx->ev_bdepth));
        LFD_CUDA(cudaGraphLaunch(ctx->gexec, st));
        LFD_CUDA(cudaEventRecord(ctx->stage.event(), st));
        LFD_CUDA(cudaEventRecord(ctx->ev_bdepth, st));
        for (int k = 0; k < LFD_STAGES; k++) ctx->launches[k] += ctx->glaunches[k];
        return LFD_OK;
    }

    drop_graph(ctx);
    ctx->bound = false;
    if ((s = plan_input(ctx, n, lfs, params, false)) != LFD_OK) return s;
    int total_views = 0;
    for (int l = 0; l < n; l++) total_views += lfs[l].num_views;
    std::vector<float *> depth_flat(total_views, nullptr);
    if (depth_out)
        for (int l = 0, g = 0; l < n; l++)
            for (int v = 0; v < lfs[l].num_views; v++, g++) depth_flat[g] = depth_out[l] ? depth_out[l][v] : nullptr;

    if (o.autotune && ctx->tuned_sig != sig) {
        // the launch shapes are timed on this input, bound outside any capture
        if ((s = enqueue_input(ctx, st, true)) != LFD_OK) return s;
        if ((s = autotune(ctx, st)) != LFD_OK) return s;
        LFD_CUDA(cudaMemsetAsync(ctx->d_ctr, 0, 2 * sizeof(unsigned long long), st));
        ctx->tuned_sig = sig;
    }

    if (!o.graph) {
        std::vector<const float *> warm_flat;
        if (any_warm) {
            // views of warm light fields leave the sweep out (their records are
            // still in the pinned staging buffer, uploaded by enqueue_input)
            warm_flat.assign(total_views, nullptr);
            ViewDev *hv = (ViewDev *)ctx->stage.buf();
            for (int l = 0, g = 0; l < n; l++)
                for (int v = 0; v < lfs[l].num_views; v++, g++)
                    if (warm[l]) {
                        warm_flat[g] = warm[l][v];
                        hv[g].sweep_skip = 1;
                    }
        }
        if ((s = enqueue_input(ctx, st, true)) != LFD_OK) return s;
        float **dp = nullptr;
        if ((s = upload_depth_ptrs(ctx, depth_out ? depth_flat.data() : nullptr, st, &dp)) != LFD_OK) return s;
        if ((s = enqueue_frame(ctx, any_warm ? warm_flat.data() : nullptr, planes_out, dp, st,
                               cudaMemcpyDeviceToDevice)) != LFD_OK)
            return s;
        ctx->bound = true;
        return LFD_OK;
    }

    // capture: records and the depth table are read from pinned buffers that
    // stay unchanged while the signature does
    if (depth_out) {
        if (ctx->ev_bdepth) LFD_CUDA(cudaEventSynchronize(ctx->ev_bdepth));
        if (ctx->h_bdepth_cap < total_views) {
            if (ctx->h_bdepth) cudaFreeHost(ctx->h_bdepth);
            ctx->h_bdepth = nullptr;
            ctx->h_bdepth_cap = 0;
            LFD_CUDA(cudaMallocHost(&ctx->h_bdepth, sizeof(float *) * total_views));
            ctx->h_bdepth_cap = total_views;
        }
        for (int g = 0; g < total_views; g++) ctx->h_bdepth[g] = depth_flat[g];
    }
    long long before[LFD_STAGES];
    for (int k = 0; k < LFD_STAGES; k++) before[k] = ctx->launches[k];
    const bool prof = ctx->prof;
    ctx->prof = false;
    LFD_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    s = enqueue_input(ctx, st, false);
    if (s == LFD_OK && depth_out) {
        const cudaError_t e = cudaMemcpyAsync(ctx->d_depth_ptrs, ctx->h_bdepth, sizeof(float *) * total_views,
                                              cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = fail(ctx, LFD_ERR_CUDA, "depth table copy: %s", cudaGetErrorString(e));
    }
    if (s == LFD_OK)
        s = enqueue_frame(ctx, nullptr, planes_out, depth_out ? ctx->d_depth_ptrs : nullptr, st,
                          cudaMemcpyDeviceToDevice);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &graph);
    ctx->prof = prof;
    if (s != LFD_OK) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return s;
    }
    if (ec != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(ctx, LFD_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(ec));
    }
    const cudaError_t ei = cudaGraphInstantiate(&ctx->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        ctx->gexec = nullptr;
        cudaGetLastError();
        return fail(ctx, LFD_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
    }
    for (int k = 0; k < LFD_STAGES; k++) ctx->glaunches[k] = ctx->launches[k] - before[k];
    ctx->gsig = sig;
    LFD_CUDA(cudaGraphLaunch(ctx->gexec, st));
    LFD_CUDA(cudaEventRecord(ctx->stage.event(), st));
    LFD_CUDA(cudaEventRecord(ctx->ev_bdepth, st));
    ctx->bound = true;
    return LFD_OK;
}

}  // namespace

extern "C" {

lfd_status lfd_estimate_batch(lfd_ctx *ctx, int32_t n, const lfd_lightfield *lfs, const lfd_params *params,
                              float *const *const *planes_out, float *const *const *depth_out,
                              const lfd_batch_options *options, void *stream)
{
    return estimate_batch_impl(ctx, n, lfs, params, nullptr, planes_out, depth_out, options, stream);
}

lfd_status lfd_estimate_batch_warm(lfd_ctx *ctx, int32_t n, const lfd_lightfield *lfs, const lfd_params *params,
                                   const float *const *const *warm_planes, float *const *const *planes_out,
                                   float *const *const *depth_out, const lfd_batch_options *options, void *stream)
{
    return estimate_batch_impl(ctx, n, lfs, params, warm_planes, planes_out, depth_out, options, stream);
}

lfd_status lfd_workspace_required(int32_t n, const lfd_lightfield *lfs, uint64_t *bytes)
{
    if (n < 1 || !lfs || !bytes) return LFD_ERR_INVALID_ARG;
    for (int l = 0; l < n; l++)
        if (lfs[l].num_views < 1 || lfs[l].num_views > LFD_MAX_VIEWS || !lfs[l].cams || !lfs[l].grid_w ||
            !lfs[l].grid_h || quad_bytes(lfs[l].fmt) == 0 || lfs[l].fmt != lfs[0].fmt)
            return LFD_ERR_INVALID_ARG;
    Layout L;
    if (make_layout(nullptr, n, lfs, L) != LFD_OK) return LFD_ERR_INVALID_ARG;
    *bytes = (uint64_t)workspace_need(L, lfs[0].fmt);
    return LFD_OK;
}


lfd_status lfd_fuse(lfd_ctx *ctx, const float *const *depth_in, float *const *depth_out, double tau, void *stream)
{
    lfd_status s;
    if ((s = need_bound(ctx)) != LFD_OK) return s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    if (!depth_in || !depth_out) return fail(ctx, LFD_ERR_INVALID_ARG, "depth_in / depth_out is NULL");
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(ctx, LFD_ERR_INVALID_ARG, "tau must be > 0");
    for (int v = 0; v < ctx->L.V; v++) {
        if (!depth_in[v] || !depth_out[v]) return fail(ctx, LFD_ERR_INVALID_ARG, "depth map of view %d is NULL", v);
        if (depth_in[v] == depth_out[v]) return fail(ctx, LFD_ERR_INVALID_ARG, "view %d: depth_in aliases depth_out", v);
    }
    cudaStream_t st = (cudaStream_t)stream;
    // z-buffer and table sizes: the largest light field
    size_t zmax = 0, tmax = 0;
    for (const LfInfo &l : ctx->lfs) {
        size_t z = 0;
        for (int k = 0; k < l.V; k++) z += (size_t)(l.V - 1) * ctx->L.W[l.first_view + k] * ctx->L.H[l.first_view + k];
        zmax = std::max(zmax, z);
        const size_t t = align_up(8 * (size_t)l.V, 16) + 8 * (size_t)l.V + 16 * (size_t)l.V + 48 * (size_t)l.V * l.V;
        tmax = std::max(tmax, t);
    }
    if ((s = ensure_dev(ctx, (void **)&ctx->d_zbuf, &ctx->zbuf_cap, 4 * std::max<size_t>(zmax, 1))) != LFD_OK) return s;
    if ((s = ensure_dev(ctx, &ctx->d_ftab, &ctx->ftab_cap, tmax)) != LFD_OK) return s;
    for (const LfInfo &l : ctx->lfs) {
        const int V = l.V, f = l.first_view;
        // table: W, H (int), zoff (int64), depth_in, depth_out (pointers), mats (float)
        const size_t o_wh = 0, o_zoff = align_up(8 * (size_t)V, 16), o_in = o_zoff + 8 * (size_t)V,
                     o_out = o_in + 8 * (size_t)V, o_mats = o_out + 8 * (size_t)V;
        const size_t bytes = o_mats + 48 * (size_t)V * V;
        LFD_CUDA(ctx->ftab.next(bytes));
        char *h = (char *)ctx->ftab.buf();
        int *hw = (int *)(h + o_wh), *hh = hw + V;
        long long *hz = (long long *)(h + o_zoff);
        const float **hin = (const float **)(h + o_in);
        float **hout = (float **)(h + o_out);
        float *hm = (float *)(h + o_mats);
        long long zw = 0;
        int max_px = 0;
        for (int k = 0; k < V; k++) {
            hw[k] = ctx->L.W[f + k];
            hh[k] = ctx->L.H[f + k];
            hz[k] = zw;
            zw += (long long)(V - 1) * hw[k] * hh[k];
            max_px = std::max(max_px, hw[k] * hh[k]);
            hin[k] = depth_in[f + k];
            hout[k] = depth_out[f + k];
        }
        for (int i = 0; i < V; i++) {
            const lfd_camera &ci = ctx->cams[f + i];
            double Ki[9];
            inv_pinhole(ci.K, Ki);
            for (int r = 0; r < V; r++) {
                float *m = hm + 12 * (i * V + r);
                if (r == i) {
                    for (int k = 0; k < 12; k++) m[k] = 0.f;
                    continue;
                }
                const lfd_camera &cr = ctx->cams[f + r];
                // A = R_r R_i^T, M = K_r A K_i^-1, e = K_r (t_r - A t_i)
                double A[9], KA[9], M[9], e0[3];
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++)
                        A[3 * a + b] = cr.R[3 * a] * ci.R[3 * b] + cr.R[3 * a + 1] * ci.R[3 * b + 1] +
                                       cr.R[3 * a + 2] * ci.R[3 * b + 2];
                mat_mul(cr.K, A, KA);
                mat_mul(KA, Ki, M);
                for (int a = 0; a < 3; a++)
                    e0[a] = cr.t[a] - (A[3 * a] * ci.t[0] + A[3 * a + 1] * ci.t[1] + A[3 * a + 2] * ci.t[2]);
                for (int k = 0; k < 9; k++) m[k] = (float)M[k];
                for (int a = 0; a < 3; a++)
                    m[9 + a] = (float)(cr.K[3 * a] * e0[0] + cr.K[3 * a + 1] * e0[1] + cr.K[3 * a + 2] * e0[2]);
            }
        }
        LFD_CUDA(cudaMemcpyAsync(ctx->d_ftab, h, bytes, cudaMemcpyHostToDevice, st));
        LFD_CUDA(cudaEventRecord(ctx->ftab.event(), st));
        char *d = (char *)ctx->d_ftab;
        FuseArgs a;
        a.V = V;
        a.tau = (float)tau;
        a.W = (const int *)(d + o_wh);
        a.H = a.W + V;
        a.zoff = (const long long *)(d + o_zoff);
        a.depth_in = (const float *const *)(d + o_in);
        a.depth_out = (float *const *)(d + o_out);
        a.mats = (const float *)(d + o_mats);
        a.zbuf = ctx->d_zbuf;
        LFD_CUDA(traced(ctx, LFD_STAGE_FUSION, st, [&] { return launch_fuse(a, zw, max_px, st); }, 3));
    }
    return LFD_OK;
}


lfd_status lfd_slic(lfd_ctx *ctx, int32_t n, const void *const *views, const int64_t *view_pitch_bytes, int32_t fmt,
                    const int32_t *width, const int32_t *height, const int32_t *grid_w, const int32_t *grid_h,
                    double compactness, int32_t iterations, int32_t *const *labels_out,
                    const float *const *centres_in, float *const *centres_out, void *stream)
{
    if (!ctx) return LFD_ERR_INVALID_ARG;
    ctx->err.clear();
    lfd_status s;
    if ((s = set_device(ctx)) != LFD_OK) return s;
    const int tb = texel_bytes(fmt);
    if (n < 1 || !views || !width || !height || !grid_w || !grid_h || !labels_out || tb == 0)
        return fail(ctx, LFD_ERR_INVALID_ARG, "lfd_slic: bad arguments");
    if (!(compactness > 0.0) || iterations < 0 || iterations > 1000)
        return fail(ctx, LFD_ERR_INVALID_ARG, "compactness must be > 0 and iterations 0..1000");
    auto view_bytes = [&](int v, size_t &o_c, size_t &sz_c) {
        o_c = align_up(16 * (size_t)width[v] * height[v], 256);
        sz_c = align_up(20 * (size_t)grid_w[v] * grid_h[v], 256);
        return o_c + 2 * sz_c + align_up(48 * (size_t)grid_w[v] * grid_h[v], 256);
    };
    for (int v = 0; v < n; v++) {
        if (width[v] < 1 || height[v] < 1 || width[v] > LFD_MAX_DIM || height[v] > LFD_MAX_DIM || grid_w[v] < 1 ||
            grid_h[v] < 1 || grid_w[v] > width[v] || grid_h[v] > height[v] || !views[v] || !labels_out[v])
            return fail(ctx, LFD_ERR_INVALID_ARG, "lfd_slic: view %d: bad size, grid or pointer", v);
        const long long pitch = view_pitch_bytes && view_pitch_bytes[v] ? view_pitch_bytes[v] : (long long)width[v] * tb;
        if (pitch < (long long)width[v] * tb || pitch % tb)
            return fail(ctx, LFD_ERR_INVALID_ARG, "lfd_slic: view %d: bad pitch", v);
    }
    // scratch for one group of up to SLIC_BATCH views at a time
    size_t need = 0;
    for (int g = 0; g < n; g += SLIC_BATCH) {
        size_t sum = 0, o_c, sz_c;
        for (int v = g; v < std::min(n, g + SLIC_BATCH); v++) sum += view_bytes(v, o_c, sz_c);
        need = std::max(need, sum);
    }
    if ((s = ensure_dev(ctx, &ctx->d_slic, &ctx->slic_cap, need)) != LFD_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    for (int g = 0; g < n; g += SLIC_BATCH) {
        SlicBatch b = {};
        b.n = std::min(n - g, SLIC_BATCH);
        char *base = (char *)ctx->d_slic;
        for (int k = 0; k < b.n; k++) {
            const int v = g + k;
            SlicView &sv = b.v[k];
            size_t o_c, sz_c;
            const size_t bytes = view_bytes(v, o_c, sz_c);
            sv.W = width[v];
            sv.H = height[v];
            sv.GW = grid_w[v];
            sv.GH = grid_h[v];
            sv.fmt = fmt;
            sv.pad = 0;
            sv.pitch = view_pitch_bytes && view_pitch_bytes[v] ? view_pitch_bytes[v] : (long long)width[v] * tb;
            sv.img = views[v];
            sv.lab = (float4 *)base;
            sv.centres = (float *)(base + o_c);
            sv.centres2 = (float *)(base + o_c + sz_c);
            sv.acc = (unsigned long long *)(base + o_c + 2 * sz_c);
            sv.labels = labels_out[v];
            base += bytes;
            const double step = std::sqrt((double)sv.W * sv.H / ((double)sv.GW * sv.GH));
            b.wxy[k] = (float)((compactness / step) * (compactness / step));
            b.max_px = std::max(b.max_px, sv.W * sv.H);
            b.max_cells = std::max(b.max_cells, sv.GW * sv.GH);
        }
        LFD_CUDA(launch_slic(b, centres_in ? centres_in + g : nullptr, iterations, centres_out ? centres_out + g : nullptr,
                             st));
    }
    return LFD_OK;
}

lfd_status lfd_launch_config(const lfd_ctx *ctx, int32_t *out)
{
    if (!ctx || !out) return LFD_ERR_INVALID_ARG;
    out[0] = ctx->lc.sweep_threads;
    out[1] = ctx->lc.sweep_persistent;
    out[2] = ctx->lc.prop_blocks;
    out[3] = ctx->lc.prop_persistent;
    out[4] = ctx->lc.prop_batch;
    out[5] = ctx->lc.order_bands;
    out[6] = ctx->lc.prop_coop;
    return LFD_OK;
}
lfd_status lfd_set_pair_forms(lfd_ctx *ctx, int32_t max_form)
{
    if (!ctx) return LFD_ERR_INVALID_ARG;
    if (max_form < 0 || max_form > 2) return fail(ctx, LFD_ERR_INVALID_ARG, "max_form must be 0, 1 or 2");
    ctx->max_pair_form = max_form;
    drop_graph(ctx);
    return LFD_OK;
}
lfd_status lfd_pair_form(const lfd_ctx *ctx, int32_t *form)
{
    if (!ctx || !form) return LFD_ERR_INVALID_ARG;
    if (!ctx->bound) return LFD_ERR_STATE;
    *form = ctx->c.shift ? 2 : (ctx->c.affine ? 1 : 0);
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
    double ms[LFD_STAGES] = {};
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
