// Frame server of liblfdepth: several rigs share one GPU through a fixed set
// of slots (context + stream).  Built on the public C ABI only; the paper has
// no serving layer (each light field is processed on its own), so the warm
// start, admission and queue bound here are this library's policy, documented
// in include/lfdepth.h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lfdepth.h"

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    uint64_t id = 0;
    int rig = 0, slot = 0, warm = 0;
    int64_t frame = 0;
    int64_t submit_ns = 0;
    std::atomic<int64_t> done_ns{0};
};

// Runs on a CUDA driver thread once the slot's stream has finished the frame.
void CUDART_CB on_frame_done(void *arg)
{
    static_cast<Request *>(arg)->done_ns.store(now_ns(), std::memory_order_release);
}

struct Slot {
    lfd_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    uint64_t ws_bytes = 0;   // largest workspace of its rigs
    int nrigs = 0;
};

struct Rig {
    int slot = -1;
    std::vector<int> S;                      // superpixels per view
    std::vector<int> W, H;
    int64_t S_total = 0;
    float *planes = nullptr;                 // state, float4 per superpixel
    int64_t planes_cap = 0;
    bool has_state = false;
    int64_t frames = 0;
    int pending = 0;
    uint64_t ws_need = 0;
};

}  // namespace

struct lfd_server {
    int device = 0;
    uint64_t budget = 0;
    std::vector<Slot> slots;
    std::map<int, Rig> rigs;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_id = 1;
    int warm_iters = 3, warm_off = 3, max_pending = 2;
    std::string err;
};

namespace {

lfd_status sfail(lfd_server *srv, lfd_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    srv->err = buf;
    return s;
}

uint64_t committed_bytes(const lfd_server *srv)
{
    uint64_t b = 0;
    for (const Slot &s : srv->slots) b += s.ws_bytes;
    for (const auto &kv : srv->rigs) b += 16 * (uint64_t)kv.second.planes_cap;
    return b;
}

bool same_layout(const Rig &r, const lfd_lightfield *lf)
{
    if ((int)r.S.size() != lf->num_views) return false;
    for (int v = 0; v < lf->num_views; v++)
        if (r.S[v] != lf->grid_w[v] * lf->grid_h[v] || r.W[v] != lf->cams[v].width || r.H[v] != lf->cams[v].height)
            return false;
    return true;
}

}  // namespace

extern "C" {

int64_t lfd_server_now_ns(void) { return now_ns(); }

lfd_status lfd_server_create(lfd_server **out, int32_t device, uint64_t hbm_budget_bytes, int32_t max_slots)
{
    if (!out || max_slots < 1 || max_slots > 64) return LFD_ERR_INVALID_ARG;
    *out = nullptr;
    lfd_server *srv = new (std::nothrow) lfd_server();
    if (!srv) return LFD_ERR_OOM;
    srv->device = device;
    srv->budget = hbm_budget_bytes;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete srv;
        return LFD_ERR_INVALID_ARG;
    }
    for (int i = 0; i < max_slots; i++) {
        Slot sl;
        lfd_status s = lfd_create(&sl.ctx, device, 0);
        if (s == LFD_OK && cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            lfd_destroy(sl.ctx);
            s = LFD_ERR_CUDA;
        }
        if (s != LFD_OK) {
            lfd_server_destroy(srv);
            return s;
        }
        srv->slots.push_back(sl);
    }
    *out = srv;
    return LFD_OK;
}

lfd_status lfd_server_destroy(lfd_server *srv)
{
    if (!srv) return LFD_ERR_INVALID_ARG;
    cudaSetDevice(srv->device);
    for (Slot &s : srv->slots) {
        if (s.st) {
            cudaStreamSynchronize(s.st);
            cudaStreamDestroy(s.st);
        }
        if (s.ctx) lfd_destroy(s.ctx);
    }
    for (auto &kv : srv->rigs)
        if (kv.second.planes) cudaFree(kv.second.planes);
    delete srv;
    return LFD_OK;
}

const char *lfd_server_last_error(const lfd_server *srv) { return srv ? srv->err.c_str() : "NULL server"; }

lfd_status lfd_server_configure(lfd_server *srv, int32_t warm_iterations, int32_t warm_iter_offset,
                                int32_t max_pending_per_rig)
{
    if (!srv) return LFD_ERR_INVALID_ARG;
    if (warm_iterations < 0 || warm_iter_offset < 0 || warm_iterations + warm_iter_offset > LFD_MAX_ITER_INDEX ||
        max_pending_per_rig < 1)
        return sfail(srv, LFD_ERR_INVALID_ARG, "warm_iterations, warm_iter_offset >= 0 with sum <= %d; "
                     "max_pending_per_rig >= 1", LFD_MAX_ITER_INDEX);
    srv->warm_iters = warm_iterations;
    srv->warm_off = warm_iter_offset;
    srv->max_pending = max_pending_per_rig;
    return LFD_OK;
}

lfd_status lfd_server_submit(lfd_server *srv, int32_t rig_id, const lfd_lightfield *lf, const lfd_params *params,
                             float *const *planes_out, float *const *depth_out, uint64_t *req_id)
{
    if (!srv) return LFD_ERR_INVALID_ARG;
    srv->err.clear();
    if (!lf || !params || !req_id || rig_id < 0) return sfail(srv, LFD_ERR_INVALID_ARG, "bad submit arguments");
    if (cudaSetDevice(srv->device) != cudaSuccess) {
        cudaGetLastError();
        return sfail(srv, LFD_ERR_CUDA, "cudaSetDevice failed");
    }
    uint64_t need = 0;
    if (lfd_workspace_required(1, lf, &need) != LFD_OK)
        return sfail(srv, LFD_ERR_INVALID_ARG, "light field of rig %d is malformed", rig_id);
    int64_t S_total = 0;
    for (int v = 0; v < lf->num_views; v++) S_total += (int64_t)lf->grid_w[v] * lf->grid_h[v];

    auto it = srv->rigs.find(rig_id);
    const bool known = it != srv->rigs.end();
    if (known && it->second.pending >= srv->max_pending)
        return sfail(srv, LFD_ERR_BUSY, "rig %d has %d frames in flight", rig_id, it->second.pending);

    // admission: the rig's slot and the budget
    int slot = known ? it->second.slot : 0;
    if (!known)
        for (int i = 1; i < (int)srv->slots.size(); i++)
            if (srv->slots[i].nrigs < srv->slots[slot].nrigs) slot = i;
    const Rig *old = known ? &it->second : nullptr;
    const uint64_t slot_after = std::max(srv->slots[slot].ws_bytes, need);
    const int64_t cap_after = std::max<int64_t>(old ? old->planes_cap : 0, S_total);
    const uint64_t total_after = committed_bytes(srv) - srv->slots[slot].ws_bytes + slot_after -
                                 16 * (uint64_t)(old ? old->planes_cap : 0) + 16 * (uint64_t)cap_after;
    if (srv->budget && total_after > srv->budget)
        return sfail(srv, LFD_ERR_BUDGET, "rig %d needs %llu bytes of workspace; the server would hold %llu of %llu",
                     rig_id, (unsigned long long)need, (unsigned long long)total_after,
                     (unsigned long long)srv->budget);

    Rig &r = srv->rigs[rig_id];
    if (!known) {
        r.slot = slot;
        srv->slots[slot].nrigs++;
    }
    Slot &sl = srv->slots[r.slot];
    if (!same_layout(r, lf)) {                       // new rig or changed layout: cold start
        r.has_state = false;
        r.S.assign(lf->num_views, 0);
        r.W.assign(lf->num_views, 0);
        r.H.assign(lf->num_views, 0);
        for (int v = 0; v < lf->num_views; v++) {
            r.S[v] = lf->grid_w[v] * lf->grid_h[v];
            r.W[v] = lf->cams[v].width;
            r.H[v] = lf->cams[v].height;
        }
        r.S_total = S_total;
        if (r.planes_cap < S_total) {
            if (r.planes) {
                cudaStreamSynchronize(sl.st);
                cudaFree(r.planes);
            }
            r.planes = nullptr;
            r.planes_cap = 0;
            if (cudaMalloc(&r.planes, 16 * (size_t)S_total) != cudaSuccess) {
                cudaGetLastError();
                return sfail(srv, LFD_ERR_OOM, "rig %d: plane state allocation failed", rig_id);
            }
            r.planes_cap = S_total;
        }
    }
    r.ws_need = need;
    sl.ws_bytes = std::max(sl.ws_bytes, need);

    std::vector<float *> state(lf->num_views);
    for (int v = 0, base = 0; v < lf->num_views; base += r.S[v], v++) state[v] = r.planes + 4 * (size_t)base;
    lfd_params p = *params;
    const bool warm = r.has_state && srv->warm_iters > 0;
    if (warm) {
        p.iterations = srv->warm_iters;
        p.warm_iter_offset = srv->warm_off;
    }
    auto req = std::make_unique<Request>();
    req->id = srv->next_id++;
    req->rig = rig_id;
    req->slot = r.slot;
    req->warm = warm ? 1 : 0;
    req->frame = r.frames;
    req->submit_ns = now_ns();
    // the warm planes are gathered into the context before its output
    // overwrites the rig state, so state serves as both
    lfd_status s = lfd_estimate(sl.ctx, lf, &p, warm ? state.data() : nullptr, state.data(), depth_out, sl.st);
    if (s != LFD_OK) return sfail(srv, s, "rig %d: %s", rig_id, lfd_last_error(sl.ctx));
    if (planes_out)
        for (int v = 0; v < lf->num_views; v++)
            if (planes_out[v] &&
                cudaMemcpyAsync(planes_out[v], state[v], 16 * (size_t)r.S[v], cudaMemcpyDeviceToDevice, sl.st) !=
                    cudaSuccess) {
                cudaGetLastError();
                return sfail(srv, LFD_ERR_CUDA, "rig %d: planes copy failed", rig_id);
            }
    if (cudaLaunchHostFunc(sl.st, on_frame_done, req.get()) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(sl.st);
        req->done_ns.store(now_ns());
    }
    r.has_state = true;
    r.frames++;
    r.pending++;
    *req_id = req->id;
    srv->reqs.emplace(req->id, std::move(req));
    return LFD_OK;
}

lfd_status lfd_server_poll(lfd_server *srv, uint64_t req_id, int32_t timeout_us, lfd_result *out)
{
    if (!srv) return LFD_ERR_INVALID_ARG;
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) return sfail(srv, LFD_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)req_id);
    Request &q = *it->second;
    const int64_t deadline = now_ns() + (int64_t)timeout_us * 1000;
    int64_t done = q.done_ns.load(std::memory_order_acquire);
    while (!done) {
        if (timeout_us >= 0 && now_ns() >= deadline) return LFD_ERR_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        done = q.done_ns.load(std::memory_order_acquire);
    }
    if (out) {
        memset(out, 0, sizeof(*out));
        out->req_id = q.id;
        out->rig_id = q.rig;
        out->warm = q.warm;
        out->frame = q.frame;
        out->submit_ns = q.submit_ns;
        out->done_ns = done;
        out->status = LFD_OK;
        out->slot = q.slot;
    }
    auto r = srv->rigs.find(q.rig);
    if (r != srv->rigs.end() && r->second.pending > 0) r->second.pending--;
    srv->reqs.erase(it);
    return LFD_OK;
}

lfd_status lfd_server_export_state(lfd_server *srv, int32_t rig_id, float *planes_host, int64_t cap_sp, int64_t *n_sp)
{
    if (!srv) return LFD_ERR_INVALID_ARG;
    auto it = srv->rigs.find(rig_id);
    if (it == srv->rigs.end() || !it->second.has_state)
        return sfail(srv, LFD_ERR_STATE, "rig %d has no plane state", rig_id);
    Rig &r = it->second;
    if (n_sp) *n_sp = r.S_total;
    if (!planes_host) return LFD_OK;
    if (cap_sp < r.S_total) return sfail(srv, LFD_ERR_INVALID_ARG, "state needs %lld superpixels", (long long)r.S_total);
    cudaStream_t st = srv->slots[r.slot].st;
    if (cudaMemcpyAsync(planes_host, r.planes, 16 * (size_t)r.S_total, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return sfail(srv, LFD_ERR_CUDA, "state export failed");
    }
    return LFD_OK;
}

lfd_status lfd_server_import_state(lfd_server *srv, int32_t rig_id, const float *planes_host, int64_t n_sp)
{
    if (!srv || !planes_host) return LFD_ERR_INVALID_ARG;
    auto it = srv->rigs.find(rig_id);
    if (it == srv->rigs.end() || !it->second.planes)
        return sfail(srv, LFD_ERR_STATE, "rig %d has not submitted a frame", rig_id);
    Rig &r = it->second;
    if (n_sp != r.S_total)
        return sfail(srv, LFD_ERR_INVALID_ARG, "state has %lld superpixels, rig %d has %lld", (long long)n_sp, rig_id,
                     (long long)r.S_total);
    cudaStream_t st = srv->slots[r.slot].st;
    if (cudaMemcpyAsync(r.planes, planes_host, 16 * (size_t)n_sp, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return sfail(srv, LFD_ERR_CUDA, "state import failed");
    }
    r.has_state = true;
    return LFD_OK;
}

}  // extern "C"
