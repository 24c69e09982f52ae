// Frame server of liblfdepth: several rigs share one GPU by continuous
// batching.  Built on the public C ABI only; the paper has no serving layer
// (each light field is processed on its own), so the warm start, batching,
// admission and queue bound here are this library's policy, documented in
// include/lfdepth.h.
//
// Requests wait in one FIFO queue.  A dispatcher thread watches the slots
// (a context and a stream each): whenever one is free it takes, in arrival
// order, every queued frame it can run now -- at most one per rig, the rig
// having no frame on the device (its next frame starts from the planes its
// previous frame writes), all warm or all cold, within the HBM budget -- and
// runs them as ONE lfd_estimate_batch_warm call: every superpixel of every
// view of every frame is a work item of the same sweep and propagation
// launches (Section III-E's all-superpixels pass, across rigs).  Frames that
// arrive while batches run join the next batch that a freed slot forms.
// Completion is stamped by a stream callback that touches only atomics.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
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

struct Rig {
    std::vector<int> S, W, H;                // layout: superpixels and size per view
    int64_t S_total = 0;
    float *planes = nullptr;                 // plane state, float4 per superpixel
    int64_t planes_cap = 0;
    bool has_state = false;                  // a frame of this layout has been queued
    int64_t frames = 0;
    int queued = 0;                          // submitted and not yet polled
    std::atomic<int> inflight{0};            // 1 while a frame of the rig is on the device
};

// one frame; the light-field description is copied at submission
struct Request {
    uint64_t id = 0;
    int rig = 0, warm = 0;
    int64_t frame = 0, submit_ns = 0;
    int slot = -1, batch = 0;
    std::atomic<int64_t> start_ns{0};
    std::atomic<int64_t> done_ns{0};
    std::atomic<int> status{LFD_OK};
    lfd_lightfield lf{};
    std::vector<lfd_camera> cams;
    std::vector<const void *> views;
    std::vector<int64_t> pitch;
    std::vector<const int32_t *> labels;
    std::vector<int32_t> gw, gh;
    lfd_params p{};
    std::vector<float *> planes_out, depth_out;   // empty = none
    uint64_t ws_need = 0;
    Rig *rigp = nullptr;
};

struct Slot {
    lfd_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    uint64_t ws_cap = 0;                     // workspace its context holds (largest batch so far)
    std::atomic<int> busy{0};
    std::vector<Request *> batch;            // the frames of its batch on the device
    std::atomic<int64_t> *wake = nullptr;
};

}  // namespace

struct lfd_server {
    int device = 0;
    uint64_t budget = 0;
    std::vector<std::unique_ptr<Slot>> slots;
    std::map<int, std::unique_ptr<Rig>> rigs;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    std::deque<Request *> queue;             // waiting for a slot, arrival order
    uint64_t next_id = 1;
    int warm_iters = 3, warm_off = 3, max_pending = 2, max_batch = 0;
    std::string err;
    std::mutex mu;                           // queue, rigs, reqs, slot assignment
    std::condition_variable cv;
    std::atomic<int64_t> wake{0};            // completions (callbacks only touch atomics)
    std::atomic<bool> stop{false};
    std::thread dispatcher;
    int64_t batches = 0, batched_frames = 0;
    std::string batch_err;                   // last launch failure (dispatcher), reported by poll
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

bool same_layout(const Rig &r, const lfd_lightfield *lf)
{
    if ((int)r.S.size() != lf->num_views) return false;
    for (int v = 0; v < lf->num_views; v++)
        if (r.S[v] != lf->grid_w[v] * lf->grid_h[v] || r.W[v] != lf->cams[v].width || r.H[v] != lf->cams[v].height)
            return false;
    return true;
}

uint64_t planes_bytes(const lfd_server *srv)
{
    uint64_t b = 0;
    for (const auto &kv : srv->rigs) b += 16 * (uint64_t)kv.second->planes_cap;
    return b;
}

// Runs on a CUDA driver thread once a slot's stream has finished its batch;
// touches only atomics (no lock, no CUDA call).
void CUDART_CB on_batch_done(void *arg)
{
    Slot *sl = static_cast<Slot *>(arg);
    const int64_t t = now_ns();
    for (Request *q : sl->batch) {
        q->rigp->inflight.store(0, std::memory_order_release);
        q->done_ns.store(t, std::memory_order_release);          // last access to q
    }
    sl->busy.store(0, std::memory_order_release);
    sl->wake->fetch_add(1, std::memory_order_release);
}

// Launch `batch` on slot k (server lock held).  On failure every frame of
// the batch completes with the error status.
void launch_batch(lfd_server *srv, int k, std::vector<Request *> &batch, uint64_t need)
{
    Slot &sl = *srv->slots[k];
    const int n = (int)batch.size();
    std::vector<lfd_lightfield> lfs(n);
    std::vector<lfd_params> ps(n);
    std::vector<std::vector<float *>> state(n);
    std::vector<const float *const *> warm(n, nullptr);
    std::vector<float *const *> pout(n), dout(n, nullptr);
    bool any_depth = false;
    const int64_t t0 = now_ns();
    for (int l = 0; l < n; l++) {
        Request &q = *batch[l];
        lfs[l] = q.lf;
        ps[l] = q.p;
        Rig &r = *q.rigp;
        state[l].resize(q.lf.num_views);
        for (int v = 0, base = 0; v < q.lf.num_views; base += r.S[v], v++) state[l][v] = r.planes + 4 * (size_t)base;
        if (q.warm) warm[l] = (const float *const *)state[l].data();
        pout[l] = state[l].data();
        if (!q.depth_out.empty()) {
            dout[l] = q.depth_out.data();
            any_depth = true;
        }
        q.slot = k;
        q.batch = n;
        q.start_ns.store(t0, std::memory_order_relaxed);
        r.inflight.store(1, std::memory_order_relaxed);
    }
    lfd_status s = lfd_estimate_batch_warm(sl.ctx, n, lfs.data(), ps.data(), warm.data(), pout.data(),
                                           any_depth ? dout.data() : nullptr, nullptr, sl.st);
    if (s == LFD_OK)
        for (int l = 0; l < n && s == LFD_OK; l++) {
            Request &q = *batch[l];
            for (int v = 0; v < (int)q.planes_out.size(); v++)
                if (q.planes_out[v] && cudaMemcpyAsync(q.planes_out[v], state[l][v], 16 * (size_t)q.rigp->S[v],
                                                       cudaMemcpyDeviceToDevice, sl.st) != cudaSuccess) {
                    cudaGetLastError();
                    s = LFD_ERR_CUDA;
                }
        }
    sl.ws_cap = std::max(sl.ws_cap, need);
    srv->batches++;
    srv->batched_frames += n;
    sl.batch = batch;
    sl.busy.store(1, std::memory_order_relaxed);
    if (s != LFD_OK) {
        srv->batch_err = std::string("batch launch: ") + lfd_last_error(sl.ctx);
        for (Request *q : batch) q->status.store(s);
    }
    if (s != LFD_OK || cudaLaunchHostFunc(sl.st, on_batch_done, &sl) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(sl.st);
        cudaGetLastError();
        on_batch_done(&sl);
    }
}

// Form and launch batches on the free slots (server lock held).
void dispatch(lfd_server *srv)
{
    for (int k = 0; k < (int)srv->slots.size(); k++) {
        Slot &sl = *srv->slots[k];
        if (sl.busy.load(std::memory_order_acquire) || srv->queue.empty()) continue;
        uint64_t others = planes_bytes(srv);
        for (int j = 0; j < (int)srv->slots.size(); j++)
            if (j != k) others += srv->slots[j]->ws_cap;
        std::vector<Request *> batch;
        std::vector<lfd_lightfield> lfs;
        uint64_t need = 0;
        int cls = -1;
        for (Request *q : srv->queue) {
            if (srv->max_batch > 0 && (int)batch.size() >= srv->max_batch) break;
            if (q->rigp->inflight.load(std::memory_order_acquire)) continue;
            bool dup = false;
            for (Request *b : batch) dup = dup || b->rig == q->rig;
            if (dup) continue;
            if (cls >= 0 && (q->warm != cls || q->lf.fmt != batch[0]->lf.fmt ||
                             q->p.depth_domain != batch[0]->p.depth_domain ||
                             q->p.sweep_frame != batch[0]->p.sweep_frame))
                continue;
            lfs.push_back(q->lf);
            uint64_t nb = 0;
            if (lfd_workspace_required((int)lfs.size(), lfs.data(), &nb) != LFD_OK ||
                (srv->budget && others + std::max(sl.ws_cap, nb) > srv->budget)) {
                lfs.pop_back();
                continue;                                  // waits for memory (or a smaller batch)
            }
            need = nb;
            cls = q->warm;
            batch.push_back(q);
        }
        if (batch.empty()) continue;
        for (Request *q : batch) srv->queue.erase(std::find(srv->queue.begin(), srv->queue.end(), q));
        launch_batch(srv, k, batch, need);
    }
    // every slot idle and still nothing fits: the workspaces the slots hold
    // leave no room for the oldest frame; it completes with LFD_ERR_BUDGET
    // rather than wait for memory that will not be released
    for (const auto &sl : srv->slots)
        if (sl->busy.load(std::memory_order_acquire)) return;
    for (auto it = srv->queue.begin(); it != srv->queue.end(); ++it) {
        Request *q = *it;
        if (q->rigp->inflight.load(std::memory_order_acquire)) continue;
        srv->queue.erase(it);
        srv->batch_err = "a frame does not fit the HBM budget next to the slots' workspaces";
        q->status.store(LFD_ERR_BUDGET);
        q->start_ns.store(now_ns());
        q->done_ns.store(now_ns(), std::memory_order_release);
        return;
    }
}

bool launchable(const lfd_server *srv)
{
    bool free_slot = false;
    for (const auto &s : srv->slots) free_slot = free_slot || !s->busy.load(std::memory_order_acquire);
    if (!free_slot) return false;
    for (const Request *q : srv->queue)
        if (!q->rigp->inflight.load(std::memory_order_acquire)) return true;
    return false;
}

void dispatcher_main(lfd_server *srv)
{
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    int64_t seen = srv->wake.load();
    while (!srv->stop.load()) {
        // woken by submissions (notify under the lock) or, within 100 us, by
        // completions (callbacks bump `wake` without the lock)
        srv->cv.wait_for(lk, std::chrono::microseconds(100), [&] {
            return srv->stop.load() || srv->wake.load() != seen || launchable(srv);
        });
        seen = srv->wake.load();
        if (srv->stop.load()) break;
        if (launchable(srv)) dispatch(srv);
    }
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
        auto sl = std::make_unique<Slot>();
        sl->wake = &srv->wake;
        lfd_status s = lfd_create(&sl->ctx, device, 0);
        if (s == LFD_OK && cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            lfd_destroy(sl->ctx);
            sl->ctx = nullptr;
            s = LFD_ERR_CUDA;
        }
        if (s != LFD_OK) {
            lfd_server_destroy(srv);
            return s;
        }
        srv->slots.push_back(std::move(sl));
    }
    srv->dispatcher = std::thread(dispatcher_main, srv);
    *out = srv;
    return LFD_OK;
}

lfd_status lfd_server_destroy(lfd_server *srv)
{
    if (!srv) return LFD_ERR_INVALID_ARG;
    cudaSetDevice(srv->device);
    // frames still queued are run first (for at most a minute), then the
    // dispatcher stops
    const int64_t end = now_ns() + 60LL * 1000000000LL;
    while (now_ns() < end) {
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            if (srv->queue.empty() || !srv->dispatcher.joinable()) break;
        }
        srv->cv.notify_all();
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    srv->stop.store(true);
    srv->cv.notify_all();
    if (srv->dispatcher.joinable()) srv->dispatcher.join();
    for (auto &s : srv->slots) {
        if (s->st) {
            cudaStreamSynchronize(s->st);
            cudaStreamDestroy(s->st);
        }
        while (s->busy.load()) std::this_thread::sleep_for(std::chrono::microseconds(50));
        if (s->ctx) lfd_destroy(s->ctx);
    }
    for (auto &kv : srv->rigs)
        if (kv.second->planes) cudaFree(kv.second->planes);
    delete srv;
    return LFD_OK;
}

const char *lfd_server_last_error(const lfd_server *srv) { return srv ? srv->err.c_str() : "NULL server"; }

lfd_status lfd_server_configure(lfd_server *srv, int32_t warm_iterations, int32_t warm_iter_offset,
                                int32_t max_pending_per_rig)
{
    if (!srv) return LFD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (warm_iterations < 0 || warm_iter_offset < 0 || warm_iterations + warm_iter_offset > LFD_MAX_ITER_INDEX ||
        max_pending_per_rig < 1)
        return sfail(srv, LFD_ERR_INVALID_ARG, "warm_iterations, warm_iter_offset >= 0 with sum <= %d; "
                     "max_pending_per_rig >= 1", LFD_MAX_ITER_INDEX);
    srv->warm_iters = warm_iterations;
    srv->warm_off = warm_iter_offset;
    srv->max_pending = max_pending_per_rig;
    return LFD_OK;
}

lfd_status lfd_server_set_max_batch(lfd_server *srv, int32_t max_frames)
{
    if (!srv || max_frames < 0) return LFD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->max_batch = max_frames;
    return LFD_OK;
}

lfd_status lfd_server_stats(lfd_server *srv, int64_t *batches, int64_t *frames)
{
    if (!srv) return LFD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (batches) *batches = srv->batches;
    if (frames) *frames = srv->batched_frames;
    return LFD_OK;
}

lfd_status lfd_server_submit(lfd_server *srv, int32_t rig_id, const lfd_lightfield *lf, const lfd_params *params,
                             float *const *planes_out, float *const *depth_out, uint64_t *req_id)
{
    if (!srv) return LFD_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->err.clear();
    if (!lf || !params || !req_id || rig_id < 0) return sfail(srv, LFD_ERR_INVALID_ARG, "bad submit arguments");
    if (cudaSetDevice(srv->device) != cudaSuccess) {
        cudaGetLastError();
        return sfail(srv, LFD_ERR_CUDA, "cudaSetDevice failed");
    }
    uint64_t need = 0;
    if (lfd_workspace_required(1, lf, &need) != LFD_OK || !lf->views || !lf->labels)
        return sfail(srv, LFD_ERR_INVALID_ARG, "light field of rig %d is malformed", rig_id);
    int64_t S_total = 0;
    for (int v = 0; v < lf->num_views; v++) S_total += (int64_t)lf->grid_w[v] * lf->grid_h[v];

    auto it = srv->rigs.find(rig_id);
    const bool known = it != srv->rigs.end();
    if (known && it->second->queued >= srv->max_pending)
        return sfail(srv, LFD_ERR_BUSY, "rig %d has %d frames in flight", rig_id, it->second->queued);
    // admission: this frame alone (one slot's workspace) with every rig's plane state must fit
    const int64_t cap_after = std::max<int64_t>(known ? it->second->planes_cap : 0, S_total);
    const uint64_t planes_after = planes_bytes(srv) - 16 * (uint64_t)(known ? it->second->planes_cap : 0) +
                                  16 * (uint64_t)cap_after;
    if (srv->budget && need + planes_after > srv->budget)
        return sfail(srv, LFD_ERR_BUDGET, "rig %d needs %llu bytes of workspace and %llu of plane state; the budget "
                     "is %llu", rig_id, (unsigned long long)need, (unsigned long long)planes_after,
                     (unsigned long long)srv->budget);

    if (!known) it = srv->rigs.emplace(rig_id, std::make_unique<Rig>()).first;
    Rig &r = *it->second;
    if (!same_layout(r, lf)) {                       // new rig or changed layout: cold start
        if (r.queued > 0)
            return sfail(srv, LFD_ERR_BUSY, "rig %d changes its layout with frames in flight", rig_id);
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
            if (r.planes) cudaFree(r.planes);        // no frame of the rig is queued or running
            r.planes = nullptr;
            r.planes_cap = 0;
            if (cudaMalloc(&r.planes, 16 * (size_t)S_total) != cudaSuccess) {
                cudaGetLastError();
                return sfail(srv, LFD_ERR_OOM, "rig %d: plane state allocation failed", rig_id);
            }
            r.planes_cap = S_total;
        }
    }

    auto req = std::make_unique<Request>();
    Request &q = *req;
    q.id = srv->next_id++;
    q.rig = rig_id;
    q.rigp = &r;
    q.frame = r.frames;
    q.submit_ns = now_ns();
    q.ws_need = need;
    const int V = lf->num_views;
    q.cams.assign(lf->cams, lf->cams + V);
    q.views.assign(lf->views, lf->views + V);
    q.pitch.assign(V, 0);
    if (lf->view_pitch_bytes) q.pitch.assign(lf->view_pitch_bytes, lf->view_pitch_bytes + V);
    q.labels.assign(lf->labels, lf->labels + V);
    q.gw.assign(lf->grid_w, lf->grid_w + V);
    q.gh.assign(lf->grid_h, lf->grid_h + V);
    q.lf.num_views = V;
    q.lf.fmt = lf->fmt;
    q.lf.cams = q.cams.data();
    q.lf.views = q.views.data();
    q.lf.view_pitch_bytes = q.pitch.data();
    q.lf.labels = q.labels.data();
    q.lf.grid_w = q.gw.data();
    q.lf.grid_h = q.gh.data();
    if (planes_out) q.planes_out.assign(planes_out, planes_out + V);
    if (depth_out) q.depth_out.assign(depth_out, depth_out + V);
    q.p = *params;
    // warm when an earlier frame of this layout is queued or done: frames of a
    // rig run in order, so its planes are there when this one starts
    q.warm = r.has_state && srv->warm_iters > 0;
    if (q.warm) {
        q.p.iterations = srv->warm_iters;
        q.p.warm_iter_offset = srv->warm_off;
    }
    r.has_state = true;
    r.frames++;
    r.queued++;
    *req_id = q.id;
    srv->queue.push_back(&q);
    srv->reqs.emplace(q.id, std::move(req));
    lk.unlock();
    srv->cv.notify_all();
    return LFD_OK;
}

lfd_status lfd_server_poll(lfd_server *srv, uint64_t req_id, int32_t timeout_us, lfd_result *out)
{
    if (!srv) return LFD_ERR_INVALID_ARG;
    Request *qp = nullptr;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->reqs.find(req_id);
        if (it == srv->reqs.end())
            return sfail(srv, LFD_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)req_id);
        qp = it->second.get();
    }
    Request &q = *qp;
    const int64_t deadline = now_ns() + (int64_t)timeout_us * 1000;
    int64_t done = q.done_ns.load(std::memory_order_acquire);
    while (!done) {
        if (timeout_us >= 0 && now_ns() >= deadline) return LFD_ERR_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        done = q.done_ns.load(std::memory_order_acquire);
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    if (out) {
        memset(out, 0, sizeof(*out));
        out->req_id = q.id;
        out->rig_id = q.rig;
        out->warm = q.warm;
        out->frame = q.frame;
        out->submit_ns = q.submit_ns;
        out->done_ns = done;
        out->status = q.status.load();
        out->slot = q.slot;
        out->start_ns = q.start_ns.load();
        out->batch = q.batch;
    }
    if (q.status.load() != LFD_OK) srv->err = srv->batch_err;
    if (q.rigp->queued > 0) q.rigp->queued--;
    srv->reqs.erase(req_id);
    return LFD_OK;
}

namespace {
// wait (lock released) until rig_id has no frame queued or running; false on timeout
bool rig_idle(lfd_server *srv, std::unique_lock<std::mutex> &lk, Rig &r, int64_t timeout_ns)
{
    const int64_t end = now_ns() + timeout_ns;
    for (;;) {
        bool queued = r.inflight.load(std::memory_order_acquire) != 0;
        for (const Request *q : srv->queue) queued = queued || q->rigp == &r;
        if (!queued) return true;
        if (now_ns() > end) return false;
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(100));
        lk.lock();
    }
}
}  // namespace

lfd_status lfd_server_export_state(lfd_server *srv, int32_t rig_id, float *planes_host, int64_t cap_sp, int64_t *n_sp)
{
    if (!srv) return LFD_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->rigs.find(rig_id);
    if (it == srv->rigs.end() || !it->second->has_state)
        return sfail(srv, LFD_ERR_STATE, "rig %d has no plane state", rig_id);
    Rig &r = *it->second;
    if (n_sp) *n_sp = r.S_total;
    if (!planes_host) return LFD_OK;
    if (cap_sp < r.S_total) return sfail(srv, LFD_ERR_INVALID_ARG, "state needs %lld superpixels", (long long)r.S_total);
    if (!rig_idle(srv, lk, r, 60LL * 1000000000LL)) return sfail(srv, LFD_ERR_TIMEOUT, "rig %d stayed busy", rig_id);
    if (cudaSetDevice(srv->device) != cudaSuccess ||
        cudaMemcpy(planes_host, r.planes, 16 * (size_t)r.S_total, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return sfail(srv, LFD_ERR_CUDA, "state export failed");
    }
    return LFD_OK;
}

lfd_status lfd_server_import_state(lfd_server *srv, int32_t rig_id, const float *planes_host, int64_t n_sp)
{
    if (!srv || !planes_host) return LFD_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->rigs.find(rig_id);
    if (it == srv->rigs.end() || !it->second->planes)
        return sfail(srv, LFD_ERR_STATE, "rig %d has not submitted a frame", rig_id);
    Rig &r = *it->second;
    if (n_sp != r.S_total)
        return sfail(srv, LFD_ERR_INVALID_ARG, "state has %lld superpixels, rig %d has %lld", (long long)n_sp, rig_id,
                     (long long)r.S_total);
    if (!rig_idle(srv, lk, r, 60LL * 1000000000LL)) return sfail(srv, LFD_ERR_TIMEOUT, "rig %d stayed busy", rig_id);
    if (cudaSetDevice(srv->device) != cudaSuccess ||
        cudaMemcpy(r.planes, planes_host, 16 * (size_t)n_sp, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return sfail(srv, LFD_ERR_CUDA, "state import failed");
    }
    r.has_state = true;
    return LFD_OK;
}

}  // extern "C"
