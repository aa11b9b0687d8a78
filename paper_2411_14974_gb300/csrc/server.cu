// Serving runtime: continuous batching of novel-view requests over resident scenes.
//
// Threads:
//   caller threads   cs_server_submit queues a request (scene, camera, output buffer);
//   worker           admits queued requests in arrival order into a batch (at most max_batch
//                    views, same K, estimated transient memory within the budget left by the
//                    batches still on the GPU), orders the batch's views by estimated cost
//                    (smallest first), runs the batched forward (one preprocess, binning and sort
//                    for all views, then one persistent blend launch over the views' tiles, view
//                    by view, which raises each view's flag in mapped host memory once the view's
//                    image is written; batches of more than 32 views: one blend launch per view,
//                    each followed by that view's event) on one of two streams and goes back for
//                    the next batch -- so the preprocess and sorts of batch k+1 overlap the blends
//                    of batch k (at most one batch in flight per stream);
//   finisher         waits for the batches in order and, within a batch, for each view's flag (or
//                    event), posting each request's completion as soon as its own image is
//                    written; then frees the batch's buffers and returns its memory to the
//                    budget.
#include <cstring>
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "cs_api_internal.h"
#include "cs_common.cuh"

using namespace cs;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    uint64_t id;
    int32_t scene;
    cs_camera cam;
    float *image;
    Clock::time_point t_submit, t_admit;
    size_t est;
};

struct Scene {
    cs_scene sc;
    bool alive = true;
    double pairs_per_convex = 8.0;  // tile pairs per convex at 1920x1080, learnt from past batches
    int64_t busy = 0;               // views of this scene in admitted batches
};

struct Batch {
    std::vector<Request> reqs;
    std::vector<cudaEvent_t> view_done;  // one per request, recorded after its view's blend
    cs_fwd_state *state = nullptr;
    cudaEvent_t done = nullptr;
    size_t est = 0;
    cs_status status = CS_OK;
    double weighted_views = 0.0;  // sum of N * pixels / (1920 * 1080) over its views
    // with one persistent blend launch: the batch's flag slots (its stream's) and the value its
    // launch stores there per view; NULL: per-view launches, completions from view_done
    volatile uint32_t *flags = nullptr;
    uint32_t seq = 0;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct cs_server {
    int device = 0;
    size_t budget = 0;
    int max_batch = 1;
    bool pipelined = true;  // false: each batch finishes on the GPU before the next is admitted
    cs_settings settings{};
    cs_context *ctx = nullptr;
    cudaStream_t streams[2] = {nullptr, nullptr};
    int next_stream = 0;
    // per stream, MAX_ORDER_VIEWS completion flags of the batch in flight on it (mapped pinned
    // memory: host and device addresses)
    uint32_t *flags_host = nullptr, *flags_dev = nullptr;

    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_mem, cv_poll;
    std::deque<Request> pending;
    std::deque<Batch *> inflight;
    std::deque<cs_completion> completions;
    std::map<int32_t, Scene> scenes;
    int32_t next_scene = 0;
    uint64_t next_id = 1;
    size_t inflight_bytes = 0;
    bool stop = false;
    uint64_t n_completed = 0, n_batches = 0, max_batch_seen = 0, peak_bytes = 0;
    std::thread worker, finisher;

    size_t estimate(const Scene &s, const cs_camera &c) const {
        const double px = (double)c.width * c.height;
        const double pairs = s.pairs_per_convex * (double)s.sc.n * (px / (1920.0 * 1080.0)) + 64.0;
        const double tiles = (double)((c.width + 15) / 16) * ((c.height + 15) / 16);
        // records, keys, counts, rects, pixel boxes, tile-test radii, depth-sort buffers and offsets
        // (about 185 bytes per convex); pairs and their sort buffers; per pixel T_final and last
        // contributor; tile ranges
        return (size_t)((double)s.sc.n * 192.0 + pairs * 16.0 + px * 8.0 + tiles * 8.0 + 4096.0);
    }

    // bytes the pool has handed out and not yet taken back (the batches' real allocations)
    size_t pool_used() const {
        uint64_t used = 0;
        if (cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) return 0;
        return (size_t)used;
    }

    void complete_locked(const Request &r, cs_status st, int batch, Clock::time_point now) {
        cs_completion c;
        c.id = r.id;
        c.status = st;
        c.batch_size = batch;
        c.queue_ms = ms_between(r.t_submit, batch > 0 ? r.t_admit : now);
        c.latency_ms = ms_between(r.t_submit, now);
        completions.push_back(c);
        ++n_completed;
        cv_poll.notify_all();
    }

    void run_worker();
    void run_finisher();
};

void cs_server::run_worker() {
    cudaSetDevice(device);
    for (;;) {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || !pending.empty(); });
        if (pending.empty()) {
            if (stop) break;
            continue;
        }
        // one batch in flight per stream: running further ahead cannot feed the GPU faster, it only
        // holds memory (and makes the pool grow) while requests that could join a batch wait
        if (inflight.size() >= 2) {
            cv_mem.wait(lk);
            continue;
        }
        Batch *b = new (std::nothrow) Batch();
        if (!b) continue;
        int K = -1;
        size_t est = 0;
        const Clock::time_point now = Clock::now();
        // memory taken by the batches on the GPU: their estimates, or what the pool really holds
        // for them when that is more (nothing is held once none is in flight)
        size_t held = inflight_bytes;
        if (!inflight.empty()) {
            const size_t used = pool_used();
            if (used > held) held = used;
        }
        for (auto it = pending.begin(); it != pending.end() && (int)b->reqs.size() < max_batch;) {
            auto sit = scenes.find(it->scene);
            if (sit == scenes.end() || !sit->second.alive) {
                complete_locked(*it, CS_ERR_STATE, 0, now);
                it = pending.erase(it);
                continue;
            }
            Scene &sc = sit->second;
            if (K >= 0 && sc.sc.k != K) {  // one K per batch; keep arrival order for the rest
                ++it;
                continue;
            }
            const size_t e = estimate(sc, it->cam);
            if (e > budget) {
                complete_locked(*it, CS_ERR_BUDGET, 0, now);
                it = pending.erase(it);
                continue;
            }
            if (held + est + e > budget) break;  // wait until batches on the GPU free memory
            K = sc.sc.k;
            est += e;
            it->t_admit = now;
            it->est = e;
            b->reqs.push_back(*it);
            it = pending.erase(it);
        }
        if (b->reqs.empty()) {
            delete b;
            if (!inflight.empty()) cv_mem.wait(lk);  // memory frees up when a batch finishes
            continue;
        }
        // cheapest views first: their images are written, and their requests completed, first
        std::stable_sort(b->reqs.begin(), b->reqs.end(),
                         [](const Request &x, const Request &y) { return x.est < y.est; });
        b->est = est;
        inflight_bytes += est;
        if (inflight_bytes > peak_bytes) peak_bytes = inflight_bytes;
        for (const Request &r : b->reqs) scenes[r.scene].busy++;
        // describe the views while the scene table is locked
        cs_fwd_state *s = new (std::nothrow) cs_fwd_state();
        if (s) {
            s->ctx = ctx;
            s->k = K;
            s->settings = settings;
            s->st = to_settings(settings);
            s->views.resize(b->reqs.size());
            for (size_t v = 0; v < b->reqs.size(); ++v) {
                const Request &r = b->reqs[v];
                const cs_scene &sc = scenes[r.scene].sc;
                ViewDesc &vd = s->views[v];
                fill_view(vd, r.cam);
                vd.points = sc.points; vd.delta = sc.delta; vd.sigma = sc.sigma;
                vd.opacity = sc.opacity; vd.sh = sc.sh;
                vd.n = sc.n; vd.k = sc.k; vd.sh_degree = sc.sh_degree; vd.activation = sc.activation; vd.storage = sc.storage;
                vd.image = r.image;
                vd.t_final = nullptr;
                b->weighted_views += (double)sc.n * ((double)r.cam.width * r.cam.height / (1920.0 * 1080.0));
            }
        }
        lk.unlock();

        const int sidx = next_stream;
        cudaStream_t stream = streams[sidx];
        next_stream ^= 1;
        if (s && flags_dev && b->reqs.size() <= (size_t)MAX_ORDER_VIEWS) {
            // one persistent blend launch for the batch; its flags carry the batch's number, so
            // that values left by the stream's earlier batches never read as complete
            b->seq = (uint32_t)(n_batches + 1);
            b->flags = flags_host + sidx * MAX_ORDER_VIEWS;
            s->view_flags = flags_dev + sidx * MAX_ORDER_VIEWS;
            s->flag_value = b->seq;
        }
        if (s) {
            b->view_done.assign(b->reqs.size(), nullptr);
            for (cudaEvent_t &e : b->view_done)
                if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) e = nullptr;
            bool all = true;
            for (cudaEvent_t e : b->view_done) all = all && e;
            if (all) s->view_done = b->view_done;  // else one blend launch, completions at the batch's end
        }
        if (!s) {
            b->status = fail(CS_ERR_NOMEM, "out of host memory");
        } else {
            b->state = s;
            b->status = run_forward(ctx, s, stream);
        }
        if (cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess) cudaEventRecord(b->done, stream);
        if (!pipelined) cudaStreamSynchronize(stream);  // no overlap between batches

        lk.lock();
        inflight.push_back(b);
        ++n_batches;
        if (b->reqs.size() > max_batch_seen) max_batch_seen = b->reqs.size();
        cv_done.notify_all();
    }
    std::lock_guard<std::mutex> lk(mu);
    cv_done.notify_all();
}

void cs_server::run_finisher() {
    cudaSetDevice(device);
    for (;;) {
        Batch *b = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_done.wait(lk, [&] { return !inflight.empty() || (stop && pending.empty()); });
            if (inflight.empty()) {
                if (stop && pending.empty()) break;
                continue;
            }
            b = inflight.front();
        }
        cs_status st = b->status;
        const bool per_view = b->state && b->state->view_done.size() == b->reqs.size() && st == CS_OK;
        // each view's request completes once its own blend has run (an event that was never
        // recorded, after a failed forward, reads as complete)
        for (size_t v = 0; v < b->view_done.size(); ++v) {
            cudaEvent_t ev = b->view_done[v];
            cudaError_t e = cudaSuccess;
            if (ev && per_view) {
                // complete once the view's flag carries this batch's number (persistent launch) or
                // its event has passed (per-view launches; with the persistent launch, the end of
                // the whole batch)
                while (!(b->flags && b->flags[v] == b->seq) && (e = cudaEventQuery(ev)) == cudaErrorNotReady)
                    std::this_thread::sleep_for(std::chrono::microseconds(20));
                if (b->flags && b->flags[v] == b->seq) e = cudaSuccess;
                if (e == cudaSuccess) {
                    std::lock_guard<std::mutex> lk(mu);
                    complete_locked(b->reqs[v], CS_OK, (int)b->reqs.size(), Clock::now());
                    b->reqs[v].id = 0;  // posted
                } else if (st == CS_OK) {
                    st = fail_cuda(e, "server view");
                }
            }
        }
        if (b->done) {
            cudaError_t e;
            while ((e = cudaEventQuery(b->done)) == cudaErrorNotReady)
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            if (e != cudaSuccess && st == CS_OK) st = fail_cuda(e, "server batch");
            cudaEventDestroy(b->done);
        }
        for (cudaEvent_t ev : b->view_done)
            if (ev) cudaEventDestroy(ev);
        const Clock::time_point now = Clock::now();
        int64_t pairs = b->state ? b->state->n_pairs : 0;
        if (b->state) state_free(b->state);
        {
            std::lock_guard<std::mutex> lk(mu);
            inflight.pop_front();
            inflight_bytes -= b->est;
            const double observed = b->weighted_views > 0 ? (double)pairs / b->weighted_views : 0.0;
            for (const Request &r : b->reqs) {
                Scene &sc = scenes[r.scene];
                sc.busy--;
                if (st == CS_OK && observed > sc.pairs_per_convex) sc.pairs_per_convex = observed;
                if (r.id) complete_locked(r, st, (int)b->reqs.size(), now);
            }
            cv_mem.notify_all();
            cv_work.notify_all();
        }
        delete b;
    }
}

// ---------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------
extern "C" cs_status cs_server_create(int32_t device, size_t budget, int32_t max_batch, const cs_settings *settings,
                                      cs_server **out) {
    if (!out) return fail(CS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (max_batch < 1 || max_batch > 1024) return fail(CS_ERR_ARG, "max_batch must be in 1..1024");
    if (budget == 0) return fail(CS_ERR_ARG, "memory budget must be > 0");
    cs_status st = check_settings(settings);
    if (st != CS_OK) return st;
    cs_context *ctx = nullptr;
    if ((st = cs_context_create(device, &ctx)) != CS_OK) return st;
    cs_server *srv = new (std::nothrow) cs_server();
    if (!srv) {
        cs_context_destroy(ctx);
        return fail(CS_ERR_NOMEM, "out of host memory");
    }
    srv->device = device;
    srv->budget = budget;
    srv->max_batch = max_batch;
    srv->settings = *settings;
    srv->ctx = ctx;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    for (int i = 0; i < 2; ++i) {
        cudaError_t e = cudaStreamCreateWithFlags(&srv->streams[i], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaStreamDestroy(srv->streams[j]);
            cs_context_destroy(ctx);
            delete srv;
            cudaSetDevice(prev);
            return fail_cuda(e, "cudaStreamCreate");
        }
    }
    uint64_t zero = 0;  // the pool is the server's own: its high-water mark counts from here
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrUsedMemHigh, &zero);
    // completion flags of the persistent blend launches (without them: one launch per view)
    const size_t fbytes = 2 * MAX_ORDER_VIEWS * sizeof(uint32_t);
    if (cudaHostAlloc((void **)&srv->flags_host, fbytes, cudaHostAllocMapped) == cudaSuccess) {
        memset(srv->flags_host, 0, fbytes);
        if (cudaHostGetDevicePointer((void **)&srv->flags_dev, srv->flags_host, 0) != cudaSuccess) {
            cudaFreeHost(srv->flags_host);
            srv->flags_host = nullptr;
            srv->flags_dev = nullptr;
        }
    } else {
        srv->flags_host = nullptr;
    }
    cudaGetLastError();  // a failed flag allocation is not an error of the server
    cudaSetDevice(prev);
    srv->worker = std::thread([srv] { srv->run_worker(); });
    srv->finisher = std::thread([srv] { srv->run_finisher(); });
    *out = srv;
    return CS_OK;
}

extern "C" void cs_server_destroy(cs_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    srv->cv_mem.notify_all();
    srv->cv_done.notify_all();
    srv->worker.join();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->cv_done.notify_all();
    }
    srv->finisher.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->device);
    for (cudaStream_t s : srv->streams)
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    if (srv->flags_host) cudaFreeHost(srv->flags_host);
    cudaSetDevice(prev);
    cs_context_destroy(srv->ctx);
    delete srv;
}

extern "C" cs_status cs_server_set_pipelining(cs_server *srv, int32_t on) {
    if (!srv) return fail(CS_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->pipelined = on != 0;
    return CS_OK;
}

extern "C" cs_status cs_server_add_scene(cs_server *srv, const cs_scene *scene, int32_t *scene_id) {
    if (!srv || !scene_id) return fail(CS_ERR_ARG, "server and scene_id are required");
    cs_status st = check_scene(scene);
    if (st != CS_OK) return st;
    std::lock_guard<std::mutex> lk(srv->mu);
    const int32_t id = srv->next_scene++;
    Scene s;
    s.sc = *scene;
    srv->scenes[id] = s;
    *scene_id = id;
    return CS_OK;
}

extern "C" cs_status cs_server_remove_scene(cs_server *srv, int32_t scene_id) {
    if (!srv) return fail(CS_ERR_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->scenes.find(scene_id);
    if (it == srv->scenes.end() || !it->second.alive) return fail(CS_ERR_STATE, "unknown scene %d", scene_id);
    it->second.alive = false;
    const Clock::time_point now = Clock::now();
    for (auto p = srv->pending.begin(); p != srv->pending.end();) {
        if (p->scene == scene_id) {
            srv->complete_locked(*p, CS_ERR_STATE, 0, now);
            p = srv->pending.erase(p);
        } else {
            ++p;
        }
    }
    // admitted batches finish on their own (the GPU never waits on anything); bound the wait anyway
    const bool idle = srv->cv_mem.wait_for(lk, std::chrono::seconds(120),
                                           [&] { return srv->scenes[scene_id].busy == 0; });
    if (!idle) return fail(CS_ERR_TIMEOUT, "scene %d still in use after 120 s", scene_id);
    srv->scenes.erase(scene_id);
    return CS_OK;
}

extern "C" cs_status cs_server_submit(cs_server *srv, int32_t scene_id, const cs_camera *cam, float *image,
                                      uint64_t *request_id) {
    if (!srv || !cam || !image) return fail(CS_ERR_ARG, "server, camera and image are required");
    cs_status st = check_camera(cam);
    if (st != CS_OK) return st;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return fail(CS_ERR_STATE, "server is shutting down");
    auto it = srv->scenes.find(scene_id);
    if (it == srv->scenes.end() || !it->second.alive) return fail(CS_ERR_ARG, "unknown scene %d", scene_id);
    Request r;
    r.id = srv->next_id++;
    r.scene = scene_id;
    r.cam = *cam;
    r.image = image;
    r.t_submit = Clock::now();
    r.t_admit = r.t_submit;
    r.est = 0;
    srv->pending.push_back(r);
    if (request_id) *request_id = r.id;
    srv->cv_work.notify_one();
    return CS_OK;
}

extern "C" cs_status cs_server_poll(cs_server *srv, cs_completion *out, int32_t max, int32_t *n_out, int32_t wait_ms) {
    if (!srv || !n_out || (max > 0 && !out)) return fail(CS_ERR_ARG, "server, out and n_out are required");
    std::unique_lock<std::mutex> lk(srv->mu);
    if (srv->completions.empty() && wait_ms > 0)
        srv->cv_poll.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !srv->completions.empty(); });
    int32_t n = 0;
    while (n < max && !srv->completions.empty()) {
        out[n++] = srv->completions.front();
        srv->completions.pop_front();
    }
    *n_out = n;
    return CS_OK;
}

extern "C" cs_status cs_server_stats(cs_server *srv, uint64_t *stats) {
    if (!srv || !stats) return fail(CS_ERR_ARG, "server and stats are required");
    std::lock_guard<std::mutex> lk(srv->mu);
    uint64_t on_gpu = 0;
    for (const Batch *b : srv->inflight) on_gpu += b->reqs.size();
    stats[0] = srv->n_completed;
    stats[1] = srv->n_batches;
    stats[2] = srv->max_batch_seen;
    stats[3] = srv->peak_bytes;
    stats[4] = srv->pending.size();
    stats[5] = on_gpu;
    uint64_t high = 0;
    if (cudaMemPoolGetAttribute(srv->ctx->pool, cudaMemPoolAttrUsedMemHigh, &high) != cudaSuccess) high = 0;
    stats[6] = high;
    return CS_OK;
}
