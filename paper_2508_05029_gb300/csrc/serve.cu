// Request server: continuous admission of queries onto concurrent lanes.
//
// Paper basis: Section 3.3.1 (Compute Executor threads each drive their own
// CUDA stream and take tasks from a queue), Section 3.3.2 (tasks reserve
// device memory before they run; the reservation decides when a task may
// start).  Each worker thread owns a lane (compute stream, copy stream,
// pinned status words).  A worker admits the oldest queued request whose plan
// is not already running, as long as fewer than max_inflight run; the request
// executes on the worker's lane, overlapping on the device with the others.
// A request whose reservation does not fit goes back to the head of the queue
// and is retried after the next completion releases memory (idle cached join
// tables are evicted first); it fails with TP_E_BUDGET only when nothing else
// is running.
#include <chrono>

#include "tp_internal.h"

using namespace tp;

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    uint64_t ticket = 0;
    tp_plan* plan = nullptr;
    bool done = false;
    tp_status status = TP_OK;
    std::string message;
    tp_result* result = nullptr;
    int64_t t_submit = 0, t_start = 0, t_end = 0;
};

}  // namespace

struct tp_server {
    tp_engine* e = nullptr;
    int max_inflight = 1;
    bool cache_on = false;
    std::vector<Lane> lanes;
    std::vector<std::thread> threads;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> queue;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::map<const tp_plan*, int> running;
    uint64_t next_ticket = 1;
    int inflight = 0;
    bool stopping = false;
    uint64_t completions = 0;
    tp_server_stats stats{};
    DimCache cache;
};

namespace {

// Next admissible request (caller holds sv->mu), or nullptr.
Request* pick(tp_server* sv) {
    if (sv->inflight >= sv->max_inflight) return nullptr;
    for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
        if (sv->running.count((*it)->plan)) continue;
        Request* r = *it;
        sv->queue.erase(it);
        return r;
    }
    return nullptr;
}

void worker(tp_server* sv, int idx) {
    Lane& lane = sv->lanes[idx];
    cudaSetDevice(sv->e->device);
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait(lk, [&] {
                return (sv->stopping && sv->queue.empty()) ||
                       (sv->inflight < sv->max_inflight && !sv->queue.empty() && (r = pick(sv)) != nullptr);
            });
            if (!r) return;   // stopping and nothing left
            ++sv->inflight;
            ++sv->running[r->plan];
            if ((uint32_t)sv->inflight > sv->stats.inflight_peak) sv->stats.inflight_peak = (uint32_t)sv->inflight;
            if (!r->t_start) r->t_start = now_ns();
        }
        tp_result* res = nullptr;
        DimCache* cache = sv->cache_on ? &sv->cache : nullptr;
        tp_status st = execute_on_lane(r->plan, &lane, cache, &res);
        if (st == TP_E_BUDGET && cache && cache_evict_idle(sv->e, cache, 0) > 0)
            st = execute_on_lane(r->plan, &lane, cache, &res);
        // the execution synchronised its lane; the result's memory may be freed
        // on the engine's stream, which outlives the server's lanes
        if (res) res->stream = nullptr;
        std::unique_lock<std::mutex> lk(sv->mu);
        --sv->inflight;
        if (--sv->running[r->plan] == 0) sv->running.erase(r->plan);
        if (st == TP_E_BUDGET && sv->inflight > 0) {
            // others hold memory: retry this request after the next completion
            sv->queue.push_front(r);
            ++sv->stats.budget_waits;
            const uint64_t c0 = sv->completions;
            sv->cv.wait_for(lk, std::chrono::milliseconds(200), [&] { return sv->completions != c0; });
            sv->cv.notify_all();
            continue;
        }
        r->status = st;
        r->message = st ? tp_last_error() : "";
        r->result = res;
        r->t_end = now_ns();
        r->done = true;
        ++sv->completions;
        if (st) ++sv->stats.failed;
        else ++sv->stats.completed;
        sv->cv.notify_all();
    }
}

}  // namespace

extern "C" {

tp_status tp_server_start(tp_engine* e, int32_t workers, int32_t max_inflight, uint32_t flags, tp_server** out) {
    clear_error();
    if (!e || !out || workers < 1 || workers > 64 || max_inflight < 0)
        return fail(TP_E_INVALID, "tp_server_start: bad arguments");
    *out = nullptr;
    std::unique_ptr<tp_server> sv(new (std::nothrow) tp_server());
    if (!sv) return fail(TP_E_NOMEM, "tp_server_start: out of host memory");
    sv->e = e;
    sv->max_inflight = max_inflight ? max_inflight : workers;
    sv->cache_on = (flags & TP_SERVE_CACHE_DIM) != 0;
    TP_TRY_CUDA(cudaSetDevice(e->device));
    sv->lanes.resize(workers);
    for (Lane& l : sv->lanes) {
        TP_TRY_CUDA(cudaStreamCreateWithFlags(&l.compute, cudaStreamNonBlocking));
        TP_TRY_CUDA(cudaStreamCreateWithFlags(&l.copy, cudaStreamNonBlocking));
        TP_TRY_CUDA(cudaStreamCreateWithFlags(&l.spill, cudaStreamNonBlocking));
        TP_TRY_CUDA(cudaHostAlloc((void**)&l.host_words, 4096, cudaHostAllocDefault));
    }
    for (int i = 0; i < workers; ++i) sv->threads.emplace_back(worker, sv.get(), i);
    *out = sv.release();
    return TP_OK;
}

tp_status tp_submit(tp_server* sv, tp_plan* p, tp_ticket* out) {
    clear_error();
    if (!sv || !p || !out || p->eng != sv->e) return fail(TP_E_INVALID, "tp_submit: bad arguments");
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return fail(TP_E_NOMEM, "tp_submit: out of host memory");
    r->plan = p;
    r->t_submit = now_ns();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stopping) return fail(TP_E_INVALID, "tp_submit: server is stopping");
    r->ticket = sv->next_ticket++;
    *out = r->ticket;
    sv->queue.push_back(r.get());
    sv->reqs[r->ticket] = std::move(r);
    ++sv->stats.submitted;
    sv->cv.notify_all();
    return TP_OK;
}

tp_status tp_wait(tp_server* sv, tp_ticket t, int64_t timeout_ns, tp_result** out, int64_t* times) {
    clear_error();
    if (!sv || !out) return fail(TP_E_INVALID, "tp_wait: NULL argument");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(t);
    if (it == sv->reqs.end()) return fail(TP_E_INVALID, "tp_wait: unknown ticket %llu", (unsigned long long)t);
    Request* r = it->second.get();
    auto ready = [&] { return r->done; };
    if (timeout_ns < 0) sv->cv.wait(lk, ready);
    else if (!sv->cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns), ready))
        return fail(TP_E_TIMEOUT, "tp_wait: ticket %llu not finished", (unsigned long long)t);
    if (times) {
        times[0] = r->t_submit;
        times[1] = r->t_start;
        times[2] = r->t_end;
    }
    const tp_status st = r->status;
    if (st == TP_OK) *out = r->result;
    else fail(st, "%s", r->message.c_str());
    sv->reqs.erase(it);
    return st;
}

tp_status tp_server_stats_get(tp_server* sv, tp_server_stats* out) {
    if (!sv || !out) return fail(TP_E_INVALID, "tp_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    std::lock_guard<std::mutex> lc(sv->cache.mu);
    out->cache_hits = sv->cache.hits;
    out->cache_misses = sv->cache.misses;
    out->cache_evictions = sv->cache.evictions;
    return TP_OK;
}

void tp_server_stop(tp_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv.notify_all();
    for (auto& th : sv->threads) th.join();
    cudaSetDevice(sv->e->device);
    for (Lane& l : sv->lanes) {
        cudaStreamSynchronize(l.compute);
        cudaStreamSynchronize(l.copy);
        cudaStreamSynchronize(l.spill);
    }
    for (auto& kv : sv->reqs)   // finished but never collected
        if (kv.second->result) tp_result_free(kv.second->result);
    cache_evict_idle(sv->e, &sv->cache, 0);
    for (Lane& l : sv->lanes) {
        cudaStreamDestroy(l.compute);
        cudaStreamDestroy(l.copy);
        cudaStreamDestroy(l.spill);
        cudaFreeHost(l.host_words);
    }
    delete sv;
}

}  // extern "C"
