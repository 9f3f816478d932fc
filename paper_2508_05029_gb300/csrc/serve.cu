// Request server: continuous batching of arriving queries, with concurrent
// lanes for the queries a batched launch cannot take.
//
// Paper basis: Section 3.3.1 (Compute Executor threads drive their own CUDA
// streams and take tasks from a queue), Section 3.3.2 (tasks reserve device
// memory before they run; the reservation decides when a task may start).
//
// Batching (TP_SERVE_BATCH): a dispatcher thread takes every queued request
// that a batched launch can run (device-resident tables, one join, at most
// SERVE_BATCH_MAX_ROWS fact rows), as many as the device budget admits, and
// starts them together as one persistent queue kernel (batch.cu: probe tiles
// and finalisations of all of them, claimed by resident CTAs) on one of two
// launch slots, each with its own stream.  Requests that arrive while a batch
// runs form the next batch, which starts at once on the other slot, so its
// work overlaps the running batch's tail on the device; a completion thread
// hands out the results of each finished batch in launch order.  Join tables
// are cached across batches (keyed by dimension table, its row count, key
// column, dimension fields, predicate and table shape) and built by a
// whole-GPU build launch the first time; a batch that needs a table another
// slot is still building waits for that build on its stream.  Each request
// keeps its own result arrays, accumulators and error word, so its result is
// the one it gets alone.  The probe tasks are compiled at run time for the
// shapes of every plan the server has seen (one kernel for all of them,
// rebuilt by the next batch after a new shape arrives); without run-time
// compilation the ahead-of-time queue kernel runs them.  Larger requests gain nothing from
// sharing a launch -- their own fused kernel streams at HBM rate -- and run
// on lanes.
//
// A lone batchable request on an idle GPU (nothing queued with it, no batch
// or lane execution in flight) does not wait for company: the dispatcher runs
// it at once on its own lane as a single query, with the cached join tables.
//
// Lanes: worker threads, each owning a lane (compute, copy and spill
// streams, pinned status words), run the other requests one tp_execute at a
// time, overlapping on the device; with batching off they run every request.
// A lane admits the oldest queued request whose plan is not already running,
// while fewer than max_inflight run.  A request whose reservation does not fit
// goes back to the head of the queue and is retried after the next
// completion releases memory (idle cached join tables are evicted first); it
// fails with TP_E_BUDGET only when nothing else ran while it tried.
#include <algorithm>
#include <chrono>
#include <cmath>

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
    bool batchable = false;   // runs in a batched launch (TP_SERVE_BATCH)
    bool done = false;
    bool waited = false;      // a tp_wait is blocked on it
    tp_status status = TP_OK;
    std::string message;
    tp_result* result = nullptr;
    int64_t t_submit = 0, t_start = 0, t_end = 0;
};

uint64_t a256(uint64_t x) { return (x + 255) & ~255ull; }

constexpr uint64_t SERVE_WAIT_NS = 2000000000ull;   // limit of every dependency wait of a batched launch
constexpr int N_SLOTS = 2;                          // batched launches in flight at once
constexpr uint64_t SERVE_BATCH_MAX_ROWS = 4ull << 20;   // larger fact tables run on lanes

// A join table kept for batched requests.  Its allocation holds the slots,
// then the side cell (2 words) and the build's error word.
struct JEntry {
    void* mem = nullptr;
    uint64_t bytes = 0;          // reserved in the engine budget
    uint64_t slot_bytes = 0;
    uint32_t* side = nullptr;
    uint32_t* err = nullptr;
    cudaEvent_t built = nullptr; // recorded after its build launch
    int users = 0;               // launched batches that read it and have not finished
    uint64_t last_use = 0;
    tp_status bad = TP_OK;       // its build's error, known once the building batch finished
    bool checked = false;
};

// What the dispatcher keeps per plan: its batched sizes and its shape id in
// the server's run-time compiled queue kernel.
struct PlanInfo {
    BatchPrep x;
    int shape = 0;
    uint64_t result_bytes = 0;   // result arrays for 2^key_bits groups
};

// One batched launch in flight.
struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    unsigned char* h_stage = nullptr;   // pinned: descriptors and tasks (to the device), then status words (back)
    uint64_t h_cap = 0;
    void* arena = nullptr;
    uint64_t reserved = 0;
    uint64_t status_off = 0;            // offset of the status words in h_stage
    std::vector<Request*> reqs;
    std::vector<tp_result*> res;
    std::vector<JEntry*> joins;         // per request: its cached join table (or nullptr)
    std::vector<std::pair<JEntry*, uint64_t>> built;   // tables built by this batch, offset of their error word
    bool busy = false;
};

}  // namespace

struct tp_server {
    tp_engine* e = nullptr;
    int max_inflight = 1;
    bool cache_on = false;
    bool batch_on = false;
    int max_batch = 256;
    std::vector<Lane> lanes;
    std::vector<std::thread> threads;
    std::mutex mu;
    // lane workers, the dispatcher, the completion thread, and whoever waits
    // for a finished request (tp_wait, budget retries) each wait on their own
    std::condition_variable cv_lane, cv_disp, cv_comp, cv_done;
    std::deque<Request*> queue;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::map<const tp_plan*, int> running;
    uint64_t next_ticket = 1;
    int inflight = 0;               // lane executions running
    bool stopping = false;
    uint64_t completions = 0;
    tp_server_stats stats{};
    DimCache cache;
    // batching
    Slot slots[N_SLOTS];
    std::deque<int> launched;       // busy slots in launch order
    bool dispatcher_done = false;
    std::thread dispatcher, completer;
    std::map<std::pair<const tp_plan*, uint64_t>, PlanInfo> plans;   // by plan and its serial; dispatcher only
    std::map<std::string, int> shape_ids;       // dispatcher thread only
    std::vector<std::string> shapes;
    const void* kernel = nullptr;               // nullptr: the ahead-of-time queue kernel
    bool kernel_stale = false;                  // shapes were added since it was compiled
    std::map<std::pair<const void*, uint32_t>, int> grids;
    std::map<std::string, JEntry> joins;        // created by the dispatcher; users/last_use under mu
    uint64_t join_tick = 0;
    Lane dlane;                                 // the dispatcher's own lane: a lone request on an idle GPU
};

namespace {

void finish(tp_server* sv, Request* r, tp_status st, const std::string& msg, tp_result* res) {
    r->status = st;
    r->message = msg;
    r->result = res;
    r->t_end = now_ns();
    r->done = true;
    ++sv->completions;
    if (st) ++sv->stats.failed;
    else ++sv->stats.completed;
    sv->cv_done.notify_all();
}

// ------------------------------------------------------------------ lanes

// Next request for a lane (caller holds sv->mu), or nullptr.
Request* pick(tp_server* sv) {
    if (sv->inflight >= sv->max_inflight) return nullptr;
    for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
        if ((*it)->batchable || sv->running.count((*it)->plan)) continue;
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
        uint64_t c0 = 0;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_lane.wait(lk, [&] {
                bool lane_work = false;
                for (Request* q : sv->queue) lane_work = lane_work || !q->batchable;
                return (sv->stopping && !lane_work) ||
                       (sv->inflight < sv->max_inflight && lane_work && (r = pick(sv)) != nullptr);
            });
            if (!r) return;   // stopping and nothing left for lanes
            ++sv->inflight;
            ++sv->running[r->plan];
            if ((uint32_t)sv->inflight > sv->stats.inflight_peak) sv->stats.inflight_peak = (uint32_t)sv->inflight;
            if (!r->t_start) r->t_start = now_ns();
            c0 = sv->completions;   // completions before this attempt
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
        const bool others = sv->inflight > 0 || !sv->launched.empty() || sv->completions != c0;
        if (st == TP_E_BUDGET && others) {
            // memory is or was held by other requests: retry after the next completion
            sv->queue.push_front(r);
            ++sv->stats.budget_waits;
            const uint64_t c1 = sv->completions;
            if (c1 == c0)
                sv->cv_done.wait_for(lk, std::chrono::milliseconds(200), [&] { return sv->completions != c1; });
            sv->cv_lane.notify_all();
            continue;
        }
        finish(sv, r, st, st ? tp_last_error() : "", res);
        sv->cv_lane.notify_all();
        sv->cv_disp.notify_one();
    }
}

// --------------------------------------------------------------- batching

// The dispatcher's record of p: sizes with probe tiles that spread one query
// over the whole GPU, and its shape in the server's kernel (a new shape
// rebuilds the kernel).
const PlanInfo& plan_info(tp_server* sv, tp_plan* p) {
    auto it = sv->plans.find({p, p->serial});
    if (it != sv->plans.end()) return it->second;
    PlanInfo pi;
    // rows per warp: about four tiles per SM for this query alone, 128..1024
    const uint64_t per = p->d.fact->rows / ((uint64_t)(tpk::BATCH_THREADS / 32) * 4 * (uint64_t)sv->e->num_sms);
    uint32_t rpw = 128;
    while (rpw < 1024 && rpw < per) rpw <<= 1;
    batch_prep(sv->e, p, 0.0f, rpw, TP_AGG_AUTO, &pi.x);
    int n_avg = 0;
    for (int a = 0; a < p->d.n_agg; ++a) n_avg += p->d.aggs[a].kind == TP_AGG_AVG;
    const uint64_t G = 1ull << p->key_bits;
    pi.result_bytes = a256(G * 8) * 2 + a256(G * 16) * p->n_sum + a256(G * 8) * n_avg;
    if (!(sv->e->cfg.flags & TP_FLAG_NO_JIT)) {
        tpk::BatchQuery B;
        tpk::OutDev od{};
        batch_query_desc(p, pi.x, nullptr, nullptr, nullptr, nullptr, od, &B);
        const std::string key = batch_shape(p, B, pi.x, "JS_");
        auto s = sv->shape_ids.find(key);
        if (s == sv->shape_ids.end()) {
            // compiled with the others when the next batch launches
            const int id = (int)sv->shapes.size();
            s = sv->shape_ids.emplace(key, id).first;
            sv->shapes.push_back(batch_shape(p, B, pi.x, "JS_" + std::to_string(id)));
            sv->kernel_stale = true;
        }
        pi.shape = s->second;
    }
    return sv->plans.emplace(std::make_pair(p, p->serial), pi).first->second;
}

std::string join_key(const tp_plan* p, const BatchPrep& x) {
    const tp_plan_desc& d = p->d;
    char buf[256];
    std::string k;
    snprintf(buf, sizeof(buf), "%p/%llu/%llu/%d/%d/%d/%llu/%llu|", (const void*)d.dim, (unsigned long long)d.dim->serial,
             (unsigned long long)d.dim->rows, d.join.dim_col, x.direct ? 1 : 0, x.key64 ? 1 : 0,
             (unsigned long long)x.join_cap, (unsigned long long)x.range);
    k += buf;
    for (int g = 0; g < d.n_group; ++g) {
        if (d.group[g].side != TP_SIDE_DIM) continue;
        snprintf(buf, sizeof(buf), "g%d:%d:%d|", d.group[g].col, d.group[g].bits, p->gdpos[g]);
        k += buf;
    }
    if (d.dim_filter.col >= 0) {
        snprintf(buf, sizeof(buf), "f%d:%lld:%lld", d.dim_filter.col, (long long)d.dim_filter.lo,
                 (long long)d.dim_filter.hi);
        k += buf;
    }
    return k;
}

// Frees idle cached join tables (least recently used first) until `need`
// bytes are released (0: every idle one); caller holds sv->mu.  Idle tables
// are read by no batch in flight, so freeing on stream st is safe.
uint64_t evict_joins(tp_server* sv, uint64_t need, cudaStream_t st) {
    uint64_t freed = 0;
    while (need == 0 || freed < need) {
        auto victim = sv->joins.end();
        for (auto it = sv->joins.begin(); it != sv->joins.end(); ++it)
            if (it->second.users == 0 && (victim == sv->joins.end() || it->second.last_use < victim->second.last_use))
                victim = it;
        if (victim == sv->joins.end()) break;
        JEntry& j = victim->second;
        dev_free(sv->e, j.mem, st);
        if (j.built) cudaEventDestroy(j.built);
        release(sv->e, j.bytes);
        freed += j.bytes;
        sv->joins.erase(victim);
    }
    return freed;
}

// The cached join table of request i's plan, built now on sl's stream if
// missing (sl.built records it); a table another slot built is waited for on
// this stream.  Marks the table used by this batch.
tp_status join_entry(tp_server* sv, Slot& sl, tp_plan* p, const BatchPrep& x, JEntry** out) {
    tp_engine* e = sv->e;
    const std::string key = join_key(p, x);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->joins.find(key);
        if (it != sv->joins.end()) {
            JEntry& j = it->second;
            ++j.users;
            j.last_use = ++sv->join_tick;
            *out = &j;
        }
    }
    if (*out) {
        TP_TRY_CUDA(cudaStreamWaitEvent(sl.st, (*out)->built, 0));
        return TP_OK;
    }
    JEntry j;
    j.slot_bytes = a256(x.join_bytes);
    j.bytes = j.slot_bytes + 256;
    tp_status s = reserve(e, j.bytes);
    if (s == TP_E_BUDGET) {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (evict_joins(sv, j.bytes, sl.st) > 0) s = reserve(e, j.bytes);
    }
    if (s) return s;
    if ((s = dev_alloc(e, &j.mem, j.bytes, sl.st))) {
        release(e, j.bytes);
        return s;
    }
    j.side = (uint32_t*)((unsigned char*)j.mem + j.slot_bytes);
    j.err = j.side + 4;
    cudaError_t ce = cudaMemsetAsync(j.mem, 0xFF, j.slot_bytes, sl.st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(j.side, 0, 256, sl.st);
    tpk::BatchQuery B;
    tpk::OutDev od{};
    batch_query_desc(p, x, j.mem, j.side, nullptr, j.err, od, &B);
    if (ce == cudaSuccess && p->d.dim->rows) ce = tpk::launch_build(B.b, p->d.dim->rows, e->num_sms, sl.st);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&j.built, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventRecord(j.built, sl.st);
    if (ce != cudaSuccess) {
        if (j.built) cudaEventDestroy(j.built);
        dev_free(e, j.mem, sl.st);
        release(e, j.bytes);
        return fail(TP_E_CUDA, "join build for a batched request: %s", cudaGetErrorString(ce));
    }
    e->launches++;
    std::lock_guard<std::mutex> lk(sv->mu);
    j.users = 1;
    j.last_use = ++sv->join_tick;
    JEntry& stored = sv->joins.emplace(key, j).first->second;
    sl.built.emplace_back(&stored, 0);
    *out = &stored;
    return TP_OK;
}

// Device bytes of a batch of the plans of rs: join tables, counters, error
// words, group counts, side cells, accumulators, descriptors, tasks, wait word.
struct BatchSizes {
    uint64_t zero = 0, qbytes = 0, ibytes = 0, total = 0, results = 0, joins = 0, items = 0;
    uint32_t smem = 16;
};

BatchSizes batch_sizes(tp_server* sv, const std::vector<Request*>& rs) {
    BatchSizes z;
    const uint64_t n = rs.size();
    // counters, batch error, groups, sides, query errors, finalisation words
    z.zero = a256((1 + 2 * n) * 4) + 256 + a256(8 * n) * 5;
    std::map<std::string, bool> missing;   // join tables the batch would build
    for (Request* r : rs) {
        const PlanInfo& pi = plan_info(sv, r->plan);
        if (pi.x.join) {
            const std::string key = join_key(r->plan, pi.x);
            std::lock_guard<std::mutex> lk(sv->mu);
            if (!sv->joins.count(key) && !missing.count(key)) {
                missing[key] = true;
                z.joins += a256(pi.x.join_bytes) + 256;
            }
        }
        z.zero += pi.x.acc_bytes;
        z.items += pi.x.probe_items + pi.x.final_items;   // join tables come from the cache, built by their own launch
        z.results += pi.result_bytes;
        if (pi.x.smem) z.smem = std::max(z.smem, pi.x.smem_bytes);
    }
    z.qbytes = a256(sizeof(tpk::BatchQuery) * n);
    z.ibytes = a256(sizeof(tpk::BatchItem) * z.items);
    z.total = z.zero + z.qbytes + z.ibytes + 256;
    return z;
}

tp_status grow_stage(Slot& sl, uint64_t bytes) {
    if (bytes <= sl.h_cap) return TP_OK;
    if (sl.h_stage) cudaFreeHost(sl.h_stage);
    sl.h_stage = nullptr;
    sl.h_cap = 0;
    const uint64_t cap = std::max<uint64_t>(bytes + bytes / 2, 1 << 20);
    TP_TRY_CUDA(cudaHostAlloc((void**)&sl.h_stage, cap, cudaHostAllocDefault));
    sl.h_cap = cap;
    return TP_OK;
}

// Lays out, copies and launches the batch of sl.reqs on sl's stream; the
// device reservation of z.total is already held (sl.reserved).
tp_status launch_slot(tp_server* sv, Slot& sl, const BatchSizes& z) {
    tp_engine* e = sv->e;
    const uint64_t n = sl.reqs.size();
    tp_status s = dev_alloc(e, &sl.arena, z.total, sl.st);
    if (s) return s;
    unsigned char* base = (unsigned char*)sl.arena;
    unsigned char* zp = base;
    unsigned* d_ctr = (unsigned*)zp;
    zp += a256((1 + 2 * n) * 4);
    uint32_t* d_err = (uint32_t*)zp;
    zp += 256;
    unsigned long long* d_groups = (unsigned long long*)zp;
    zp += a256(8 * n);
    uint32_t* sides = (uint32_t*)zp;
    zp += a256(8 * n);
    uint32_t* q_err = (uint32_t*)zp;   // one error word per query: one query's failure stays its own
    zp += a256(8 * n);
    unsigned* final_done = (unsigned*)zp;
    zp += a256(8 * n);
    unsigned long long* final_end = (unsigned long long*)zp;
    zp += a256(8 * n);
    unsigned char* accp = zp;
    unsigned char* dq = base + z.zero;
    // host side: descriptors, then tasks, then the wait limit, in the pinned stage
    const uint64_t status_bytes = 16 * n + 8 + 8 * n;
    if ((s = grow_stage(sl, z.qbytes + z.ibytes + 256 + a256(status_bytes)))) return s;
    tpk::BatchQuery* hq = (tpk::BatchQuery*)sl.h_stage;
    tpk::BatchItem* hi = (tpk::BatchItem*)(sl.h_stage + z.qbytes);
    (void)sides;
    std::vector<tpk::BatchItem> items;
    items.reserve(z.items);
    sl.res.assign(n, nullptr);
    sl.joins.assign(n, nullptr);
    uint32_t smem = 16;
    for (uint64_t i = 0; i < n; ++i) {
        tp_plan* p = sl.reqs[i]->plan;
        const PlanInfo& pi = plan_info(sv, p);
        if (pi.x.join && (s = join_entry(sv, sl, p, pi.x, &sl.joins[i]))) return s;
        tpk::OutDev od;
        if ((s = alloc_result(e, p, 1ull << p->key_bits, &sl.res[i], &od, d_groups + i, sl.st))) return s;
        JEntry* j = sl.joins[i];
        batch_query_desc(p, pi.x, j ? j->mem : nullptr, j ? j->side : nullptr, (uint64_t*)accp, q_err + 2 * i, od,
                         &hq[i], final_done + 2 * i, final_end + i);
        hq[i].shape = pi.shape;
        hq[i].build_items = 0;   // the table is built (or being built) by its own launch
        accp += pi.x.acc_bytes;
        if (pi.x.smem) smem = std::max(smem, pi.x.smem_bytes);
    }
    for (uint64_t i = 0; i < n; ++i) batch_items(sl.reqs[i]->plan, plan_info(sv, sl.reqs[i]->plan).x, (uint32_t)i,
                                                 tpk::BI_PROBE, &items);
    for (uint64_t i = 0; i < n; ++i) batch_items(sl.reqs[i]->plan, plan_info(sv, sl.reqs[i]->plan).x, (uint32_t)i,
                                                 tpk::BI_FINAL, &items);
    memcpy(hi, items.data(), items.size() * sizeof(tpk::BatchItem));
    memcpy(sl.h_stage + z.qbytes + z.ibytes, &SERVE_WAIT_NS, 8);
    const uint64_t* d_wait = (const uint64_t*)(dq + z.qbytes + z.ibytes);
    TP_TRY_CUDA(cudaMemcpyAsync(dq, sl.h_stage, z.qbytes + z.ibytes + 8, cudaMemcpyHostToDevice, sl.st));
    TP_TRY_CUDA(cudaMemsetAsync(base, 0, z.zero, sl.st));
    if (sv->kernel_stale) {   // one kernel for every shape registered so far
        std::string why;
        sv->kernel = jit_kernel(e, batch_kernel_source(sv->shapes), "tpj_batch", &why);
        sv->kernel_stale = false;
    }
    const void* k = sv->kernel;
    auto g = sv->grids.find({k, smem});
    if (g == sv->grids.end()) g = sv->grids.emplace(std::make_pair(k, smem), batch_kernel_grid(k, smem, e->num_sms)).first;
    // no more resident CTAs than tasks: a small batch retires its grid sooner
    const int grid = (int)std::min<uint64_t>((uint64_t)g->second, items.size());
    const tpk::BatchQuery* a_q = (const tpk::BatchQuery*)dq;
    const tpk::BatchItem* a_items = (const tpk::BatchItem*)(dq + z.qbytes);
    uint32_t a_n = (uint32_t)items.size(), a_nq = (uint32_t)n;
    if (k) {
        void* args[] = {&a_q, &a_items, &a_n, &a_nq, &d_ctr, &d_err, &d_wait};
        TP_TRY_CUDA(cudaLaunchKernel(k, dim3(grid), dim3(tpk::BATCH_THREADS), args, smem, sl.st));
        e->jit_launches++;
    } else {
        TP_TRY_CUDA(tpk::launch_batch(a_q, a_items, a_n, a_nq, d_ctr, d_err, d_wait, smem, grid, sl.st));
    }
    e->launches++;
    // status words back: group counts, per-query error words, the batch error word
    sl.status_off = z.qbytes + z.ibytes + 256;
    unsigned char* hs = sl.h_stage + sl.status_off;
    TP_TRY_CUDA(cudaMemcpyAsync(hs, d_groups, 8 * n, cudaMemcpyDeviceToHost, sl.st));
    TP_TRY_CUDA(cudaMemcpyAsync(hs + 8 * n, q_err, 8 * n, cudaMemcpyDeviceToHost, sl.st));
    TP_TRY_CUDA(cudaMemcpyAsync(hs + 16 * n, d_err, 4, cudaMemcpyDeviceToHost, sl.st));
    for (size_t k2 = 0; k2 < sl.built.size(); ++k2) {   // error words of the tables this batch built
        sl.built[k2].second = sl.status_off + 16 * n + 8 + 8 * k2;
        TP_TRY_CUDA(cudaMemcpyAsync(sl.h_stage + sl.built[k2].second, sl.built[k2].first->err, 4,
                                    cudaMemcpyDeviceToHost, sl.st));
    }
    TP_TRY_CUDA(cudaEventRecord(sl.ev, sl.st));
    e->d2h_bytes += 16 * n + 4;
    ++sv->stats.batches;
    return TP_OK;
}

tp_status map_err_word(uint32_t err) {
    if (err & tpk::ERR_TIMEOUT) return fail(TP_E_TIMEOUT, "a bounded wait of the batched launch expired");
    if (err & tpk::ERR_DUP) return fail(TP_E_DUP_KEY, "the join build side holds a duplicate key");
    if (err & tpk::ERR_RANGE) return fail(TP_E_RANGE, "a group field value does not fit its bit width");
    if (err & tpk::ERR_INTERNAL) return fail(TP_E_INTERNAL, "device consistency check failed");
    return TP_OK;
}

// The batch of sl no longer reads its join tables (caller holds sv->mu); a
// table whose build failed is dropped once nothing reads it, so a later
// request builds it again and meets the same error itself.
void unuse_joins(tp_server* sv, Slot& sl) {
    for (JEntry* j : sl.joins)
        if (j) --j->users;
    for (auto it = sv->joins.begin(); it != sv->joins.end();) {
        JEntry& j = it->second;
        if (j.bad && j.users == 0) {
            dev_free(sv->e, j.mem, sl.st);
            if (j.built) cudaEventDestroy(j.built);
            release(sv->e, j.bytes);
            it = sv->joins.erase(it);
        } else {
            ++it;
        }
    }
    sl.joins.clear();
    sl.built.clear();
}

// Frees what a slot's batch holds (after its stream is done with it).
void slot_release(tp_server* sv, Slot& sl) {
    if (sl.arena) dev_free(sv->e, sl.arena, sl.st);
    sl.arena = nullptr;
    if (sl.reserved) release(sv->e, sl.reserved);
    sl.reserved = 0;
}

void dispatcher(tp_server* sv) {
    tp_engine* e = sv->e;
    cudaSetDevice(e->device);
    for (;;) {
        std::vector<Request*> take;
        int si = -1;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            bool work = false;
            sv->cv_disp.wait(lk, [&] {
                work = false;
                for (Request* q : sv->queue) work = work || q->batchable;
                si = -1;
                for (int k = 0; k < N_SLOTS; ++k)
                    if (!sv->slots[k].busy) si = k;
                return (sv->stopping && !work) || (work && si >= 0);
            });
            if (!work) break;   // stopping, nothing batchable left
            for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)take.size() < sv->max_batch;) {
                if ((*it)->batchable) {
                    take.push_back(*it);
                    it = sv->queue.erase(it);
                } else {
                    ++it;
                }
            }
            // a lone request on an idle GPU runs at once as a single query
            // (its fused kernel), without waiting for a batch to form
            if (take.size() == 1 && sv->launched.empty() && sv->inflight == 0) {
                Request* r = take[0];
                if (!r->t_start) r->t_start = now_ns();
                ++sv->inflight;
                const uint64_t c0 = sv->completions;
                lk.unlock();
                plan_info(sv, r->plan);   // its shape joins the batched kernel's next compilation
                tp_result* res = nullptr;
                DimCache* cache = sv->cache_on ? &sv->cache : nullptr;
                tp_status st1 = execute_on_lane(r->plan, &sv->dlane, cache, &res);
                if (st1 == TP_E_BUDGET && cache && cache_evict_idle(e, cache, 0) > 0)
                    st1 = execute_on_lane(r->plan, &sv->dlane, cache, &res);
                if (res) res->stream = nullptr;
                const std::string msg = st1 ? tp_last_error() : "";
                lk.lock();
                --sv->inflight;
                if (st1 == TP_E_BUDGET && (sv->inflight > 0 || sv->completions != c0)) {
                    sv->queue.push_front(r);   // memory is or was held by others: retry
                    ++sv->stats.budget_waits;
                } else {
                    finish(sv, r, st1, msg, res);
                }
                sv->cv_lane.notify_all();
                continue;
            }
            sv->slots[si].busy = true;
        }
        // admission by the device budget: the longest prefix (in arrival order)
        // whose batch and result arrays fit beside what else is reserved
        Slot& sl = sv->slots[si];
        size_t n = take.size();
        BatchSizes z;
        tp_status st = TP_E_BUDGET;
        while (n > 0) {
            std::vector<Request*> part(take.begin(), take.begin() + n);
            z = batch_sizes(sv, part);
            if (reserve(e, z.total + z.results + z.joins) == TP_OK) {
                release(e, z.results + z.joins);   // result arrays and new join tables reserve their own below
                st = TP_OK;
                break;
            }
            bool evicted;
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                evicted = evict_joins(sv, z.total + z.results + z.joins, sl.st) > 0;
            }
            if (!evicted) n /= 2;
        }
        std::unique_lock<std::mutex> lk(sv->mu);
        if (st != TP_OK) {
            // nothing fits now: wait for a running batch or lane, else fail the oldest
            const bool others = sv->inflight > 0 || !sv->launched.empty();
            for (auto it = take.rbegin(); it != take.rend(); ++it) sv->queue.push_front(*it);
            sl.busy = false;
            if (others) {
                ++sv->stats.budget_waits;
                const uint64_t c0 = sv->completions;
                sv->cv_done.wait_for(lk, std::chrono::milliseconds(200), [&] { return sv->completions != c0; });
            } else {
                Request* r = sv->queue.front();
                sv->queue.pop_front();
                if (!r->t_start) r->t_start = now_ns();
                finish(sv, r, TP_E_BUDGET, tp_last_error(), nullptr);
            }
            sv->cv_lane.notify_all();
            continue;
        }
        for (size_t i = n; i < take.size(); ++i) sv->queue.insert(sv->queue.begin() + (long)(i - n), take[i]);
        take.resize(n);
        const int64_t t0 = now_ns();
        for (Request* r : take)
            if (!r->t_start) r->t_start = t0;
        sl.reqs = take;
        sl.reserved = z.total;
        const uint32_t peak = (uint32_t)(sv->inflight + (int)n);
        if (peak > sv->stats.inflight_peak) sv->stats.inflight_peak = peak;
        lk.unlock();
        st = launch_slot(sv, sl, z);
        lk.lock();
        if (st != TP_OK) {
            const std::string msg = tp_last_error();
            cudaStreamSynchronize(sl.st);
            for (size_t i = 0; i < sl.res.size(); ++i)
                if (sl.res[i]) tp_result_free(sl.res[i]);
            slot_release(sv, sl);
            unuse_joins(sv, sl);
            const bool others = sv->inflight > 0 || !sv->launched.empty();
            if (st == TP_E_BUDGET && (others || sl.reqs.size() > 1)) {
                // memory went to others meanwhile: back to the queue, in order
                for (auto it = sl.reqs.rbegin(); it != sl.reqs.rend(); ++it) sv->queue.push_front(*it);
                ++sv->stats.budget_waits;
                if (others) {
                    const uint64_t c0 = sv->completions;
                    sv->cv_done.wait_for(lk, std::chrono::milliseconds(200), [&] { return sv->completions != c0; });
                }
            } else {
                for (Request* r : sl.reqs) finish(sv, r, st, msg, nullptr);
            }
            sl.reqs.clear();
            sl.res.clear();
            sl.busy = false;
            sv->cv_lane.notify_all();
            continue;
        }
        sv->launched.push_back(si);
        sv->cv_comp.notify_one();
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->dispatcher_done = true;
    sv->cv_comp.notify_all();
}

void completer(tp_server* sv) {
    cudaSetDevice(sv->e->device);
    for (;;) {
        int si;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_comp.wait(lk, [&] { return !sv->launched.empty() || sv->dispatcher_done; });
            if (sv->launched.empty()) return;
            si = sv->launched.front();
        }
        Slot& sl = sv->slots[si];
        const cudaError_t ce = cudaEventSynchronize(sl.ev);
        const size_t n = sl.reqs.size();
        const unsigned char* hs = sl.h_stage + sl.status_off;
        const uint32_t batch_err = ce == cudaSuccess ? *(const uint32_t*)(hs + 16 * n) : 0;
        {
            // the tables this batch built: their builds' errors (a duplicate
            // key, a field out of range) stay with every request that reads them
            std::lock_guard<std::mutex> lk(sv->mu);
            for (auto& b : sl.built) {
                b.first->checked = true;
                if (ce == cudaSuccess) {
                    const uint32_t w = *(const uint32_t*)(sl.h_stage + b.second);
                    if (w & tpk::ERR_DUP) b.first->bad = TP_E_DUP_KEY;
                    else if (w & tpk::ERR_INTERNAL) b.first->bad = TP_E_INTERNAL;
                }
            }
        }
        std::vector<tp_status> sts(n, TP_OK);
        std::vector<std::string> msgs(n);
        for (size_t i = 0; i < n; ++i) {
            tp_result* r = sl.res[i];
            if (ce != cudaSuccess) {
                sts[i] = fail(TP_E_CUDA, "batched launch: %s", cudaGetErrorString(ce));
            } else {
                const uint32_t err = batch_err | *(const uint32_t*)(hs + 8 * n + 8 * i);
                sts[i] = map_err_word(err);
                const JEntry* j = sl.joins[i];
                if (sts[i] == TP_OK && j && j->bad)
                    sts[i] = j->bad == TP_E_DUP_KEY ? fail(TP_E_DUP_KEY, "the join build side holds a duplicate key")
                                                    : fail(TP_E_INTERNAL, "device consistency check failed");
            }
            if (sts[i]) {
                msgs[i] = tp_last_error();
                tp_result_free(r);
                sl.res[i] = nullptr;
            } else {
                r->n_groups = ((const uint64_t*)hs)[i];
                r->stream = nullptr;   // its memory may be freed on the engine's stream
            }
        }
        slot_release(sv, sl);
        std::lock_guard<std::mutex> lk(sv->mu);
        for (size_t i = 0; i < n; ++i) finish(sv, sl.reqs[i], sts[i], msgs[i], sl.res[i]);
        unuse_joins(sv, sl);
        sl.reqs.clear();
        sl.res.clear();
        sl.busy = false;
        sv->launched.pop_front();
        sv->cv_disp.notify_one();
        sv->cv_lane.notify_all();
    }
}

void server_free(tp_server* sv) {
    if (!sv) return;
    cudaSetDevice(sv->e->device);
    sv->lanes.push_back(sv->dlane);   // freed with the others below
    for (Lane& l : sv->lanes) {
        if (l.compute) cudaStreamSynchronize(l.compute);
        if (l.copy) cudaStreamSynchronize(l.copy);
        if (l.spill) cudaStreamSynchronize(l.spill);
    }
    for (Slot& sl : sv->slots)
        if (sl.st) cudaStreamSynchronize(sl.st);
    for (auto& kv : sv->reqs)   // finished but never collected
        if (kv.second->result) tp_result_free(kv.second->result);
    cache_evict_idle(sv->e, &sv->cache, 0);
    evict_joins(sv, 0, sv->e->compute);
    for (Lane& l : sv->lanes) {
        if (l.compute) cudaStreamDestroy(l.compute);
        if (l.copy) cudaStreamDestroy(l.copy);
        if (l.spill) cudaStreamDestroy(l.spill);
        if (l.host_words) cudaFreeHost(l.host_words);
    }
    for (Slot& sl : sv->slots) {
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.h_stage) cudaFreeHost(sl.h_stage);
    }
    delete sv;
}

}  // namespace

extern "C" {

tp_status tp_server_start(tp_engine* e, int32_t workers, int32_t max_inflight, uint32_t flags, tp_server** out) {
    clear_error();
    if (!e || !out || workers < 1 || workers > 64 || max_inflight < 0)
        return fail(TP_E_INVALID, "tp_server_start: bad arguments");
    *out = nullptr;
    std::unique_ptr<tp_server, void (*)(tp_server*)> sv(new (std::nothrow) tp_server(), server_free);
    if (!sv) return fail(TP_E_NOMEM, "tp_server_start: out of host memory");
    sv->e = e;
    sv->max_inflight = max_inflight ? max_inflight : workers;
    sv->cache_on = (flags & TP_SERVE_CACHE_DIM) != 0;
    sv->batch_on = (flags & TP_SERVE_BATCH) != 0;
    if (sv->batch_on && max_inflight) sv->max_batch = max_inflight;
    TP_TRY_CUDA(cudaSetDevice(e->device));
    sv->lanes.resize(workers);
    for (Lane& l : sv->lanes) {
        TP_TRY_CUDA(cudaStreamCreateWithFlags(&l.compute, cudaStreamNonBlocking));
        TP_TRY_CUDA(cudaStreamCreateWithFlags(&l.copy, cudaStreamNonBlocking));
        TP_TRY_CUDA(cudaStreamCreateWithFlags(&l.spill, cudaStreamNonBlocking));
        TP_TRY_CUDA(cudaHostAlloc((void**)&l.host_words, 4096, cudaHostAllocDefault));
    }
    if (sv->batch_on) {
        TP_TRY_CUDA(cudaStreamCreateWithFlags(&sv->dlane.compute, cudaStreamNonBlocking));
        TP_TRY_CUDA(cudaStreamCreateWithFlags(&sv->dlane.copy, cudaStreamNonBlocking));
        TP_TRY_CUDA(cudaStreamCreateWithFlags(&sv->dlane.spill, cudaStreamNonBlocking));
        TP_TRY_CUDA(cudaHostAlloc((void**)&sv->dlane.host_words, 4096, cudaHostAllocDefault));
        for (Slot& sl : sv->slots) {
            TP_TRY_CUDA(cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking));
            TP_TRY_CUDA(cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming));
        }
        sv->dispatcher = std::thread(dispatcher, sv.get());
        sv->completer = std::thread(completer, sv.get());
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
    r->batchable = sv->batch_on && batch_check_plan(sv->e, p, 0) == TP_OK && p->d.fact->rows <= SERVE_BATCH_MAX_ROWS;
    clear_error();
    r->t_submit = now_ns();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stopping) return fail(TP_E_INVALID, "tp_submit: server is stopping");
    r->ticket = sv->next_ticket++;
    *out = r->ticket;
    const bool r_batchable = r->batchable;
    sv->queue.push_back(r.get());
    sv->reqs[r->ticket] = std::move(r);
    ++sv->stats.submitted;
    if (r_batchable) sv->cv_disp.notify_one();
    else sv->cv_lane.notify_one();
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
    if (r->waited) return fail(TP_E_INVALID, "tp_wait: ticket %llu is being waited on by another thread",
                               (unsigned long long)t);
    r->waited = true;
    auto ready = [&] { return r->done; };
    if (timeout_ns < 0) {
        sv->cv_done.wait(lk, ready);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), ready)) {
        r->waited = false;
        return fail(TP_E_TIMEOUT, "tp_wait: ticket %llu not finished", (unsigned long long)t);
    }
    if (times) {
        times[0] = r->t_submit;
        times[1] = r->t_start;
        times[2] = r->t_end;
    }
    const tp_status st = r->status;
    if (st == TP_OK) *out = r->result;
    else fail(st, "%s", r->message.c_str());
    sv->reqs.erase(sv->reqs.find(t));
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
    sv->cv_lane.notify_all();
    sv->cv_disp.notify_all();
    sv->cv_comp.notify_all();
    sv->cv_done.notify_all();
    for (auto& th : sv->threads) th.join();
    if (sv->dispatcher.joinable()) sv->dispatcher.join();
    if (sv->completer.joinable()) sv->completer.join();
    server_free(sv);
}

}  // extern "C"
