// Plans, execution and results behind the C ABI.
//
// One execution (Section 3.3.1: a compute task reserves memory, loads its
// input batches into GPU memory, then computes):
//   reserve -> build the join table -> per fact batch: [copy stream: H2D of
//   the batch's pages into a free staging slot] -> [compute stream: fused
//   filter/probe/aggregate] -> finalise -> release.
// Batches of a paged fact table are copied ahead of the kernel that consumes
// them (Section 3.3.3, compute-task pre-loading); with prefetch_depth 0 the
// compute stream copies each batch itself.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <string>

#include "tp_internal.h"

using namespace tp;

namespace {


uint64_t pow2_at_least(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

bool valid_col(const tp_table* t, int32_t c) { return t && c >= 0 && c < (int32_t)t->types.size(); }

// Value of one column at one row of a paged table (host read of the pages).
int64_t paged_value(const tp_table* t, int c, uint64_t row) {
    auto it = std::upper_bound(t->batches.begin(), t->batches.end(), row,
                               [](uint64_t r, const Batch& b) { return r < b.row0; });
    const Batch& b = *(it - 1);
    if (b.packed(c)) {   // the bytes holding the value's bits, gathered across extents
        const int bits = b.enc_bits[c];
        const uint64_t at = (row - b.row0) * (uint64_t)bits;
        uint64_t d = 0;
        for (uint64_t byte = at / 8, k = 0; byte <= (at + bits - 1) / 8; ++byte, ++k) {
            uint64_t off = byte;
            for (const Extent& x : b.cols[c]) {
                if (off < x.bytes) {
                    d |= (uint64_t)((const uint8_t*)tp_page_ptr(t->eng, x.page))[x.offset + off] << (8 * k);
                    break;
                }
                off -= x.bytes;
            }
        }
        d = (d >> (at % 8)) & ((1ull << bits) - 1);
        return (int64_t)((uint64_t)b.enc_base[c] + d);
    }
    const int sz = b.width(c, t->types[c]);
    uint64_t off = (row - b.row0) * sz;
    for (const Extent& x : b.cols[c]) {
        if (off < x.bytes) {   // column starts are 256-byte aligned and pages whole 4 KiB multiples: no value straddles two extents
            const uint8_t* p = (const uint8_t*)tp_page_ptr(t->eng, x.page) + x.offset + off;
            if (b.narrow(c)) {
                uint64_t d = 0;
                for (int k = 0; k < sz; ++k) d |= (uint64_t)p[k] << (8 * k);
                return (int64_t)((uint64_t)b.enc_base[c] + d);
            }
            switch (t->types[c]) {
            case TP_I32: { int32_t v; memcpy(&v, p, 4); return v; }
            case TP_I64: { int64_t v; memcpy(&v, p, 8); return v; }
            default: return *p;
            }
        }
        off -= x.bytes;
    }
    return 0;
}

// Device memory of one execution, released together at the end.
struct Scratch {
    tp_engine* e;
    cudaStream_t st;
    std::vector<void*> ptrs;
    uint64_t reserved = 0;
    explicit Scratch(tp_engine* eng, cudaStream_t s) : e(eng), st(s) {}
    tp_status alloc(void** p, uint64_t bytes) {
        tp_status s = dev_alloc(e, p, bytes, st);
        if (s == TP_OK) ptrs.push_back(*p);
        return s;
    }
    void free_all() {
        for (void* p : ptrs) dev_free(e, p, st);
        ptrs.clear();
        if (reserved) release(e, reserved);
        reserved = 0;
    }
    ~Scratch() { free_all(); }
};

struct ExecState {
    tp_plan* p;
    tp_engine* e;
    tp_table* fact;
    tp_table* dim;
    std::vector<int> used;          // fact columns the query reads
    bool key64 = false;
    uint64_t join_cap = 0;
    tpk::JoinTable jt{};
    tpk::JoinTable jtx[tpk::MAX_XJOIN] = {};   // further tables of a star join
    uint32_t* err = nullptr;        // device error word
    unsigned long long* counters = nullptr;   // [0] agg used, [1] compact count, [2] max key, [3] sample
    bool eager = true;
    Lane* lane = nullptr;           // streams and status words of this execution
};

void mark_launch(tp_engine* e) { e->launches++; }

// Host wall time of one phase of a partitioned join, added to the engine's
// statistics (phase < 0: not timed).
struct PhaseTimer {
    tp_engine* e;
    int phase;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    PhaseTimer(tp_engine* eng, int ph) : e(eng), phase(ph) {}
    ~PhaseTimer() {
        if (phase < 0) return;
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        std::lock_guard<std::mutex> lk(e->time_mu);
        e->part_ms[phase] += ms;
    }
};

// Brackets fused-kernel launches with events on the compute stream when the
// engine was created with TP_FLAG_TIME_KERNELS; totals are folded into the
// engine statistics once the execution has synchronised.
struct KernelTimer {
    tp_engine* e;
    bool on;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    uint64_t rows = 0;
    explicit KernelTimer(tp_engine* eng) : e(eng), on((eng->cfg.flags & TP_FLAG_TIME_KERNELS) != 0) {}
    template <class F>
    cudaError_t run(cudaStream_t st, uint64_t n, F&& launch) {
        if (!on) return launch();
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
        cudaError_t r = launch();
        cudaEventRecord(b, st);
        ev.emplace_back(a, b);
        rows += n;
        return r;
    }
    void collect() {  // after a stream synchronisation
        if (!on) return;
        double ms = 0;
        for (auto& p : ev) {
            float t = 0;
            if (cudaEventElapsedTime(&t, p.first, p.second) == cudaSuccess) ms += t;
            cudaEventDestroy(p.first);
            cudaEventDestroy(p.second);
        }
        std::lock_guard<std::mutex> lk(e->time_mu);
        e->agg_ms += ms;
        e->agg_launches += ev.size();
        e->agg_rows += rows;
        ev.clear();
        rows = 0;
    }
    ~KernelTimer() {
        for (auto& p : ev) {
            cudaEventDestroy(p.first);
            cudaEventDestroy(p.second);
        }
    }
};

tpk::DevCol devcol(const tp_table* t, int c, const void* ptr) {
    tpk::DevCol d{};
    d.ptr = ptr;
    d.type = t->types[c];
    return d;
}

// QueryDev for one batch: colptr[c] is the device address of fact column c's
// first row in this batch (nullptr for columns the query does not read).
tpk::QueryDev make_query(const ExecState& S, const std::vector<const void*>& colptr) {
    return tp::plan_query_dev(S.p, colptr, S.jt, S.err, S.eager, S.jtx);
}

tp_status cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return TP_OK;
    cudaGetLastError();
    return fail(TP_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ----------------------------------------------------------------- build

// Build-side parameters of dimension k (0: the first join) without columns:
// its group fields packed into the payload, its predicate's bounds.
tpk::BuildDev build_proto(const ExecState& S, int k = 0) {
    const tp_plan_desc& d = S.p->d;
    tpk::BuildDev b{};
    b.jt = k == 0 ? S.jt : S.jtx[k - 1];
    b.err = S.err;
    int nf = 0;
    for (int g = 0; g < d.n_group; ++g) {
        if (S.p->gdim[g] != k) continue;
        b.dbits[nf] = d.group[g].bits;
        b.dpos[nf] = S.p->gdpos[g];
        ++nf;
    }
    b.n_dfield = nf;
    b.has_filter = S.p->dflt[k].col >= 0;
    b.flo = S.p->dflt[k].lo;
    b.fhi = S.p->dflt[k].hi;
    return b;
}

// Calls fn(build, rows) for every batch of dimension k with the key,
// group-field and predicate columns on the device.
template <class F>
tp_status for_each_dim_batch(ExecState& S, Scratch& sc, const tpk::BuildDev& proto, F&& fn, int dk = 0) {
    tp_engine* e = S.e;
    const tp_plan_desc& d = S.p->d;
    tp_table* t = S.p->dims[dk];
    const tp_filter& flt = S.p->dflt[dk];
    std::vector<int> bcols = {S.p->joins[dk].dim_col};
    for (int g = 0; g < d.n_group; ++g)
        if (S.p->gdim[g] == dk) bcols.push_back(d.group[g].col);
    const int nf = (int)bcols.size() - 1;
    if (flt.col >= 0) bcols.push_back(flt.col);
    tpk::BuildDev b = proto;
    auto bind = [&](const std::vector<const void*>& ptr) {
        b.key = devcol(t, bcols[0], ptr[0]);
        for (int k = 1; k <= nf; ++k) b.dcol[k - 1] = devcol(t, bcols[k], ptr[k]);
        if (flt.col >= 0) b.fcol = devcol(t, bcols[nf + 1], ptr[nf + 1]);
    };
    if (t->placement != PL_PAGES) {
        std::vector<const void*> ptr;
        for (int c : bcols) ptr.push_back(t->dev_cols[c]);
        bind(ptr);
        return fn(b, t->rows);
    }
    uint64_t max_rows = 0;
    for (auto& bt : t->batches) max_rows = std::max(max_rows, bt.rows);
    std::vector<void*> stage(bcols.size(), nullptr), enc(bcols.size(), nullptr);
    const bool narrow = has_narrow(t);
    for (size_t i = 0; i < bcols.size(); ++i) {
        tp_status s = sc.alloc(&stage[i], align256(max_rows * type_size(t->types[bcols[i]])));
        const int w = narrow ? narrow_width_max(t, bcols[i]) : 0;
        if (!s && w) s = sc.alloc(&enc[i], align256(max_rows * (uint64_t)w + 16));   // + the decoder's word overrun
        if (s) return s;
    }
    for (auto& bt : t->batches) {
        for (size_t i = 0; i < bcols.size(); ++i) {
            tp_status s = copy_batch_column(e, t, bt, bcols[i], stage[i], enc[i], 0, S.lane->compute);
            if (s) return s;
        }
        if (narrow) {
            tp_status s = widen_batch(e, t, bt, bcols, stage, enc, 0, S.lane->compute);
            if (s) return s;
        }
        bind(std::vector<const void*>(stage.begin(), stage.end()));
        tp_status s = fn(b, bt.rows);
        if (s) return s;
    }
    return TP_OK;
}

// Builds the join table of dimension k (S.jt, or S.jtx[k - 1]).
tp_status build_join(ExecState& S, Scratch& sc, int k = 0) {
    tp_engine* e = S.e;
    cudaStream_t st = S.lane->compute;
    return for_each_dim_batch(S, sc, build_proto(S, k), [&](const tpk::BuildDev& b, uint64_t rows) {
        mark_launch(e);
        return cuda_check(tpk::launch_build(b, rows, e->num_sms, st), "build");
    }, k);
}

// Fan-out build of the first join: the admitted rows' (key, payload) pairs
// sorted by key; the table maps each key to the index of its run's first row.
tp_status build_join_many(ExecState& S, Scratch& sc) {
    tp_engine* e = S.e;
    cudaStream_t st = S.lane->compute;
    const uint64_t n_rows = S.dim->rows;
    void *k0 = nullptr, *v0 = nullptr, *k1 = nullptr, *v1 = nullptr, *hist = nullptr, *hk = nullptr, *hv = nullptr,
         *ctr = nullptr;
    const uint64_t c = n_rows ? n_rows : 1;
    tp_status s;
    if ((s = sc.alloc(&k0, c * 8)) || (s = sc.alloc(&v0, c * 4)) || (s = sc.alloc(&k1, c * 8)) ||
        (s = sc.alloc(&v1, c * 4)) || (s = sc.alloc(&hist, tpk::radix_sort_hist_words(c) * 4)) ||
        (s = sc.alloc(&hk, c * 8)) || (s = sc.alloc(&hv, c * 4)) || (s = sc.alloc(&ctr, 16)))
        return s;
    TP_TRY_CUDA(cudaMemsetAsync(ctr, 0, 16, st));
    unsigned long long* cnt = (unsigned long long*)ctr;
    s = for_each_dim_batch(S, sc, build_proto(S), [&](const tpk::BuildDev& b, uint64_t rows) {
        mark_launch(e);
        return cuda_check(tpk::launch_many_collect(b, rows, (uint64_t*)k0, (uint32_t*)v0, cnt, e->num_sms, st),
                          "fan-out build");
    });
    if (s) return s;
    TP_TRY_CUDA(cudaMemcpyAsync(S.lane->host_words, cnt, 8, cudaMemcpyDeviceToHost, st));
    TP_TRY_CUDA(cudaStreamSynchronize(st));
    const uint64_t n = S.lane->host_words[0];
    if (n >= (1ull << 31)) return fail(TP_E_INVALID, "fan-out join: more than 2^31 build rows");
    uint64_t *kk = (uint64_t*)k0, *tk = (uint64_t*)k1;
    uint32_t *vv = (uint32_t*)v0, *tv = (uint32_t*)v1;
    TP_TRY_CUDA(tpk::radix_sort_pairs(&kk, &vv, &tk, &tv, (uint32_t*)hist, n, 64, st));
    e->launches += 3 * 8;
    TP_TRY_CUDA(tpk::launch_many_heads(kk, n, (int64_t*)hk, (uint32_t*)hv, cnt + 1, e->num_sms, st));
    mark_launch(e);
    TP_TRY_CUDA(cudaMemcpyAsync(S.lane->host_words, cnt + 1, 8, cudaMemcpyDeviceToHost, st));
    TP_TRY_CUDA(cudaStreamSynchronize(st));
    const uint64_t heads = S.lane->host_words[0];
    TP_TRY_CUDA(tpk::launch_build_pairs(S.jt, (const int64_t*)hk, (const uint32_t*)hv, heads, S.err, e->num_sms, st));
    mark_launch(e);
    S.jt.mkeys = kk;
    S.jt.mpay = vv;
    S.jt.mn = n;
    S.jt.many = 1;
    return TP_OK;
}

// Bytes build_join_many allocates for a dimension of n rows.
uint64_t many_build_bytes(uint64_t n) {
    const uint64_t c = n ? n : 1;
    return 3 * align256(c * 8) + 3 * align256(c * 4) + align256(tpk::radix_sort_hist_words(c) * 4) + 256;
}

// ------------------------------------------------------- fact batch driver

// Runs `kernel(q, rows, colptr)` over every batch of the fact table; colptr[c]
// is the device address of column c in the batch (nullptr when unused).
// Consecutive batches smaller than the table's batch size (a spilled
// partition gets one per fact batch that spilled into it) are copied into one
// staging slot and run as one, up to that size.
template <class F>
tp_status for_each_batch(ExecState& S, Scratch& sc, F&& kernel) {
    tp_engine* e = S.e;
    tp_table* t = S.fact;
    const int nc = (int)t->types.size();
    std::vector<const void*> colptr(nc, nullptr);
    if (t->placement != PL_PAGES) {
        for (int c : S.used) colptr[c] = t->dev_cols[c];
        if (t->rows == 0) return TP_OK;
        tpk::QueryDev q = make_query(S, colptr);
        e->batches++;
        return kernel(q, t->rows, colptr);
    }
    if (t->batches.empty()) return TP_OK;
    // groups of consecutive batches [first, last) of at most `merge` rows
    const uint64_t merge = std::max<uint64_t>(t->batch_rows, 1);
    std::vector<std::pair<size_t, size_t>> groups;
    uint64_t max_rows = 0;
    for (size_t i = 0; i < t->batches.size();) {
        size_t j = i;
        uint64_t rows = 0;
        while (j < t->batches.size() && (j == i || rows + t->batches[j].rows <= merge)) rows += t->batches[j++].rows;
        groups.emplace_back(i, j);
        max_rows = std::max(max_rows, rows);
        i = j;
    }
    const bool prefetch = e->cfg.prefetch_depth > 0;
    const int n_slots = prefetch ? e->cfg.prefetch_depth + 1 : 1;
    // staging slots: every used column of one group, and where batches store
    // narrow columns a second set they are copied into before widening
    const bool narrow = has_narrow(t);
    std::vector<std::vector<void*>> slot(n_slots, std::vector<void*>(nc, nullptr));
    std::vector<std::vector<void*>> enc(n_slots, std::vector<void*>(nc, nullptr));
    std::vector<std::vector<void*>> full_used(n_slots), enc_used(n_slots);
    for (int s = 0; s < n_slots; ++s)
        for (int c : S.used) {
            tp_status st = sc.alloc(&slot[s][c], align256(max_rows * type_size(t->types[c])));
            const int w = narrow ? narrow_width_max(t, c) : 0;
            if (!st && w) st = sc.alloc(&enc[s][c], align256(max_rows * (uint64_t)w + 16));   // + the decoder's word overrun
            if (st) return st;
            full_used[s].push_back(slot[s][c]);
            enc_used[s].push_back(enc[s][c]);
        }
    std::vector<cudaEvent_t> loaded(n_slots), freed(n_slots);
    for (int s = 0; s < n_slots; ++s) {
        cudaEventCreateWithFlags(&loaded[s], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&freed[s], cudaEventDisableTiming);
    }
    tp_status rc = TP_OK;
    if (prefetch) {  // the copy stream may touch the slots only after they exist
        cudaEventRecord(freed[0], S.lane->compute);
        cudaStreamWaitEvent(S.lane->copy, freed[0], 0);
    }
    cudaStream_t cs = prefetch ? S.lane->copy : S.lane->compute;
    std::vector<std::vector<const void*>> gptr(n_slots, std::vector<const void*>(nc, nullptr));
    // copies of group g into slot g % n_slots (after the kernel that last used it)
    // without a page pool (TP_COPY_PINNED_PER_BATCH, an ablation): each group
    // goes through a page-locked buffer allocated for it and freed after its
    // copies
    const bool per_batch_pinned = (e->copy_flags & TP_COPY_PINNED_PER_BATCH) != 0;
    auto issue = [&](size_t g) -> tp_status {
        const int s = (int)(g % n_slots);
        if (prefetch && g >= (size_t)n_slots) cudaStreamWaitEvent(S.lane->copy, freed[s], 0);
        uint8_t* buf = nullptr;
        uint8_t* at = nullptr;
        if (per_batch_pinned) {
            uint64_t bytes = 0;
            for (int c : S.used)
                for (size_t bi = groups[g].first; bi < groups[g].second; ++bi)
                    for (const Extent& x : t->batches[bi].cols[c]) bytes += x.bytes;
            TP_TRY_CUDA(cudaHostAlloc((void**)&buf, bytes ? bytes : 1, cudaHostAllocDefault));
            at = buf;
        }
        for (int c : S.used) {
            uint64_t row_off = 0;
            for (size_t bi = groups[g].first; bi < groups[g].second; ++bi) {
                tp_status r = copy_batch_column(e, t, t->batches[bi], c, slot[s][c], enc[s][c], row_off, cs,
                                                buf ? &at : nullptr);
                if (r) {
                    if (buf) {
                        cudaStreamSynchronize(cs);
                        cudaFreeHost(buf);
                    }
                    return r;
                }
                row_off += t->batches[bi].rows;
            }
            gptr[s][c] = slot[s][c];
        }
        if (buf) {
            TP_TRY_CUDA(cudaStreamSynchronize(cs));
            TP_TRY_CUDA(cudaFreeHost(buf));
        }
        if (prefetch) cudaEventRecord(loaded[s], S.lane->copy);
        return TP_OK;
    };
    // the copy stream runs prefetch_depth groups ahead of the kernels, even
    // while the host waits inside a kernel callback
    const size_t ahead = prefetch ? (size_t)e->cfg.prefetch_depth : 0;
    for (size_t g = 0; g < std::min(ahead, groups.size()) && rc == TP_OK; ++g) rc = issue(g);
    for (size_t g = 0; g < groups.size() && rc == TP_OK; ++g) {
        const int s = (int)(g % n_slots);
        if (g + ahead < groups.size() && (rc = issue(g + ahead))) break;
        if (!prefetch && (rc = issue(g))) break;
        uint64_t rows = 0;
        for (size_t bi = groups[g].first; bi < groups[g].second; ++bi) rows += t->batches[bi].rows;
        if (prefetch) cudaStreamWaitEvent(S.lane->compute, loaded[s], 0);
        if (narrow) {  // widen the narrow columns of every batch of the group, in as few launches as fit
            rc = widen_batches(e, t, groups[g].first, groups[g].second, S.used, full_used[s], enc_used[s],
                               S.lane->compute);
            if (rc) break;
        }
        for (int c : S.used) colptr[c] = gptr[s][c];
        tpk::QueryDev q = make_query(S, colptr);
        rc = kernel(q, rows, colptr);
        e->batches++;
        if (prefetch) cudaEventRecord(freed[s], S.lane->compute);
    }
    if (prefetch) {  // the slots are freed on the compute stream after the last copy
        cudaEventRecord(loaded[0], S.lane->copy);
        cudaStreamWaitEvent(S.lane->compute, loaded[0], 0);
    }
    for (int s = 0; s < n_slots; ++s) {
        cudaEventDestroy(loaded[s]);
        cudaEventDestroy(freed[s]);
        for (int c : S.used) {  // the staging slots go back to the pool after the last kernel
            for (void* p : {slot[s][c], enc[s][c]}) {
                if (!p) continue;
                dev_free(e, p, S.lane->compute);
                sc.ptrs.erase(std::find(sc.ptrs.begin(), sc.ptrs.end(), p));
            }
        }
    }
    return rc;
}

tp_status sample_selectivity(ExecState& S) {
    tp_plan* p = S.p;
    const tp_plan_desc& d = p->d;
    if (d.filter.col < 0) { p->selectivity = 1.0; return TP_OK; }
    tp_table* t = S.fact;
    const uint32_t samples = 4096;
    if (t->rows == 0) { p->selectivity = 1.0; return TP_OK; }
    if (t->placement == PL_PAGES) {
        uint64_t pass = 0;
        for (uint32_t j = 0; j < samples; ++j) {
            uint64_t row = (uint64_t)(((unsigned __int128)j * t->rows) / samples);
            int64_t v = paged_value(t, d.filter.col, row);
            pass += (v >= d.filter.lo && v <= d.filter.hi);
        }
        p->selectivity = (double)pass / samples;
        return TP_OK;
    }
    std::vector<const void*> colptr(t->types.size(), nullptr);
    for (int c : S.used) colptr[c] = t->dev_cols[c];
    tpk::QueryDev q = make_query(S, colptr);
    tp_engine* e = S.e;
    TP_TRY_CUDA(cudaMemsetAsync(S.counters + 3, 0, sizeof(unsigned long long), S.lane->compute));
    TP_TRY_CUDA(tpk::launch_sample_filter(q, t->rows, samples, S.counters + 3, S.lane->compute));
    mark_launch(e);
    TP_TRY_CUDA(cudaMemcpyAsync(S.lane->host_words, S.counters + 3, 8, cudaMemcpyDeviceToHost, S.lane->compute));
    TP_TRY_CUDA(cudaStreamSynchronize(S.lane->compute));
    p->selectivity = (double)S.lane->host_words[0] / samples;
    return TP_OK;
}

// Pass rate of dimension k's predicate on 4096 evenly spaced rows (sizes the
// lookahead filter).
tp_status sample_dim_selectivity(ExecState& S, int k) {
    tp_plan* p = S.p;
    const tp_filter& f = p->dflt[k];
    tp_table* t = p->dims[k];
    const uint32_t samples = 4096;
    if (f.col < 0 || !t || t->rows == 0) { p->dim_sel[k] = 1.0; return TP_OK; }
    const int c = f.col;
    if (t->placement == PL_PAGES) {
        uint64_t pass = 0;
        for (uint32_t j = 0; j < samples; ++j) {
            const int64_t v = paged_value(t, c, (uint64_t)(((unsigned __int128)j * t->rows) / samples));
            pass += (v >= f.lo && v <= f.hi);
        }
        p->dim_sel[k] = (double)pass / samples;
        return TP_OK;
    }
    tpk::QueryDev q{};
    q.fcol = devcol(t, c, t->dev_cols[c]);
    q.flo = f.lo;
    q.fhi = f.hi;
    cudaStream_t st = S.lane->compute;
    TP_TRY_CUDA(cudaMemsetAsync(S.counters + 3, 0, sizeof(unsigned long long), st));
    TP_TRY_CUDA(tpk::launch_sample_filter(q, t->rows, samples, S.counters + 3, st));
    mark_launch(S.e);
    TP_TRY_CUDA(cudaMemcpyAsync(S.lane->host_words, S.counters + 3, 8, cudaMemcpyDeviceToHost, st));
    TP_TRY_CUDA(cudaStreamSynchronize(st));
    p->dim_sel[k] = (double)S.lane->host_words[0] / samples;
    return TP_OK;
}

tp_status map_err(uint32_t err) {
    if (err & tpk::ERR_DUP) return fail(TP_E_DUP_KEY, "join build side holds a duplicate key");
    if (err & tpk::ERR_RANGE) return fail(TP_E_RANGE, "a group field value does not fit its bit width");
    if (err & tpk::ERR_TIMEOUT) return fail(TP_E_TIMEOUT, "a bounded device wait expired");
    if (err & tpk::ERR_INTERNAL) return fail(TP_E_INTERNAL, "device consistency check failed");
    return TP_OK;
}

}  // namespace

namespace tp {

// Output arrays for `cap` groups carved from one allocation.
tp_status alloc_result(tp_engine* e, tp_plan* p, uint64_t cap, tp_result** out, tpk::OutDev* od,
                       unsigned long long* n_groups_dev, cudaStream_t st) {
    const tp_plan_desc& d = p->d;
    int n_avg = 0;
    for (int a = 0; a < d.n_agg; ++a) n_avg += d.aggs[a].kind == TP_AGG_AVG;
    const uint64_t c = cap ? cap : 1;
    uint64_t bytes = align256(c * 8) * 2 + align256(c * 16) * p->n_sum + align256(c * 8) * n_avg;
    tp_status s = reserve(e, bytes);
    if (s) return s;
    tp_result* r = new (std::nothrow) tp_result();
    if (!r) { release(e, bytes); return fail(TP_E_NOMEM, "result: out of host memory"); }
    r->eng = e;
    r->stream = st;
    r->reserved = bytes;
    s = dev_alloc(e, &r->dev, bytes, st);
    if (s) { release(e, bytes); delete r; return s; }
    uint8_t* base = (uint8_t*)r->dev;
    r->d_keys = (uint64_t*)base; base += align256(c * 8);
    r->d_counts = (int64_t*)base; base += align256(c * 8);
    memset(od, 0, sizeof(*od));
    od->keys = r->d_keys;
    od->counts = r->d_counts;
    for (int a = 0; a < d.n_agg; ++a) {
        const int si = p->sum_of_agg[a];
        r->sum_of_agg[a] = si;
        r->is_avg[a] = d.aggs[a].kind == TP_AGG_AVG;
    }
    for (int si = 0; si < p->n_sum; ++si) {
        r->d_sums[si] = (uint64_t*)base;
        od->sums[si] = r->d_sums[si];
        base += align256(c * 16);
    }
    for (int a = 0; a < d.n_agg; ++a) {
        if (!r->is_avg[a]) continue;
        const int si = p->sum_of_agg[a];
        r->d_avgs[si] = (double*)base;
        od->avgs[si] = r->d_avgs[si];
        od->has_avg[si] = 1;
        base += align256(c * 8);
    }
    od->n_groups = n_groups_dev;
    r->n_agg = d.n_agg;
    r->n_sum = p->n_sum;
    r->have_sum.assign(8, false);
    r->have_avg.assign(8, false);
    r->h_sums.resize(8);
    r->h_avgs.resize(8);
    *out = r;
    return TP_OK;
}

}  // namespace tp

namespace {

// Copies rows [0, n) of every array of src to rows [at, at + n) of dst (both
// results of the same plan), on the device.
tp_status copy_result_rows(tp_result* dst, uint64_t at, const tp_result* src, uint64_t n, int n_sum,
                           cudaStream_t st) {
    if (n == 0) return TP_OK;
    TP_TRY_CUDA(cudaMemcpyAsync(dst->d_keys + at, src->d_keys, n * 8, cudaMemcpyDeviceToDevice, st));
    TP_TRY_CUDA(cudaMemcpyAsync(dst->d_counts + at, src->d_counts, n * 8, cudaMemcpyDeviceToDevice, st));
    for (int si = 0; si < n_sum; ++si) {
        TP_TRY_CUDA(cudaMemcpyAsync(dst->d_sums[si] + 2 * at, src->d_sums[si], n * 16, cudaMemcpyDeviceToDevice, st));
        if (dst->d_avgs[si])
            TP_TRY_CUDA(cudaMemcpyAsync(dst->d_avgs[si] + at, src->d_avgs[si], n * 8, cudaMemcpyDeviceToDevice, st));
    }
    return TP_OK;
}

// Rows [0, n) of every array of r copied to host memory (keys, counts, then
// per sum slot the sums and, where present, the averages), and back.
tp_status stash_result_rows(const tp_result* r, uint64_t n, int n_sum, std::vector<uint8_t>* out, cudaStream_t st) {
    uint64_t bytes = 16 * n;
    for (int si = 0; si < n_sum; ++si) bytes += n * (r->d_avgs[si] ? 24 : 16);
    out->resize(bytes);
    uint8_t* h = out->data();
    auto get = [&](const void* dev, uint64_t b) {
        cudaError_t c = cudaMemcpyAsync(h, dev, b, cudaMemcpyDeviceToHost, st);
        h += b;
        return c;
    };
    TP_TRY_CUDA(get(r->d_keys, n * 8));
    TP_TRY_CUDA(get(r->d_counts, n * 8));
    for (int si = 0; si < n_sum; ++si) {
        TP_TRY_CUDA(get(r->d_sums[si], n * 16));
        if (r->d_avgs[si]) TP_TRY_CUDA(get(r->d_avgs[si], n * 8));
    }
    TP_TRY_CUDA(cudaStreamSynchronize(st));
    return TP_OK;
}

tp_status unstash_result_rows(tp_result* r, uint64_t n, int n_sum, const std::vector<uint8_t>& in, cudaStream_t st) {
    const uint8_t* h = in.data();
    auto put = [&](void* dev, uint64_t b) {
        cudaError_t c = cudaMemcpyAsync(dev, h, b, cudaMemcpyHostToDevice, st);
        h += b;
        return c;
    };
    TP_TRY_CUDA(put(r->d_keys, n * 8));
    TP_TRY_CUDA(put(r->d_counts, n * 8));
    for (int si = 0; si < n_sum; ++si) {
        TP_TRY_CUDA(put(r->d_sums[si], n * 16));
        if (r->d_avgs[si]) TP_TRY_CUDA(put(r->d_avgs[si], n * 8));
    }
    TP_TRY_CUDA(cudaStreamSynchronize(st));
    return TP_OK;
}

// Output arrays of od moved on by `at` rows.
tpk::OutDev out_at(tpk::OutDev od, uint64_t at, int n_sum) {
    od.keys += at;
    od.counts += at;
    for (int si = 0; si < n_sum; ++si) {
        od.sums[si] += 2 * at;
        if (od.avgs[si]) od.avgs[si] += at;
    }
    return od;
}

// ------------------------------------------------------ hybrid hash join
//
// A hashed join whose table does not fit the device budget runs partitioned
// (Section 3.3.2: reserve, and spill what is not needed soon; Section 3.1:
// Batch Holders move data to a larger tier).  The build keys are split into
// P partitions by the top bits of fmix64(key).  Partitions whose table fits
// the table budget stay resident: their rows are inserted into one table and
// the fact stream probes it, skipping rows of other partitions.  The build
// and fact rows of the other partitions are spilled to pool pages, then
// joined one partition at a time against the same accumulators.

// Direct-addressed aggregation tables: at most this many slots, and used
// when the key range is at most four times the expected groups (or below
// DIRECT_AGG_ALWAYS slots).
constexpr uint64_t DIRECT_AGG_MAX_SLOTS = 1ull << 27;
// Global aggregation under a filter keeping fewer than this fraction of the
// rows (sampled) selects the passing rows first, then aggregates them; the
// selection vector covers at most SEL_SLICE_ROWS rows (4 bytes each) at once.
constexpr double SELECT_MAX_SELECTIVITY = 0.25;
constexpr uint64_t SEL_SLICE_ROWS = 1ull << 26;

constexpr uint64_t DIRECT_AGG_ALWAYS = 1ull << 20;

// Lookahead filter: used automatically when the join table takes at least
// this; LIP_BITS_PER_KEY filter bits per expected admitted key, at most
// LIP_MAX_BLOCKS 32-byte blocks (32 MB, a quarter of L2).
constexpr uint64_t LIP_TABLE_BYTES = 64ull << 20;
constexpr double LIP_BITS_PER_KEY = 16.0;
constexpr uint64_t LIP_MAX_BLOCKS = 1ull << 20;

// A global aggregation whose table cannot be reserved runs as passes over
// disjoint ranges of the packed group key, each range halved until its table
// fits (Section 3.3.2: a task that runs out of memory is divided up and
// retried); at most this many ranges.
constexpr size_t MAX_AGG_RANGES = 256;

// Device bytes of a global aggregation table and the arrays that turn it into
// a result: direct (span slots, chunk counts and offsets) or hashed (cap + 1
// slots, compaction keys and indices, radix sort histograms).
uint64_t agg_table_bytes(bool direct, uint64_t span, uint64_t cap, uint32_t words) {
    if (direct) {
        const uint64_t n_chunks = (span + tpk::DIRECT_CHUNK - 1) / tpk::DIRECT_CHUNK;
        return align256(span * words * 8) + align256(n_chunks * 4) + align256((n_chunks + 1) * 8);
    }
    return align256((cap + 1) * words * 8) + 2 * align256((cap + 1) * 12) +
           align256(tpk::radix_sort_hist_words(cap + 1) * 4);
}

// Batches whose fact spill copies may still be running when the next batch
// spills (each holds a staging buffer).
constexpr size_t SPILL_BACKLOG = 2;

struct PartJoin {
    bool on = false;
    int P = 0;
    int shift = 0;
    uint64_t spill_mask = 0;               // partitions not resident
    std::vector<uint64_t> dim_count;
    std::vector<tp_table*> build_spill;    // (key i64, payload i32) per spilled partition
    std::vector<tp_table*> fact_spill;     // fact-shaped tables per spilled partition
    unsigned long long* counts = nullptr;  // device: P per-batch counters
    unsigned long long* cursor = nullptr;  // device: P cursors
    bool spill_fact = true;                // false on a retry: the fact spill already happened
    std::deque<cudaEvent_t> inflight;      // fact spill copies still running on the spill stream
    uint64_t table_budget = 0;             // bytes the resident table and one phase-2 table may take
    uint64_t resident_bytes = 0;           // bytes of the resident table
    uint64_t stage_bytes = 0;              // fact spill staging reserved in the budget
    // fact spill accumulation: two device buffer sets, each holding a region
    // of acc_cap rows per spilled partition (every used column, narrow); one
    // set fills over several fact batches while the other's copies to host
    // pages run, so the link sees fewer and larger copies each way
    struct Acc {
        std::vector<void*> col;            // per fact column
        std::vector<uint64_t> fill;        // rows held per partition
        cudaEvent_t done = nullptr;        // its last flush's copies
    };
    Acc acc[2];
    int acc_cur = 0;
    uint64_t acc_cap = 0;                  // rows per partition region; 0 = accumulation off
    bool acc_tried = false;
    std::vector<uint64_t> acc_region;      // first row of each partition's region
    std::vector<uint8_t> enc_w;            // the spill encoding (by the fact table's bounds)
    std::vector<int64_t> enc_base;
    std::vector<int> width;
    ~PartJoin() {
        for (cudaEvent_t ev : inflight) {
            cudaEventSynchronize(ev);
            cudaEventDestroy(ev);
        }
        for (Acc& a : acc)
            if (a.done) {
                cudaEventSynchronize(a.done);
                cudaEventDestroy(a.done);
            }
        for (tp_table* t : build_spill) tp_table_destroy(t);
        for (tp_table* t : fact_spill) tp_table_destroy(t);
    }
};

tp_table* spill_table(tp_engine* e, const std::vector<int32_t>& types) {
    tp_table* t = new (std::nothrow) tp_table();
    if (!t) return nullptr;
    t->eng = e;
    t->types = types;
    t->scales.assign(types.size(), 0);
    t->names.assign(types.size(), "");
    t->batch_rows = e->cfg.batch_rows;
    t->cmin.assign(types.size(), INT64_MIN);
    t->cmax.assign(types.size(), INT64_MAX);
    return t;
}

// Appends nrows rows held in device memory (dev[c] per column, nullptr for a
// column that is not kept) to a spill table as one batch.  The batch's
// columns lie back to back where the previous append ended, in the table's
// page chain (new pool pages as needed), so a partition wastes at most one
// partial page.  Device -> host copies on `st`, synchronised unless !sync
// (the caller then synchronises st before the pages are read).  enc_w /
// enc_base: the columns arrive narrow, with that encoding.
tp_status append_device_rows(tp_engine* e, tp_table* t, const std::vector<const void*>& dev, uint64_t nrows,
                             cudaStream_t st, bool sync = true, const std::vector<uint8_t>* enc_w = nullptr,
                             const std::vector<int64_t>* enc_base = nullptr) {
    if (nrows == 0) return TP_OK;
    const uint64_t pb = e->pool.page_bytes;
    const int nc = (int)t->types.size();
    Batch b;
    b.row0 = t->rows;
    b.rows = nrows;
    b.cols.resize(nc);
    if (enc_w) {   // the rows arrive narrow (frame of reference)
        b.enc_w = *enc_w;
        b.enc_base = *enc_base;
    }
    uint64_t pos = t->chain_used;
    for (int c = 0; c < nc; ++c) {
        if (!dev[c]) continue;
        pos = align256(pos);
        const uint8_t* src = (const uint8_t*)dev[c];
        uint64_t left = nrows * b.width(c, t->types[c]);
        while (left) {
            const uint64_t pi = pos / pb, po = pos % pb, take = std::min<uint64_t>(left, pb - po);
            while (t->chain.size() <= pi) {
                tp_page pg;
                if (tp_page_alloc(e, &pg)) {
                    cudaStreamSynchronize(st);
                    return fail(TP_E_POOL_EMPTY, "spilling a join partition: the page pool is exhausted");
                }
                t->chain.push_back(pg);
            }
            TP_TRY_CUDA(cudaMemcpyAsync((uint8_t*)tp_page_ptr(e, t->chain[pi]) + po, src, take,
                                        cudaMemcpyDeviceToHost, st));
            b.cols[c].push_back(Extent{t->chain[pi], 0, po, take});
            e->d2h_bytes += take;
            src += take;
            pos += take;
            left -= take;
        }
    }
    if (sync) TP_TRY_CUDA(cudaStreamSynchronize(st));
    t->chain_used = pos;
    t->batches.push_back(std::move(b));
    t->rows += nrows;
    return TP_OK;
}

// Histogram of the build keys, residency by table budget, the resident table
// (into S.jt, with the partition filter) and the build-side spill.
tp_status part_setup(ExecState& S, Scratch& sc, PartJoin& pj, uint64_t table_budget, float lf,
                     tpk::BuildDev proto) {
    tp_engine* e = S.e;
    cudaStream_t st = S.lane->compute;
    const int P = pj.P;
    void* words = nullptr;
    tp_status s = sc.alloc(&words, 2 * 8 * (uint64_t)P);
    if (s) return s;
    pj.counts = (unsigned long long*)words;
    pj.cursor = pj.counts + P;
    TP_TRY_CUDA(cudaMemsetAsync(pj.counts, 0, 8 * (uint64_t)P, st));
    const uint64_t slot = S.key64 ? 16 : 8;
    auto table_bytes = [&](uint64_t rows) {
        return pow2_at_least(std::max<uint64_t>(64, (uint64_t)std::ceil(rows / lf))) * slot;
    };
    // the per-partition counts decide residency only when not every build
    // row fits: otherwise the histogram pass over the build side is skipped
    std::vector<unsigned long long> cnt(P, 0);
    if (table_bytes(S.dim->rows) > table_budget) {
        s = for_each_dim_batch(S, sc, proto, [&](const tpk::BuildDev& b, uint64_t rows) {
            mark_launch(e);
            return cuda_check(tpk::launch_part_hist(b, rows, pj.shift, pj.counts, e->num_sms, st),
                              "partition");
        });
        if (s) return s;
        TP_TRY_CUDA(cudaMemcpyAsync(cnt.data(), pj.counts, 8 * (uint64_t)P, cudaMemcpyDeviceToHost, st));
        TP_TRY_CUDA(cudaStreamSynchronize(st));
    } else {
        cnt[0] = S.dim->rows;   // only the total matters below
    }
    pj.dim_count.assign(cnt.begin(), cnt.end());
    // every partition resident when one table of all rows fits; otherwise
    // keep room for the largest partition's own table (phase 2) and fill the
    // rest with resident partitions, in partition order
    const uint64_t all_mask = P == 64 ? ~0ull : ((1ull << P) - 1);
    uint64_t resident_rows = 0, mask = 0, total_rows = 0, largest = 0;
    for (int p = 0; p < P; ++p) {
        total_rows += cnt[p];
        largest = std::max<uint64_t>(largest, table_bytes(cnt[p]));
    }
    if (table_bytes(total_rows) <= table_budget) {
        mask = all_mask;
        resident_rows = total_rows;
    } else {
        const uint64_t room = table_budget > largest ? table_budget - largest : 0;
        for (int p = 0; p < P; ++p) {
            if (table_bytes(resident_rows + cnt[p]) <= room) {
                resident_rows += cnt[p];
                mask |= 1ull << p;
            }
        }
    }
    pj.spill_mask = all_mask & ~mask;
    // the resident table
    const uint64_t cap = pow2_at_least(std::max<uint64_t>(64, (uint64_t)std::ceil(resident_rows / lf)));
    pj.resident_bytes = cap * slot;
    void* slots = nullptr;
    if ((s = sc.alloc(&slots, cap * slot))) return s;
    TP_TRY_CUDA(cudaMemsetAsync(slots, 0xFF, cap * slot, st));
    S.jt.slots = (uint64_t*)slots;
    S.jt.mask = cap - 1;
    S.jt.part_mask = mask;
    S.jt.part_shift = pj.spill_mask ? pj.shift : 0;   // no filter when every partition is resident
    proto.jt = S.jt;
    pj.build_spill.assign(P, nullptr);
    pj.fact_spill.assign(P, nullptr);
    for (int p = 0; p < P; ++p) {
        if (!((pj.spill_mask >> p) & 1ull)) continue;
        pj.build_spill[p] = spill_table(e, {TP_I64, TP_I32});
        pj.fact_spill[p] = spill_table(e, S.fact->types);
        if (!pj.build_spill[p] || !pj.fact_spill[p]) return fail(TP_E_NOMEM, "partition tables: out of host memory");
    }
    // insert resident rows, spill the others
    void *skeys = nullptr, *spays = nullptr;
    uint64_t max_rows = S.dim->placement == PL_PAGES ? 0 : S.dim->rows;
    for (auto& bt : S.dim->batches) max_rows = std::max(max_rows, bt.rows);
    if (pj.spill_mask) {
        if ((s = sc.alloc(&skeys, align256(max_rows * 8))) || (s = sc.alloc(&spays, align256(max_rows * 4)))) return s;
    }
    return for_each_dim_batch(S, sc, proto, [&](const tpk::BuildDev& b, uint64_t rows) -> tp_status {
        mark_launch(e);
        if (!pj.spill_mask) return cuda_check(tpk::launch_build(b, rows, e->num_sms, st), "build");
        TP_TRY_CUDA(cudaMemsetAsync(pj.counts, 0, 2 * 8 * (uint64_t)P, st));
        TP_TRY_CUDA(tpk::launch_part_hist(b, rows, pj.shift, pj.counts, e->num_sms, st));
        std::vector<unsigned long long> bc(P), base(P, 0);
        TP_TRY_CUDA(cudaMemcpyAsync(bc.data(), pj.counts, 8 * (uint64_t)P, cudaMemcpyDeviceToHost, st));
        TP_TRY_CUDA(cudaStreamSynchronize(st));
        uint64_t run = 0;
        for (int p = 0; p < P; ++p) {
            base[p] = run;
            if ((pj.spill_mask >> p) & 1ull) run += bc[p];
        }
        TP_TRY_CUDA(cudaMemcpyAsync(pj.counts, base.data(), 8 * (uint64_t)P, cudaMemcpyHostToDevice, st));
        mark_launch(e);
        TP_TRY_CUDA(tpk::launch_build_part(b, rows, pj.counts, pj.cursor, (int64_t*)skeys, (uint32_t*)spays,
                                           e->num_sms, st));
        for (int p = 0; p < P; ++p) {
            if (!((pj.spill_mask >> p) & 1ull) || bc[p] == 0) continue;
            tp_status r = append_device_rows(e, pj.build_spill[p],
                                             {(const int64_t*)skeys + base[p], (const uint32_t*)spays + base[p]}, bc[p],
                                             st);
            if (r) return r;
        }
        return TP_OK;
    });
}

// Copies every partition's accumulated rows of the current set to its spill
// table (on the spill stream, after the scatters queued so far) and switches
// to the other set once its own previous copies are done.
tp_status part_acc_flush(ExecState& S, PartJoin& pj) {
    PartJoin::Acc& a = pj.acc[pj.acc_cur];
    bool any = false;
    for (uint64_t f : a.fill) any = any || f > 0;
    if (!any) return TP_OK;
    tp_engine* e = S.e;
    cudaStream_t sp = S.lane->spill;
    cudaEvent_t ready = nullptr;
    TP_TRY_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    cudaError_t ce = cudaEventRecord(ready, S.lane->compute);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(sp, ready, 0);
    cudaEventDestroy(ready);
    TP_TRY_CUDA(ce);
    tp_status s = TP_OK;
    for (int p = 0; p < pj.P && s == TP_OK; ++p) {
        if (a.fill[p] == 0) continue;
        std::vector<const void*> part(S.fact->types.size(), nullptr);
        for (int c : S.used) part[c] = (const uint8_t*)a.col[c] + pj.acc_region[p] * (uint64_t)pj.width[c];
        s = append_device_rows(e, pj.fact_spill[p], part, a.fill[p], sp, false, &pj.enc_w, &pj.enc_base);
        a.fill[p] = 0;
    }
    if (s) return s;
    if (!a.done) TP_TRY_CUDA(cudaEventCreateWithFlags(&a.done, cudaEventDisableTiming));
    TP_TRY_CUDA(cudaEventRecord(a.done, sp));
    pj.acc_cur ^= 1;
    PartJoin::Acc& b = pj.acc[pj.acc_cur];
    if (b.done) TP_TRY_CUDA(cudaStreamWaitEvent(S.lane->compute, b.done, 0));   // its copies read it
    return TP_OK;
}

// Sets up the accumulation sets in the spill staging the plan reserved (once;
// off when a partition's region would hold fewer than 4096 rows).
tp_status part_acc_setup(ExecState& S, Scratch& sc, PartJoin& pj) {
    pj.acc_tried = true;
    int n_sp = 0;
    for (int p = 0; p < pj.P; ++p) n_sp += (pj.spill_mask >> p) & 1ull;
    uint64_t row_bytes = 0;
    for (int c : S.used) row_bytes += (uint64_t)pj.width[c];
    if (n_sp == 0 || row_bytes == 0) return TP_OK;
    const uint64_t slack = 2 * 256 * (uint64_t)S.used.size();
    const uint64_t set_bytes = pj.stage_bytes > 2 * slack ? (pj.stage_bytes - 2 * slack) / 2 : 0;
    const uint64_t cap = set_bytes / row_bytes / (uint64_t)n_sp;
    if (cap < 4096) return TP_OK;
    pj.acc_region.assign(pj.P, 0);
    uint64_t at = 0;
    for (int p = 0; p < pj.P; ++p)
        if ((pj.spill_mask >> p) & 1ull) {
            pj.acc_region[p] = at;
            at += cap;
        }
    for (PartJoin::Acc& a : pj.acc) {
        a.col.assign(S.fact->types.size(), nullptr);
        a.fill.assign(pj.P, 0);
        for (int c : S.used) {
            tp_status s = sc.alloc(&a.col[c], align256(at * (uint64_t)pj.width[c]));
            if (s) return s;
        }
    }
    pj.acc_cap = cap;
    return TP_OK;
}

// Fact rows of spilled partitions in this batch go to their spill tables.
tp_status part_spill_fact(ExecState& S, Scratch& sc, PartJoin& pj, const tpk::QueryDev& q, uint64_t rows,
                          const std::vector<const void*>& colptr) {
    if (!pj.spill_mask || !pj.spill_fact || rows == 0) return TP_OK;
    tp_engine* e = S.e;
    cudaStream_t st = S.lane->compute;
    const int P = pj.P;
    TP_TRY_CUDA(cudaMemsetAsync(pj.counts, 0, 2 * 8 * (uint64_t)P, st));
    mark_launch(e);
    TP_TRY_CUDA(tpk::launch_part_hist_fact(q, rows, pj.shift, pj.spill_mask, pj.counts, e->num_sms, st));
    std::vector<unsigned long long> bc(P), base(P, 0);
    TP_TRY_CUDA(cudaMemcpyAsync(bc.data(), pj.counts, 8 * (uint64_t)P, cudaMemcpyDeviceToHost, st));
    TP_TRY_CUDA(cudaStreamSynchronize(st));
    uint64_t total = 0;
    for (int p = 0; p < P; ++p) {
        base[p] = total;
        total += bc[p];
    }
    if (total == 0) return TP_OK;
    if (pj.width.empty()) {   // the spill encoding: narrow by the fact table's bounds, as host pages are
        const int nct = (int)S.fact->types.size();
        const bool narrow = !(e->cfg.flags & TP_FLAG_RAW_PAGES);
        pj.enc_w.assign(nct, 0);
        pj.enc_base.assign(nct, 0);
        pj.width.assign(nct, 0);
        for (int c : S.used) {
            const int full = type_size(S.fact->types[c]);
            pj.enc_w[c] = narrow ? (uint8_t)frame_width(S.fact->cmin[c], S.fact->cmax[c], full) : 0;
            pj.enc_base[c] = S.fact->cmin[c];
            pj.width[c] = pj.enc_w[c] ? pj.enc_w[c] : full;
        }
    }
    if (!pj.acc_tried) {
        tp_status r = part_acc_setup(S, sc, pj);
        if (r) return r;
    }
    bool fits = pj.acc_cap > 0;
    for (int p = 0; p < P && fits; ++p) fits = bc[p] <= pj.acc_cap;
    if (fits) {   // accumulate: scatter into the current set, flushing it first when it is full
        bool full = false;
        for (int p = 0; p < P && !full; ++p) full = pj.acc[pj.acc_cur].fill[p] + bc[p] > pj.acc_cap;
        if (full) {
            tp_status r = part_acc_flush(S, pj);
            if (r) return r;
        }
        PartJoin::Acc& a = pj.acc[pj.acc_cur];
        for (int p = 0; p < P; ++p) base[p] = (pj.spill_mask >> p) & 1ull ? pj.acc_region[p] + a.fill[p] : 0;
        TP_TRY_CUDA(cudaMemcpyAsync(pj.counts, base.data(), 8 * (uint64_t)P, cudaMemcpyHostToDevice, st));
        tpk::SpillCols cols{};
        for (int c : S.used) {
            cols.src[cols.n] = colptr[c];
            cols.dst[cols.n] = a.col[c];
            cols.esize[cols.n] = type_size(S.fact->types[c]);
            cols.w[cols.n] = pj.width[c];
            cols.base[cols.n] = pj.enc_base[c];
            ++cols.n;
        }
        mark_launch(e);
        TP_TRY_CUDA(tpk::launch_fact_spill(q, rows, pj.spill_mask, cols, pj.counts, pj.cursor, e->num_sms, st));
        for (int p = 0; p < P; ++p) a.fill[p] += bc[p];
        return TP_OK;
    }
    // a partition got more rows from this batch than a region holds: flush,
    // then spill this batch on its own
    if (pj.acc_cap) {
        tp_status r = part_acc_flush(S, pj);
        if (r) return r;
    }
    TP_TRY_CUDA(cudaMemcpyAsync(pj.counts, base.data(), 8 * (uint64_t)P, cudaMemcpyHostToDevice, st));
    // at most SPILL_BACKLOG batches' staging waits on its device -> host copies
    while (pj.inflight.size() >= SPILL_BACKLOG) {
        TP_TRY_CUDA(cudaEventSynchronize(pj.inflight.front()));
        cudaEventDestroy(pj.inflight.front());
        pj.inflight.pop_front();
    }
    // spilled rows travel narrow where the fact table's bounds allow, as
    // host pages do: fewer bytes each way over the link
    const int nct = (int)S.fact->types.size();
    std::vector<uint8_t> enc_w(nct, 0);
    std::vector<int64_t> enc_base(nct, 0);
    const bool narrow = !(e->cfg.flags & TP_FLAG_RAW_PAGES);
    tpk::SpillCols cols{};
    std::vector<void*> out(S.fact->types.size(), nullptr);
    std::vector<int> width(nct, 0);
    for (int c : S.used) {
        const int full = type_size(S.fact->types[c]);
        enc_w[c] = narrow ? (uint8_t)frame_width(S.fact->cmin[c], S.fact->cmax[c], full) : 0;
        enc_base[c] = S.fact->cmin[c];
        width[c] = enc_w[c] ? enc_w[c] : full;
        tp_status s = sc.alloc(&out[c], align256(total * (uint64_t)width[c]));
        if (s) return s;
        cols.src[cols.n] = colptr[c];
        cols.dst[cols.n] = out[c];
        cols.esize[cols.n] = full;
        cols.w[cols.n] = width[c];
        cols.base[cols.n] = enc_base[c];
        ++cols.n;
    }
    mark_launch(e);
    TP_TRY_CUDA(tpk::launch_fact_spill(q, rows, pj.spill_mask, cols, pj.counts, pj.cursor, e->num_sms, st));
    // the copies to host pages run on the spill stream (the link's other
    // direction from the prefetch), overlapping the next batches
    cudaStream_t sp = S.lane->spill;
    cudaEvent_t ready = nullptr, done = nullptr;
    TP_TRY_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    cudaError_t ce = cudaEventRecord(ready, st);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(sp, ready, 0);
    cudaEventDestroy(ready);
    TP_TRY_CUDA(ce);
    tp_status s = TP_OK;
    for (int p = 0; p < P && s == TP_OK; ++p) {
        if (bc[p] == 0) continue;
        std::vector<const void*> part(S.fact->types.size(), nullptr);
        for (int c : S.used) part[c] = (const uint8_t*)out[c] + base[p] * (uint64_t)width[c];
        s = append_device_rows(e, pj.fact_spill[p], part, bc[p], sp, false, &enc_w, &enc_base);
    }
    for (int c : S.used) {  // staging goes back (stream-ordered) once its copies are done
        dev_free(e, out[c], sp);
        sc.ptrs.erase(std::find(sc.ptrs.begin(), sc.ptrs.end(), out[c]));
    }
    TP_TRY_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    ce = cudaEventRecord(done, sp);
    if (ce != cudaSuccess) {
        cudaEventDestroy(done);
        TP_TRY_CUDA(ce);
    }
    pj.inflight.push_back(done);
    return s;
}

// Joins every spilled partition: its table from the spilled build pairs, then
// its spilled fact rows through agg (the same per-batch launcher).
template <class F>
tp_status part_phase2(ExecState& S, Scratch& sc, PartJoin& pj, float lf, F&& agg) {
    if (!pj.spill_mask) return TP_OK;
    tp_engine* e = S.e;
    cudaStream_t st = S.lane->compute;
    if (pj.acc_cap) {   // the rows still accumulated on the device
        tp_status r = part_acc_flush(S, pj);
        if (r) return r;
    }
    TP_TRY_CUDA(cudaStreamSynchronize(S.lane->spill));   // every spilled fact row is in its pages
    for (cudaEvent_t ev : pj.inflight) cudaEventDestroy(ev);
    pj.inflight.clear();
    const uint64_t slot = S.key64 ? 16 : 8;
    uint64_t max_cap = 64, max_rows = 0;
    for (int p = 0; p < pj.P; ++p) {
        if (!((pj.spill_mask >> p) & 1ull)) continue;
        max_cap = std::max(max_cap, pow2_at_least(std::max<uint64_t>(64, (uint64_t)std::ceil(pj.dim_count[p] / lf))));
        max_rows = std::max<uint64_t>(max_rows, pj.build_spill[p]->rows);   // a partition's pairs in one launch
    }
    if (max_cap * slot > pj.table_budget - std::min(pj.table_budget, pj.resident_bytes))
        return fail(TP_E_BUDGET, "a spilled join partition needs a %llu-byte table, over the %llu-byte budget; "
                    "use more partitions", (unsigned long long)(max_cap * slot),
                    (unsigned long long)pj.table_budget);
    void *slots = nullptr, *keys = nullptr, *pays = nullptr, *side = nullptr;
    tp_status s;
    if ((s = sc.alloc(&slots, max_cap * slot)) || (s = sc.alloc(&side, 256)) ||
        (s = sc.alloc(&keys, align256(std::max<uint64_t>(1, max_rows) * 8))) ||
        (s = sc.alloc(&pays, align256(std::max<uint64_t>(1, max_rows) * 4))))
        return s;
    tp_table* fact = S.fact;
    const tpk::JoinTable resident = S.jt;
    for (int p = 0; p < pj.P && s == TP_OK; ++p) {
        if (!((pj.spill_mask >> p) & 1ull) || pj.fact_spill[p]->rows == 0) continue;
        const uint64_t cap = pow2_at_least(std::max<uint64_t>(64, (uint64_t)std::ceil(pj.dim_count[p] / lf)));
        TP_TRY_CUDA(cudaMemsetAsync(slots, 0xFF, cap * slot, st));
        TP_TRY_CUDA(cudaMemsetAsync(side, 0, 256, st));
        tpk::JoinTable jt = resident;
        jt.slots = (uint64_t*)slots;
        jt.mask = cap - 1;
        jt.side = (uint32_t*)side;
        jt.part_shift = 0;
        jt.part_mask = 0;
        // every spilled build batch of the partition back to back, then one insert launch
        uint8_t* o[2] = {(uint8_t*)keys, (uint8_t*)pays};
        for (auto& bt : pj.build_spill[p]->batches) {
            for (int c = 0; c < 2; ++c) {
                for (const Extent& x : bt.cols[c]) {
                    TP_TRY_CUDA(cudaMemcpyAsync(o[c], (uint8_t*)tp_page_ptr(e, x.page) + x.offset, x.bytes,
                                                cudaMemcpyHostToDevice, st));
                    o[c] += x.bytes;
                    e->h2d_bytes += x.bytes;
                }
            }
        }
        mark_launch(e);
        TP_TRY_CUDA(tpk::launch_build_pairs(jt, (const int64_t*)keys, (const uint32_t*)pays, pj.build_spill[p]->rows,
                                            S.err, e->num_sms, st));
        S.fact = pj.fact_spill[p];
        S.jt = jt;
        s = for_each_batch(S, sc, agg);
        S.fact = fact;
        S.jt = resident;
    }
    return s;
}


// ------------------------------------------------------- dimension cache

// One execution's use of the dimension cache: a hit (S.jt from the cache), or
// the build of a new entry into cu.mem.
struct CacheUse {
    DimCache* cache = nullptr;
    std::string key;
    bool hit = false;
    bool building = false;
    void* mem = nullptr;
    uint64_t bytes = 0;
    ~CacheUse() {
        if (!cache || (!hit && !building)) return;
        std::lock_guard<std::mutex> lk(cache->mu);
        auto it = cache->entries.find(key);
        if (it != cache->entries.end() && it->second.users > 0) --it->second.users;
        cache->cv.notify_all();
    }
};

std::string cache_key(const ExecState& S) {
    const tp_plan_desc& d = S.p->d;
    char buf[160];
    snprintf(buf, sizeof(buf), "%p:%d:%d:%d:%.4f", (const void*)S.dim, d.join.dim_col, S.jt.direct, S.key64 ? 1 : 0,
             (double)S.p->load_factor);
    std::string k = buf;
    if (d.dim_filter.col >= 0) {
        snprintf(buf, sizeof(buf), "|f%d:%lld:%lld", d.dim_filter.col, (long long)d.dim_filter.lo,
                 (long long)d.dim_filter.hi);
        k += buf;
    }
    for (int g = 0; g < d.n_group; ++g) {
        if (S.p->gdim[g] != 0) continue;   // fields of the cached (first) dimension
        snprintf(buf, sizeof(buf), "|%d:%d:%d", d.group[g].col, d.group[g].bits, S.p->gdpos[g]);
        k += buf;
    }
    return k;
}

tp_status cache_lookup_or_build(ExecState& S, Scratch& sc, DimCache* c, uint64_t join_bytes, CacheUse* cu) {
    (void)sc;
    cu->cache = c;
    cu->key = cache_key(S);
    std::unique_lock<std::mutex> lk(c->mu);
    for (;;) {
        auto it = c->entries.find(cu->key);
        if (it == c->entries.end()) break;
        if (it->second.ready) {
            ++it->second.users;
            it->second.last_use = ++c->tick;
            ++c->hits;
            cu->hit = true;
            S.jt = it->second.jt;
            return TP_OK;
        }
        c->cv.wait(lk);   // another lane is building it
    }
    DimCache::Entry& en = c->entries[cu->key];
    en.users = 1;
    ++c->misses;
    lk.unlock();
    const uint64_t bytes = align256(join_bytes) + 256;   // table + side cell
    tp_status s = reserve(S.e, bytes);
    if (!s) s = dev_alloc(S.e, &cu->mem, bytes, S.lane->compute);
    if (s) {
        if (cu->mem) dev_free(S.e, cu->mem, S.lane->compute);
        lk.lock();
        c->entries.erase(cu->key);
        c->cv.notify_all();
        cu->cache = nullptr;
        return s;
    }
    cu->bytes = bytes;
    cu->building = true;
    return TP_OK;
}

// After S.jt points into cu->mem: build, check the build on this lane, publish.
tp_status cache_publish(ExecState& S, Scratch& sc, DimCache* c, CacheUse* cu) {
    tp_status s = build_join(S, sc);
    uint32_t err = 0;
    if (!s) {
        cudaError_t ce = cudaMemcpyAsync(&err, S.err, 4, cudaMemcpyDeviceToHost, S.lane->compute);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(S.lane->compute);
        if (ce != cudaSuccess) s = fail(TP_E_CUDA, "cached join build: %s", cudaGetErrorString(ce));
        else if (err & tpk::ERR_DUP) s = fail(TP_E_DUP_KEY, "join build side holds a duplicate key");
        else if (err & tpk::ERR_INTERNAL) s = fail(TP_E_INTERNAL, "device consistency check failed");
    }
    std::lock_guard<std::mutex> lk(c->mu);
    if (s) {
        dev_free(S.e, cu->mem, S.lane->compute);
        release(S.e, cu->bytes);
        c->entries.erase(cu->key);
        cu->building = false;
        cu->cache = nullptr;
        c->cv.notify_all();
        return s;
    }
    DimCache::Entry& en = c->entries[cu->key];
    en.jt = S.jt;
    en.mem = cu->mem;
    en.bytes = cu->bytes;
    en.ready = true;
    en.last_use = ++c->tick;
    c->cv.notify_all();
    return TP_OK;
}

// ------------------------------------------------------------- execution

tp_status execute_locked(tp_plan* p, Lane* lane, DimCache* cache, tp_result** out) {
    tp_engine* e = p->eng;
    const tp_plan_desc& d = p->d;
    cudaStream_t st = lane->compute;
    TP_TRY_CUDA(cudaSetDevice(e->device));
    ExecState S;
    S.lane = lane;
    S.p = p;
    S.e = e;
    S.fact = d.fact;
    S.dim = d.join.fact_col >= 0 ? d.dim : nullptr;
    {
        std::vector<bool> u(d.fact->types.size(), false);
        if (d.filter.col >= 0) u[d.filter.col] = true;
        for (int k = 0; k < p->n_dims; ++k) u[p->joins[k].fact_col] = true;
        for (int g = 0; g < d.n_group; ++g)
            if (d.group[g].side == TP_SIDE_FACT) u[d.group[g].col] = true;
        for (int a = 0; a < d.n_agg; ++a) {
            if (d.aggs[a].kind == TP_AGG_COUNT) continue;
            u[d.aggs[a].col_a] = true;
            if (d.aggs[a].kind == TP_AGG_SUM_MUL_SUB) u[d.aggs[a].col_b] = true;
        }
        for (size_t c = 0; c < u.size(); ++c)
            if (u[c]) S.used.push_back((int)c);
    }
    const int ns = p->n_sum;
    const float lf = p->load_factor;
    Scratch sc(e, st);
    // ---- misc words: error word, counters, join side cell
    tp_status s = reserve(e, 4096);
    if (s) return s;
    sc.reserved = 4096;
    void* misc = nullptr;
    if ((s = sc.alloc(&misc, 4096))) return s;
    TP_TRY_CUDA(cudaMemsetAsync(misc, 0, 4096, st));
    S.err = (uint32_t*)misc;
    S.counters = (unsigned long long*)((uint8_t*)misc + 256);
    // ---- filter selectivity from a sample, once per plan (decides eager loads
    // and the first size estimate of a global aggregation table)
    if (p->selectivity < 0 && (s = sample_selectivity(S))) return s;
    for (int k = 0; k < p->n_dims; ++k)
        if (p->dim_sel[k] < 0 && (s = sample_dim_selectivity(S, k))) return s;
    S.eager = p->selectivity >= 0.25;
    // ---- reservation estimate (Section 3.3.2): streaming buffers and the
    // aggregation table first; a hashed join table that would crowd what is
    // left runs partitioned, its table budget taken from the remainder
    uint64_t est = 0;
    if (S.fact->placement == PL_PAGES) {
        const int n_slots = e->cfg.prefetch_depth > 0 ? e->cfg.prefetch_depth + 1 : 1;
        uint64_t max_rows = 0;
        for (auto& b : S.fact->batches) max_rows = std::max(max_rows, b.rows);
        for (int c : S.used)   // full-width slots, and the narrow copies widened into them
            est += n_slots * (align256(max_rows * type_size(S.fact->types[c])) +
                              align256(max_rows * (uint64_t)narrow_width_max(S.fact, c)));
    }
    const bool shared = p->strategy == TP_AGG_SHARED;
    const uint32_t G = shared ? (1u << p->key_bits) : 0;
    // many groups under a selective filter: a selection vector of the passing
    // rows' indices, filled and consumed per slice of at most SEL_SLICE_ROWS
    // rows of a batch
    uint64_t sel_rows = 0;
    if (!shared && !(e->cfg.flags & TP_FLAG_NO_STAGED) && d.filter.col >= 0 && p->n_dims <= 1 && !d.join_many &&
        p->selectivity < SELECT_MAX_SELECTIVITY) {
        uint64_t max_rows = S.fact->placement == PL_PAGES ? 0 : S.fact->rows;
        for (auto& b : S.fact->batches) max_rows = std::max(max_rows, b.rows);
        sel_rows = std::min<uint64_t>(SEL_SLICE_ROWS, max_rows);
        est += align256(sel_rows * 4);
    }
    uint64_t agg_cap = 0;
    bool gdirect = false;           // direct-addressed global table over [rmin, rmin + rspan)
    bool have_range = false;        // packed group keys inside [rmin, rmin + rspan) by the column bounds
    uint64_t rmin = 0, rspan = 0;
    uint64_t groups = 0;            // expected groups (global aggregation)
    uint64_t agg_est = 0;           // global table bytes inside est, reserved per key range later
    const uint32_t words = 2 + 2 * ns;
    uint64_t result_groups = G;
    if (shared) {
        est += align256((uint64_t)G * (1 + 2 * ns) * 8);
    } else {
        groups = d.expected_groups ? d.expected_groups : p->history_groups;
        if (groups == 0) {
            groups = (uint64_t)std::ceil(S.fact->rows * std::min(1.0, p->selectivity * 1.25)) + 16;
            if (p->key_bits < 40) groups = std::min<uint64_t>(groups, 1ull << p->key_bits);
        }
        result_groups = groups;
        have_range = direct_group_range(p, S.fact, S.dim, &rmin, &rspan) && rspan > 0;
        // a dense key range (column bounds) that the groups fill well enough
        // gets a direct-addressed table: no probing, groups come out sorted
        if (!(e->cfg.flags & TP_FLAG_NO_DIRECT_AGG) && have_range && rspan <= DIRECT_AGG_MAX_SLOTS &&
            rspan <= 4 * std::max<uint64_t>(groups, DIRECT_AGG_ALWAYS)) {
            gdirect = true;
            result_groups = std::min(groups, rspan);
            agg_est = agg_table_bytes(true, rspan, 0, words);
        } else {
            // the plan's load factor, also for a group count an earlier
            // execution measured: a fuller table (0.75) cost the staged
            // aggregation more in probe rounds (3M groups: 0.26 -> 0.47 ms)
            // than it saved in table reset and compaction
            agg_cap = pow2_at_least(std::max<uint64_t>(1024, (uint64_t)std::ceil(groups / lf)));
            agg_est = agg_table_bytes(false, 0, agg_cap, words);
        }
        est += agg_est;
    }
    // ---- further tables of a star join: always resident, each sized like a
    // first join's unpartitioned table, with its own lookahead filter under
    // the same rule
    struct XTab {
        bool direct = false, key64 = false;
        uint64_t range = 0, cap = 0, bytes = 0, lip_blocks = 0;
    };
    XTab xt[tpk::MAX_XJOIN];
    for (int j = 0; j + 1 < p->n_dims; ++j) {
        tp_table* t = p->dims[1 + j];
        const int kc = p->joins[1 + j].dim_col;
        XTab& x = xt[j];
        x.key64 = t->types[kc] == TP_I64;
        if (!(e->cfg.flags & TP_FLAG_NO_DIRECT_JOIN) && direct_join_range(t, kc, &x.range)) {
            x.direct = true;
            x.bytes = x.range * 4;
        } else {
            x.cap = pow2_at_least(std::max<uint64_t>(64, (uint64_t)std::ceil(t->rows / lf)));
            x.bytes = x.cap * (x.key64 ? 16 : 8);
        }
        est += align256(x.bytes);
        if (t->placement == PL_PAGES)   // build staging: key, fields and predicate columns
            est += (has_narrow(t) ? 8 : 6) * align256(t->batch_rows * 8);
        if (p->dflt[1 + j].col >= 0 && d.lip != TP_LIP_OFF && (d.lip == TP_LIP_ON || x.bytes >= LIP_TABLE_BYTES)) {
            const double keys = std::ceil((double)t->rows * p->dim_sel[1 + j] * 1.5) + 1024;
            x.lip_blocks = pow2_at_least((uint64_t)std::ceil(keys * LIP_BITS_PER_KEY / 256.0));
            x.lip_blocks = std::min<uint64_t>(std::max<uint64_t>(x.lip_blocks, 2), LIP_MAX_BLOCKS);
            est += x.lip_blocks * 32;
        }
    }
    uint64_t join_bytes = 0, full_join_bytes = 0;
    const bool lip_possible = S.dim && d.dim_filter.col >= 0 && d.lip != TP_LIP_OFF;
    uint64_t lip_blocks = 0, lip_bytes = 0;   // lookahead filter size, when possible
    PartJoin pj;
    uint64_t part_table_budget = 0;
    if (S.dim) {
        S.key64 = S.dim->types[d.join.dim_col] == TP_I64;
        uint64_t range = 0;
        if (!(e->cfg.flags & TP_FLAG_NO_DIRECT_JOIN) && direct_join_range(S.dim, d.join.dim_col, &range)) {
            S.jt.direct = 1;
            S.jt.kmin = S.dim->cmin[d.join.dim_col];
            S.jt.range = range;
            join_bytes = range * 4;
        } else {
            S.join_cap = pow2_at_least(std::max<uint64_t>(64, (uint64_t)std::ceil(S.dim->rows / lf)));
            join_bytes = S.join_cap * (S.key64 ? 16 : 8);
        }
        full_join_bytes = join_bytes;
        if (lip_possible) {
            const double keys = std::ceil((double)S.dim->rows * p->dim_sel[0] * 1.5) + 1024;
            lip_blocks = pow2_at_least((uint64_t)std::ceil(keys * LIP_BITS_PER_KEY / 256.0));
            lip_blocks = std::min<uint64_t>(std::max<uint64_t>(lip_blocks, 2), LIP_MAX_BLOCKS);
            lip_bytes = lip_blocks * 32;
        }
        uint64_t dim_stage =
            S.dim->placement == PL_PAGES ? (has_narrow(S.dim) ? 6 : 4) * align256(S.dim->batch_rows * 8) : 0;
        if (S.dim->placement == PL_PAGES && d.dim_filter.col >= 0)   // the predicate column's staging
            dim_stage += (has_narrow(S.dim) ? 2 : 1) * align256(S.dim->batch_rows * 8);
        if (!S.jt.direct) {  // hybrid hash join when the table would crowd the budget
            uint64_t reserved_now = 0, cap_now = 0;
            tp_budget_query(e, &reserved_now, &cap_now);
            // the result arrays are reserved when the groups are known
            int n_avg = 0;
            for (int a = 0; a < d.n_agg; ++a) n_avg += d.aggs[a].kind == TP_AGG_AVG;
            const uint64_t rg = std::max<uint64_t>(1, result_groups);
            const uint64_t result_est =
                2 * align256(rg * 8) + ns * align256(rg * 16) + (uint64_t)n_avg * align256(rg * 8);
            // room for the lookahead filter too, when the plan may use one
            const uint64_t taken = reserved_now + est + dim_stage + result_est + (lip_possible ? lip_bytes : 0);
            const uint64_t avail = cap_now > taken ? cap_now - taken : 0;
            const int jp = d.join_partitions;
            if (!d.join_many && (jp > 1 || (jp == 0 && join_bytes > avail / 2))) {   // fan-out: never partitioned
                pj.on = true;
                pj.P = jp > 1 ? jp : 64;
                pj.shift = 64;
                for (int v = pj.P; v > 1; v >>= 1) --pj.shift;
                uint64_t fact_rows = 0;
                for (auto& bt : S.fact->batches) fact_rows = std::max(fact_rows, bt.rows);
                if (S.fact->placement != PL_PAGES) fact_rows = S.fact->rows;
                uint64_t used_bytes = 0;
                for (int c : S.used) used_bytes += type_size(S.fact->types[c]);
                // build-pair and fact spill staging, then two tables (the
                // resident one and one spilled partition's) share the rest
                const uint64_t stage =
                    align256(S.dim->batch_rows * 12) + (SPILL_BACKLOG + 1) * align256(fact_rows * used_bytes);
                // a tenth stays free for retries of a table that outgrew its estimate
                part_table_budget = avail > stage ? (avail - stage) / 10 * 9 : 0;
                pj.table_budget = part_table_budget;
                pj.stage_bytes = (SPILL_BACKLOG + 1) * align256(fact_rows * used_bytes);
                join_bytes = part_table_budget + stage;
            }
        }
        if (!(cache && !pj.on) || d.join_many) est += align256(join_bytes);   // a cached table holds its own reservation
        if (d.join_many) est += many_build_bytes(S.dim->rows);
        est += dim_stage;
    }
    est -= agg_est;   // the global table is reserved per key range
    if ((s = reserve(e, est))) return s;
    sc.reserved += est;
    // ---- lookahead filter (Section 5): with a dimension predicate, when the
    // join table would not stay in L2 or the join is partitioned (or asked
    // for); tables shared through the cache go without.  Optional: when its
    // reservation is refused the query runs without it.
    if (lip_possible && !(cache && !pj.on && !d.join_many) &&
        (d.lip == TP_LIP_ON || pj.on || full_join_bytes >= LIP_TABLE_BYTES)) {
        if (reserve(e, lip_bytes) == TP_OK) {
            sc.reserved += lip_bytes;
            void* lip = nullptr;
            if ((s = sc.alloc(&lip, lip_bytes))) return s;
            TP_TRY_CUDA(cudaMemsetAsync(lip, 0, lip_bytes, st));
            int lg = 0;
            while ((1ull << lg) < lip_blocks) ++lg;
            S.jt.lip = (uint32_t*)lip;
            S.jt.lip_shift = 64 - lg;
            e->lip_filters++;
        } else {
            clear_error();
        }
    }
    // ---- join table
    CacheUse cu;
    if (S.dim && cache && !pj.on && !d.join_many) {
        s = cache_lookup_or_build(S, sc, cache, join_bytes, &cu);
        if (s) return s;
    }
    if (S.dim && !cu.hit) {
        void* slots = nullptr;
        if (cu.building) {
            slots = cu.mem;
            TP_TRY_CUDA(cudaMemsetAsync(slots, 0xFF, join_bytes, st));
            TP_TRY_CUDA(cudaMemsetAsync((uint8_t*)slots + align256(join_bytes), 0, 256, st));
        } else if (!pj.on) {
            if ((s = sc.alloc(&slots, join_bytes))) return s;
            TP_TRY_CUDA(cudaMemsetAsync(slots, 0xFF, join_bytes, st));
        }
        S.jt.slots = (uint64_t*)slots;
        S.jt.mask = S.join_cap ? S.join_cap - 1 : 0;
        S.jt.side = cu.building ? (uint32_t*)((uint8_t*)slots + align256(join_bytes))
                                : (uint32_t*)((uint8_t*)misc + 128);
        S.jt.key64 = S.key64 ? 1 : 0;
        if (pj.on) {
            const tpk::BuildDev proto = build_proto(S);
            PhaseTimer pt(e, 0);
            if ((s = part_setup(S, sc, pj, part_table_budget, lf, proto))) return s;
        } else if (d.join_many) {
            if ((s = build_join_many(S, sc))) return s;
        } else if (cu.building) {
            if ((s = cache_publish(S, sc, cache, &cu))) return s;
        } else if ((s = build_join(S, sc))) {
            return s;
        }
    }
    for (int j = 0; j + 1 < p->n_dims; ++j) {   // the further tables of a star join
        const XTab& x = xt[j];
        tpk::JoinTable& jt = S.jtx[j];
        void* slots = nullptr;
        if ((s = sc.alloc(&slots, x.bytes))) return s;
        TP_TRY_CUDA(cudaMemsetAsync(slots, 0xFF, x.bytes, st));
        jt.slots = (uint64_t*)slots;
        jt.direct = x.direct ? 1 : 0;
        jt.kmin = x.direct ? p->dims[1 + j]->cmin[p->joins[1 + j].dim_col] : 0;
        jt.range = x.range;
        jt.mask = x.cap ? x.cap - 1 : 0;
        jt.side = (uint32_t*)((uint8_t*)misc + 136 + 8 * j);   // zeroed with misc
        jt.key64 = x.key64 ? 1 : 0;
        if (x.lip_blocks) {
            void* lip = nullptr;
            if ((s = sc.alloc(&lip, x.lip_blocks * 32))) return s;
            TP_TRY_CUDA(cudaMemsetAsync(lip, 0, x.lip_blocks * 32, st));
            int lg = 0;
            while ((1ull << lg) < x.lip_blocks) ++lg;
            jt.lip = (uint32_t*)lip;
            jt.lip_shift = 64 - lg;
            e->lip_filters++;
        }
        if ((s = build_join(S, sc, 1 + j))) return s;
    }
    // ---- aggregate
    tp_result* res = nullptr;
    KernelTimer timer(e);
    if (shared) {
        void* gacc = nullptr;
        const uint64_t gbytes = (uint64_t)G * (1 + 2 * ns) * 8;
        if ((s = sc.alloc(&gacc, gbytes))) return s;
        TP_TRY_CUDA(cudaMemsetAsync(gacc, 0, gbytes, st));
        const int grid = tpk::agg_shared_grid(p->key_bits, ns, e->num_sms);
        const bool want_staged = !(e->cfg.flags & TP_FLAG_NO_STAGED);
        bool fast = want_staged && !(e->cfg.flags & TP_FLAG_EXACT_ONLY) && sums_fit_int64(p, S.fact);
        tpk::TermBounds bounds[tpk::MAX_SUM] = {};
        if (fast) term_bounds(p, S.fact, bounds);
        int narrow[tpk::MAX_SUM] = {};
        narrow_products(p, S.fact, narrow);
        const bool want_jit = want_staged && !(e->cfg.flags & TP_FLAG_NO_JIT);
        int mode = -1;  // 0 plain exact, 1 staged exact, 2 staged 64-bit
        auto shared_core = [&](const tpk::QueryDev& q, uint64_t rows) -> tp_status {
            tpk::StageLayout L;
            bool can = want_staged && tpk::staged_layout_shared(q, p->key_bits, mode != 1 && fast, bounds, rows,
                                                                e->num_sms, tpk::AOT_GEOM, tpk::ST_MAX_STAGES, &L);
            if (mode < 0 && !can && fast) {  // no 32-bit table fits: exact staged table instead
                fast = false;
                can = want_staged && tpk::staged_layout_shared(q, p->key_bits, false, bounds, rows, e->num_sms,
                                                               tpk::AOT_GEOM, tpk::ST_MAX_STAGES, &L);
            }
            if (mode < 0) mode = can ? (fast ? 2 : 1) : 0;
            if (mode == 2 && !can) return fail(TP_E_INTERNAL, "staged layout changed between batches");
            mark_launch(e);
            // star joins and fan-out: run-time compiled or plain kernels only
            const bool multi = q.n_xjoin > 0 || q.jt.many;
            if (mode > 0 && can) {
                const void* jk = nullptr;
                if (want_jit) {
                    tpk::StageLayout LJ;
                    if (tpk::staged_layout_shared(q, p->key_bits, mode == 2, bounds, rows, e->num_sms,
                                                  tpk::JIT_DENSE_GEOM, tpk::JIT_DENSE_STAGES, &LJ) &&
                        LJ.n_stages == tpk::JIT_DENSE_STAGES && rows >= (uint64_t)LJ.tile) {
                        std::string why;
                        jk = jit_kernel(e, dense_shape(q, LJ, mode == 2, narrow), "tpj_dense", &why);
                        if (jk) {
                            L = LJ;   // the ahead-of-time kernel keeps its own layout
                            e->jit_launches++;
                        }
                    }
                }
                if (multi && !jk) {
                    return cuda_check(timer.run(st, rows, [&] {
                        return tpk::launch_agg_shared(q, rows, (uint64_t*)gacc, p->key_bits, grid, st);
                    }), "aggregate");
                }
                // the run-time compiled kernel takes the ragged tail itself
                const uint64_t whole = jk ? rows : rows / (uint64_t)L.tile * (uint64_t)L.tile;
                tp_status r = cuda_check(timer.run(st, whole, [&] {
                    if (jk)
                        return tpk::launch_agg_shared_staged_jit(jk, q, L, rows, (uint64_t*)gacc, p->key_bits,
                                                                 e->num_sms, st);
                    return tpk::launch_agg_shared_staged(q, L, rows, (uint64_t*)gacc, p->key_bits, mode == 2,
                                                         e->num_sms, st);
                }), "aggregate");
                if (r || whole == rows) return r;
                mark_launch(e);  // rows after the last whole tile
                const tpk::QueryDev qt = tpk::offset_rows(q, whole);
                return cuda_check(tpk::launch_agg_shared(qt, rows - whole, (uint64_t*)gacc, p->key_bits, grid, st),
                                  "aggregate tail");
            }
            return cuda_check(timer.run(st, rows, [&] {
                return tpk::launch_agg_shared(q, rows, (uint64_t*)gacc, p->key_bits, grid, st);
            }), "aggregate");
        };
        auto shared_batch = [&](const tpk::QueryDev& q, uint64_t rows, const std::vector<const void*>& colptr) {
            tp_status r = shared_core(q, rows);
            if (r == TP_OK && pj.on) r = part_spill_fact(S, sc, pj, q, rows, colptr);
            return r;
        };
        {
            PhaseTimer pt(e, pj.on ? 1 : -1);
            s = for_each_batch(S, sc, shared_batch);
        }
        if (s == TP_OK && pj.on) {
            pj.spill_fact = false;
            PhaseTimer pt(e, 2);
            s = part_phase2(S, sc, pj, lf, shared_batch);
        }
        if (s) return s;
        tpk::OutDev od;
        if ((s = alloc_result(e, p, G, &res, &od, S.counters + 1, st))) return s;
        std::unique_ptr<tp_result, void (*)(tp_result*)> guard(res, tp_result_free);
        TP_TRY_CUDA(tpk::launch_final_dense((const uint64_t*)gacc, p->key_bits, ns, od, st, mode == 2));
        mark_launch(e);
        TP_TRY_CUDA(cudaMemcpyAsync(lane->host_words, misc, 8, cudaMemcpyDeviceToHost, st));
        TP_TRY_CUDA(cudaMemcpyAsync(lane->host_words + 1, S.counters + 1, 8, cudaMemcpyDeviceToHost, st));
        TP_TRY_CUDA(cudaStreamSynchronize(st));
        e->d2h_bytes += 16;
        if ((s = map_err((uint32_t)lane->host_words[0]))) return s;
        res->n_groups = lane->host_words[1];
        timer.collect();
        guard.release();
    } else {
        // selective filters: the passing rows are selected first, then
        // aggregated; otherwise the staged kernel unless disabled (all columns
        // staged); 64-bit low-word updates when column bounds rule out
        // overflow (any mix of the kernels then agrees on the low words)
        const bool g_staged = !(e->cfg.flags & TP_FLAG_NO_STAGED);
        const bool gfast = g_staged && !(e->cfg.flags & TP_FLAG_EXACT_ONLY) && sums_fit_int64(p, S.fact);
        const bool stage_all = p->selectivity >= 0.25;
        uint32_t* sel = nullptr;
        unsigned long long* sel_cursor = (unsigned long long*)((uint8_t*)misc + 1024);
        if (sel_rows && (s = sc.alloc((void**)&sel, align256(sel_rows * 4)))) return s;
        // key ranges still to aggregate, the next one at the back (ascending
        // keys come out in order); one range covering every key unless a
        // table had to be split
        struct KeyRange {
            uint64_t lo, span;     // packed keys [lo, lo + span); span 0 = every key
            uint64_t min_cap;      // hashed: capacity learned from an overflow
        };
        std::vector<KeyRange> todo{{rmin, have_range ? rspan : 0, 0}};
        // the result the ranges append to in key order: rows [0, res_at) written
        // of res_cap; a split aggregation sizes it from the keys covered so
        // far and grows it when a later range brings more groups
        uint64_t res_cap = 0, res_at = 0;
        tpk::OutDev res_od{};
        std::unique_ptr<tp_result, void (*)(tp_result*)> res_guard(nullptr, tp_result_free);
        size_t n_ranges = 1;
        uint64_t table_reserved = 0;   // reservation held for the current range's table
        double gscale = 1.0;           // growth of the group estimate learned from overflows
        int attempt = 0;
        auto drop = [&](void* ptr) {
            dev_free(e, ptr, st);
            sc.ptrs.erase(std::find(sc.ptrs.begin(), sc.ptrs.end(), ptr));
        };
        int n_avg = 0;
        for (int a = 0; a < d.n_agg; ++a) n_avg += d.aggs[a].kind == TP_AGG_AVG;
        const uint64_t row_bytes = 16 + 16 * (uint64_t)ns + 8 * (uint64_t)n_avg;
        // room for n more rows in the result (span_end: end of the keys covered)
        auto result_room = [&](uint64_t n, uint64_t span_end) -> tp_status {
            if (res_guard && res_at + n <= res_cap) return TP_OK;
            const uint64_t need_rows = res_at + n;
            uint64_t want = need_rows;
            if (todo.size() > 1) {   // more ranges follow: extrapolate over the key range
                const double covered = (double)(span_end - rmin);
                const double x = std::ceil((double)need_rows * 1.125 * (double)rspan / std::max(1.0, covered));
                want = std::max(need_rows, (uint64_t)std::min(x, (double)rspan));
            }
            const uint64_t want0 = want;
            tp_result* r = nullptr;
            tpk::OutDev od;
            auto alloc_rows = [&]() {   // the extrapolated capacity, else just the rows needed
                tp_status t = alloc_result(e, p, want, &r, &od, nullptr, st);
                if (t == TP_E_BUDGET && want > need_rows) {
                    want = need_rows;
                    t = alloc_result(e, p, want, &r, &od, nullptr, st);
                }
                return t;
            };
            tp_status t = alloc_rows();
            std::vector<uint8_t> stash;
            if (t == TP_E_BUDGET && res_guard) {
                // no room for the old and the new result at once: the rows so
                // far wait in host memory meanwhile (Section 3.1: data moves
                // to a larger memory tier)
                if ((t = stash_result_rows(res_guard.get(), res_at, ns, &stash, st))) return t;
                e->d2h_bytes += stash.size();
                res_guard.reset();
                want = want0;
                t = alloc_rows();
            }
            if (t) return t;
            std::unique_ptr<tp_result, void (*)(tp_result*)> fresh(r, tp_result_free);
            if (!stash.empty()) {
                if ((t = unstash_result_rows(r, res_at, ns, stash, st))) return t;
                e->h2d_bytes += stash.size();
            } else if (res_guard) {
                if ((t = copy_result_rows(r, 0, res_guard.get(), res_at, ns, st))) return t;
                TP_TRY_CUDA(cudaStreamSynchronize(st));
            }
            res_guard.reset(fresh.release());
            res_od = od;
            res_cap = want;
            return TP_OK;
        };
        while (!todo.empty()) {
            const KeyRange kr = todo.back();
            const bool whole = kr.span == 0 || (kr.lo == rmin && kr.span == rspan);
            bool rdirect = gdirect;
            uint64_t rcap = std::max(agg_cap, kr.min_cap);
            if (!whole) {   // table of a part of the key range, sized in proportion
                const uint64_t g = (uint64_t)std::ceil((double)groups * gscale * (double)kr.span / (double)rspan) + 1;
                rdirect = !(e->cfg.flags & TP_FLAG_NO_DIRECT_AGG) && kr.span <= DIRECT_AGG_MAX_SLOTS &&
                          kr.span <= 4 * std::max<uint64_t>(g, DIRECT_AGG_ALWAYS);
                rcap = rdirect ? 0 : std::max(kr.min_cap, pow2_at_least(std::max<uint64_t>(1024, (uint64_t)std::ceil(g / lf))));
            }
            const uint64_t need = agg_table_bytes(rdirect, kr.span, rcap, words);
            s = TP_OK;
            if (need > table_reserved) {
                s = reserve(e, need - table_reserved);
                if (s == TP_OK) sc.reserved += need - table_reserved;
            } else {
                release(e, table_reserved - need);
                sc.reserved -= table_reserved - need;
            }
            if (s == TP_OK) table_reserved = need;
            if (s == TP_OK && have_range) {
                // the range's result rows must fit beside its table: those
                // beyond the result's capacity, at the expected groups
                const double share = whole ? 1.0 : (double)kr.span / (double)rspan;
                const uint64_t g = std::min(kr.span, (uint64_t)std::ceil((double)groups * gscale * share));
                const uint64_t rows = res_at + g > res_cap ? res_at + g - res_cap : 0;
                const uint64_t room = rows ? align256(rows * row_bytes) + 4096 : 0;
                if (room && (s = reserve(e, room)) == TP_OK) release(e, room);
            }
            if (s == TP_E_BUDGET && have_range && kr.span > 1 && n_ranges < MAX_AGG_RANGES) {
                // halve the range (Section 3.3.2: divide the task and retry)
                const uint64_t h = kr.span / 2;
                todo.back() = {kr.lo + h, kr.span - h, 0};
                todo.push_back({kr.lo, h, 0});
                ++n_ranges;
                continue;
            }
            if (s) return s;
            void* tab = nullptr;
            const uint64_t tbytes = rdirect ? kr.span * words * 8 : (rcap + 1) * words * 8;
            if ((s = sc.alloc(&tab, tbytes))) return s;
            if (rdirect) {
                TP_TRY_CUDA(cudaMemsetAsync(tab, 0, tbytes, st));
            } else {
                TP_TRY_CUDA(tpk::launch_init_agg((uint64_t*)tab, rcap + 1, words, st));
                mark_launch(e);
            }
            TP_TRY_CUDA(cudaMemsetAsync(S.counters, 0, 3 * sizeof(unsigned long long), st));
            tpk::AggTable at{};
            at.slots = (uint64_t*)tab;
            at.mask = rdirect ? kr.span - 1 : rcap - 1;
            at.words = words;
            at.direct = rdirect ? 1 : 0;
            at.kmin = kr.lo;
            at.used = S.counters;
            at.max_used = (uint64_t)(rcap * 0.9);
            at.split = whole ? 0 : 1;
            at.key_lo = kr.lo;
            at.key_hi = kr.lo + (kr.span - 1);
            auto global_core = [&](const tpk::QueryDev& q, uint64_t rows) -> tp_status {
                if (sel && tpk::select_usable(q, std::min(rows, sel_rows))) {
                    // selective filter: select the passing rows, then aggregate them
                    // (overlapping a slice's gather with the next selection on a
                    // second stream was measured slower: both contend for DRAM)
                    for (uint64_t off = 0; off < rows; off += sel_rows) {
                        const uint64_t nr = std::min(sel_rows, rows - off);
                        const tpk::QueryDev qs = off ? tpk::offset_rows(q, off) : q;
                        TP_TRY_CUDA(cudaMemsetAsync(sel_cursor, 0, sizeof(unsigned long long), st));
                        mark_launch(e);
                        mark_launch(e);
                        tp_status r = cuda_check(timer.run(st, nr, [&] {
                            cudaError_t ce = tpk::launch_select(qs, nr, sel, sel_cursor, e->num_sms, st);
                            if (ce != cudaSuccess) return ce;
                            return tpk::launch_agg_selected(qs, sel, sel_cursor, nr, at, gfast, e->num_sms, st);
                        }), "aggregate");
                        if (r) return r;
                    }
                    return TP_OK;
                }
                mark_launch(e);
                tpk::StageLayout L;
                if (g_staged && q.n_xjoin == 0 && !q.jt.many && tpk::staged_layout_global(q, stage_all, &L)) {
                    const uint64_t whole_rows = rows / tpk::ST_TILE * tpk::ST_TILE;
                    tp_status r = cuda_check(timer.run(st, whole_rows, [&] {
                        return tpk::launch_agg_global_staged(q, L, rows, at, gfast, e->num_sms, st);
                    }), "aggregate");
                    if (r || whole_rows == rows) return r;
                    mark_launch(e);  // rows after the last whole tile
                    return cuda_check(tpk::launch_agg_global(tpk::offset_rows(q, whole_rows), rows - whole_rows, at,
                                                             e->num_sms, st), "aggregate tail");
                }
                return cuda_check(timer.run(st, rows, [&] {
                    return tpk::launch_agg_global(q, rows, at, e->num_sms, st);
                }), "aggregate");
            };
            auto global_batch = [&](const tpk::QueryDev& q, uint64_t rows, const std::vector<const void*>& colptr) {
                tp_status r = global_core(q, rows);
                if (r == TP_OK && pj.on) r = part_spill_fact(S, sc, pj, q, rows, colptr);
                return r;
            };
            {
                PhaseTimer pt(e, pj.on ? 1 : -1);
                s = for_each_batch(S, sc, global_batch);
            }
            if (s == TP_OK && pj.on) {
                pj.spill_fact = false;   // later passes re-read the spilled partitions, they do not spill again
                PhaseTimer pt(e, 2);
                s = part_phase2(S, sc, pj, lf, global_batch);
            }
            if (s) return s;
            TP_TRY_CUDA(cudaMemcpyAsync(lane->host_words, misc, 8, cudaMemcpyDeviceToHost, st));
            TP_TRY_CUDA(cudaMemcpyAsync(lane->host_words + 1, S.counters, 8, cudaMemcpyDeviceToHost, st));
            TP_TRY_CUDA(cudaStreamSynchronize(st));
            const uint32_t err = (uint32_t)lane->host_words[0];
            if ((s = map_err(err))) return s;
            if (err & tpk::ERR_OVERFLOW) {
                timer.ev.clear();  // a discarded attempt is not counted
                if (++attempt > 6) return fail(TP_E_INTERNAL, "aggregation table overflow after retries");
                // retry with a table sized from what was seen so far (Section 3.3.2:
                // a task that ran out of memory is retried with a better estimate);
                // a table that no longer fits the budget splits the range
                const uint64_t seen = std::max<uint64_t>(lane->host_words[1], rcap);
                const uint64_t ncap = pow2_at_least((uint64_t)std::ceil(4.0 * seen / lf));
                drop(tab);
                gscale *= (double)ncap / (double)rcap;
                if (whole) agg_cap = ncap;
                else todo.back().min_cap = ncap;
                TP_TRY_CUDA(cudaMemsetAsync(misc, 0, 4, st));
                e->retries++;
                continue;
            }
            const uint64_t span_end = kr.lo + kr.span;   // wraps to 0 only for a whole 64-bit range
            uint64_t n = 0;
            if (rdirect) {
                // occupied slots are already in key order: count per chunk,
                // scan, write the rows at their offsets
                const uint64_t n_chunks = (kr.span + tpk::DIRECT_CHUNK - 1) / tpk::DIRECT_CHUNK;
                void *cnts = nullptr, *offs = nullptr;
                if ((s = sc.alloc(&cnts, n_chunks * 4)) || (s = sc.alloc(&offs, (n_chunks + 1) * 8))) return s;
                TP_TRY_CUDA(tpk::launch_direct_count(at, kr.span, (uint32_t*)cnts, e->num_sms, st));
                TP_TRY_CUDA(tpk::launch_direct_scan((const uint32_t*)cnts, n_chunks, (unsigned long long*)offs, st));
                mark_launch(e);
                mark_launch(e);
                TP_TRY_CUDA(cudaMemcpyAsync(lane->host_words, (unsigned long long*)offs + n_chunks, 8,
                                            cudaMemcpyDeviceToHost, st));
                TP_TRY_CUDA(cudaStreamSynchronize(st));
                e->d2h_bytes += 8;
                n = lane->host_words[0];
                if ((s = result_room(n, span_end))) return s;
                TP_TRY_CUDA(tpk::launch_direct_emit(at, kr.span, (const unsigned long long*)offs, ns,
                                                    out_at(res_od, res_at, ns), gfast, e->num_sms, st));
                mark_launch(e);
                TP_TRY_CUDA(cudaStreamSynchronize(st));
                drop(cnts);
                drop(offs);
            } else {
                // compact occupied slots, sort them by key, gather the rows
                void *k0 = nullptr, *k1 = nullptr, *v0 = nullptr, *v1 = nullptr, *hist = nullptr;
                if ((s = sc.alloc(&k0, (rcap + 1) * 8)) || (s = sc.alloc(&k1, (rcap + 1) * 8)) ||
                    (s = sc.alloc(&v0, (rcap + 1) * 4)) || (s = sc.alloc(&v1, (rcap + 1) * 4)) ||
                    (s = sc.alloc(&hist, tpk::radix_sort_hist_words(rcap + 1) * 4)))
                    return s;
                TP_TRY_CUDA(tpk::launch_compact_global(at, rcap + 1, (uint64_t*)k0, (uint32_t*)v0, S.counters + 1,
                                                       S.counters + 2, e->num_sms, st));
                mark_launch(e);
                TP_TRY_CUDA(cudaMemcpyAsync(lane->host_words, S.counters + 1, 16, cudaMemcpyDeviceToHost, st));
                TP_TRY_CUDA(cudaStreamSynchronize(st));
                e->d2h_bytes += 32;
                n = lane->host_words[0];
                const uint64_t maxkey = lane->host_words[1];
                int bits = 0;
                while (bits < 64 && (maxkey >> bits) != 0) ++bits;
                uint64_t *kk = (uint64_t*)k0, *tk = (uint64_t*)k1;
                uint32_t *vv = (uint32_t*)v0, *tv = (uint32_t*)v1;
                TP_TRY_CUDA(tpk::radix_sort_pairs(&kk, &vv, &tk, &tv, (uint32_t*)hist, n, bits, st));
                e->launches += 3 * ((bits + 7) / 8);
                if ((s = result_room(n, span_end))) return s;
                TP_TRY_CUDA(tpk::launch_gather_global(at, kk, vv, n, ns, out_at(res_od, res_at, ns), e->num_sms,
                                                      st, gfast));
                mark_launch(e);
                TP_TRY_CUDA(cudaStreamSynchronize(st));
                for (void* ptr : {k0, k1, v0, v1, hist}) drop(ptr);
            }
            res_at += n;
            drop(tab);
            timer.collect();
            todo.pop_back();
        }
        e->split_passes += n_ranges - 1;
        res = res_guard.release();
        res->n_groups = res_at;
        p->history_groups = res_at;
    }
    sc.free_all();
    *out = res;
    return TP_OK;
}

}  // namespace

namespace tp {

tpk::QueryDev plan_query_dev(const tp_plan* p, const std::vector<const void*>& colptr, const tpk::JoinTable& jt,
                             uint32_t* err, bool eager, const tpk::JoinTable* jtx) {
    const tp_plan_desc& d = p->d;
    tpk::QueryDev q{};
    if (jtx) {   // star join: the further tables and their fact key columns
        q.n_xjoin = p->n_dims > 1 ? p->n_dims - 1 : 0;
        for (int j = 0; j < q.n_xjoin; ++j) {
            const int c = p->joins[1 + j].fact_col;
            q.fkx[j] = devcol(p->d.fact, c, colptr[c]);
            q.jtx[j] = jtx[j];
        }
    }
    q.has_filter = d.filter.col >= 0;
    if (q.has_filter) {
        q.fcol = devcol(p->d.fact, d.filter.col, colptr[d.filter.col]);
        q.flo = d.filter.lo;
        q.fhi = d.filter.hi;
    }
    q.has_join = d.join.fact_col >= 0;
    if (q.has_join) {
        q.fk = devcol(p->d.fact, d.join.fact_col, colptr[d.join.fact_col]);
        q.jt = jt;
    }
    q.n_group = d.n_group;
    for (int g = 0; g < d.n_group; ++g) {
        q.gside[g] = d.group[g].side == TP_SIDE_FACT ? 0 : 1;
        q.gdim[g] = p->gdim[g] < 0 ? 0 : p->gdim[g];
        q.gbits[g] = d.group[g].bits;
        q.gdpos[g] = p->gdpos[g];
        if (d.group[g].side == TP_SIDE_FACT) q.gcol[g] = devcol(p->d.fact, d.group[g].col, colptr[d.group[g].col]);
    }
    q.n_sum = p->n_sum;
    for (int a = 0; a < d.n_agg; ++a) {
        const int s = p->sum_of_agg[a];
        if (s < 0) continue;
        const tp_agg& ag = d.aggs[a];
        q.sa[s] = devcol(p->d.fact, ag.col_a, colptr[ag.col_a]);
        if (ag.kind == TP_AGG_SUM_MUL_SUB) {
            q.skind[s] = tpk::S_MUL_SUB;
            q.sb[s] = devcol(p->d.fact, ag.col_b, colptr[ag.col_b]);
            q.sk[s] = ag.k;
        } else {
            q.skind[s] = tpk::S_SUM;
        }
    }
    q.eager = eager ? 1 : 0;
    q.err = err;
    return q;
}

// True when column bounds prove that every sum of the query stays inside
// int64 over all n fact rows, so kernels may accumulate 64-bit values without
// carry handling.  |a| <= A and |K - b| <= D give |term| <= A * D < 2^127.
bool direct_join_range(const tp_table* dim, int col, uint64_t* range) {
    if (dim->rows == 0) return false;
    const __int128 r = (__int128)dim->cmax[col] - (__int128)dim->cmin[col] + 1;
    if (r <= 0 || r > (__int128)2 * (__int128)dim->rows || r >= ((__int128)1 << 31)) return false;
    *range = (uint64_t)r;
    return true;
}

bool sums_fit_int64(const tp_plan* p, const tp_table* fact) {
    const uint64_t n = fact->rows;
    if (n == 0) return true;
    if (n >= (1ull << 32)) return false;   // per-CTA 32-bit counts
    const tp_plan_desc& d = p->d;
    typedef __int128 i128;
    auto mag = [](i128 v) { return v < 0 ? -v : v; };
    const i128 limit = ((i128)1 << 63) - 1;
    for (int a = 0; a < d.n_agg; ++a) {
        const tp_agg& ag = d.aggs[a];
        if (ag.kind == TP_AGG_COUNT) continue;
        const i128 A = std::max(mag(fact->cmin[ag.col_a]), mag(fact->cmax[ag.col_a]));
        i128 B = A;
        if (ag.kind == TP_AGG_SUM_MUL_SUB) {
            const i128 D = std::max(mag((i128)ag.k - fact->cmin[ag.col_b]), mag((i128)ag.k - fact->cmax[ag.col_b]));
            if (D > limit) return false;
            B = A * D;
        }
        if (B > limit / (i128)n) return false;
    }
    return true;
}

bool direct_group_range(const tp_plan* p, const tp_table* fact, const tp_table* dim, uint64_t* kmin,
                        uint64_t* span) {
    const tp_plan_desc& d = p->d;
    if (d.n_group == 0) return false;
    unsigned __int128 lo = 0, hi = 0;
    for (int g = 0; g < d.n_group; ++g) {
        const tp_table* t = p->gdim[g] < 0 ? fact : (p->gdim[g] == 0 ? dim : p->dims[p->gdim[g]]);
        const int col = d.group[g].col, bits = d.group[g].bits;
        if (!t || t->rows == 0 || t->cmin[col] < 0) return false;
        if (bits < 64 && ((uint64_t)t->cmax[col] >> bits) != 0) return false;
        lo = (lo << bits) | (uint64_t)t->cmin[col];
        hi = (hi << bits) | (uint64_t)t->cmax[col];
    }
    *kmin = (uint64_t)lo;
    *span = (uint64_t)(hi - lo + 1);
    return true;
}

// Sum slots whose product a * (k - b) has both factors inside int32 by the
// column statistics (the run-time compiled kernels multiply those in 32 bits).
void narrow_products(const tp_plan* p, const tp_table* fact, int* out) {
    const tp_plan_desc& d = p->d;
    for (int a = 0; a < d.n_agg; ++a) {
        const int s = p->sum_of_agg[a];
        const tp_agg& ag = d.aggs[a];
        if (s < 0 || ag.kind != TP_AGG_SUM_MUL_SUB || fact->rows == 0) continue;
        const __int128 d0 = (__int128)ag.k - fact->cmax[ag.col_b], d1 = (__int128)ag.k - fact->cmin[ag.col_b];
        out[s] = fact->cmin[ag.col_a] >= INT32_MIN && fact->cmax[ag.col_a] <= INT32_MAX && d0 >= INT32_MIN &&
                 d1 <= INT32_MAX;
    }
}

// A plan shape as a struct of compile-time constants for the run-time
// compiled kernels (fields: jit_common.cuh).  mode[s]: 32-bit accumulation
// mode of sum s (fast only).
std::string shape_struct(const std::string& name, const tpk::QueryDev& q, const int8_t* mode_in, bool fast,
                         bool lo_only, const int* narrow) {
    auto arr = [](const char* nm, const int* v, int n) {
        std::string r = std::string(nm) + "[" + std::to_string(n) + "] = {";
        for (int i = 0; i < n; ++i) r += (i ? ", " : "") + std::to_string(v[i]);
        return r + "}";
    };
    int gside[tpk::MAX_GROUP] = {}, gtype[tpk::MAX_GROUP] = {}, gbits[tpk::MAX_GROUP] = {};
    for (int g = 0; g < q.n_group; ++g) {
        gside[g] = q.gside[g];
        gtype[g] = q.gside[g] == 0 ? q.gcol[g].type : 0;
        gbits[g] = q.gbits[g];
    }
    int skind[tpk::MAX_SUM] = {}, atype[tpk::MAX_SUM] = {}, btype[tpk::MAX_SUM] = {}, mode[tpk::MAX_SUM] = {},
        nar[tpk::MAX_SUM] = {};
    for (int s = 0; s < q.n_sum; ++s) {
        skind[s] = q.skind[s];
        atype[s] = q.sa[s].type;
        btype[s] = q.skind[s] == tpk::S_MUL_SUB ? q.sb[s].type : 0;
        mode[s] = fast ? mode_in[s] : 0;
        nar[s] = fast && mode[s] == 2 && q.skind[s] == tpk::S_MUL_SUB ? narrow[s] : 0;
    }
    const int join = !q.has_join ? 0 : (q.jt.direct ? 1 : (q.jt.key64 ? 3 : 2));
    int xjoin[tpk::MAX_XJOIN] = {}, xktype[tpk::MAX_XJOIN] = {}, xlip[tpk::MAX_XJOIN] = {}, gdim[tpk::MAX_GROUP] = {};
    for (int j = 0; j < q.n_xjoin; ++j) {
        xjoin[j] = q.jtx[j].direct ? 1 : (q.jtx[j].key64 ? 3 : 2);
        xktype[j] = q.fkx[j].type;
        xlip[j] = q.jtx[j].lip != nullptr ? 1 : 0;
    }
    for (int g = 0; g < q.n_group; ++g) gdim[g] = q.gside[g] != 0 ? q.gdim[g] : 0;
    std::string r = "struct " + name + " {\n";
    r += "    static constexpr int filter = " + std::to_string(q.has_filter ? 1 : 0) +
         ", ftype = " + std::to_string(q.has_filter ? q.fcol.type : 0) + ", join = " + std::to_string(join) +
         ", ktype = " + std::to_string(q.has_join ? q.fk.type : 0) +
         ", part = " + std::to_string(q.has_join && q.jt.part_shift != 0 ? 1 : 0) +
         ", lip = " + std::to_string(q.has_join && q.jt.lip != nullptr ? 1 : 0) +
         ", many = " + std::to_string(q.has_join && q.jt.many ? 1 : 0) + ";\n";
    r += "    static constexpr int nx = " + std::to_string(q.n_xjoin) + ", " + arr("xjoin", xjoin, tpk::MAX_XJOIN) +
         ", " + arr("xktype", xktype, tpk::MAX_XJOIN) + ", " + arr("xlip", xlip, tpk::MAX_XJOIN) + ";\n";
    r += "    static constexpr int ng = " + std::to_string(q.n_group) + ", " + arr("gdim", gdim, tpk::MAX_GROUP) + ";\n";
    r += "    static constexpr int " + arr("gside", gside, tpk::MAX_GROUP) + ", " + arr("gtype", gtype, tpk::MAX_GROUP) +
         ", " + arr("gbits", gbits, tpk::MAX_GROUP) + ";\n";
    r += "    static constexpr int ns = " + std::to_string(q.n_sum) + ";\n";
    r += "    static constexpr int " + arr("skind", skind, tpk::MAX_SUM) + ", " + arr("atype", atype, tpk::MAX_SUM) +
         ", " + arr("btype", btype, tpk::MAX_SUM) + ", " + arr("mode", mode, tpk::MAX_SUM) + ", " +
         arr("narrow", nar, tpk::MAX_SUM) + ";\n";
    r += std::string("    static constexpr bool fast = ") + (fast ? "true" : "false") +
         ", lo_only = " + (!fast && lo_only ? "true" : "false") + ";\n};\n";
    return r;
}

// The source of a dense staged launch's run-time compiled kernel.
std::string dense_shape(const tpk::QueryDev& q, const tpk::StageLayout& L, bool fast, const int* narrow) {
    return shape_struct("JS", q, L.sum_mode, fast, false, narrow) + "#include \"jit_dense.cuh\"\n";
}

// Per-row term range of every sum slot, from column statistics.
void term_bounds(const tp_plan* p, const tp_table* fact, tpk::TermBounds* out) {
    const tp_plan_desc& d = p->d;
    typedef __int128 i128;
    for (int a = 0; a < d.n_agg; ++a) {
        const int s = p->sum_of_agg[a];
        if (s < 0) continue;
        const tp_agg& ag = d.aggs[a];
        i128 lo = fact->cmin[ag.col_a], hi = fact->cmax[ag.col_a];
        if (ag.kind == TP_AGG_SUM_MUL_SUB) {
            const i128 d0 = (i128)ag.k - fact->cmax[ag.col_b], d1 = (i128)ag.k - fact->cmin[ag.col_b];
            const i128 c[4] = {lo * d0, lo * d1, hi * d0, hi * d1};
            lo = hi = c[0];
            for (int i = 1; i < 4; ++i) {
                lo = c[i] < lo ? c[i] : lo;
                hi = c[i] > hi ? c[i] : hi;
            }
        }
        // only used when sums_fit_int64 holds, so both ends fit in int64
        out[s].lo = (int64_t)lo;
        out[s].span = (uint64_t)(hi - lo);
    }
}

tp_status execute_on_lane(tp_plan* p, Lane* lane, DimCache* cache, tp_result** out) {
    clear_error();
    if (!p || !out || !lane) return fail(TP_E_INVALID, "execute: NULL argument");
    *out = nullptr;
    return execute_locked(p, lane, cache, out);
}

int cache_evict_idle(tp_engine* e, DimCache* c, uint64_t need) {
    std::lock_guard<std::mutex> lk(c->mu);
    int n = 0;
    uint64_t freed = 0;
    for (;;) {
        auto victim = c->entries.end();
        for (auto it = c->entries.begin(); it != c->entries.end(); ++it)
            if (it->second.ready && it->second.users == 0 &&
                (victim == c->entries.end() || it->second.last_use < victim->second.last_use))
                victim = it;
        if (victim == c->entries.end()) break;
        cudaFree(victim->second.mem);   // idle: no work of any stream references it
        release(e, victim->second.bytes);
        freed += victim->second.bytes;
        c->entries.erase(victim);
        ++c->evictions;
        ++n;
        if (need && freed >= need) break;
    }
    return n;
}

}  // namespace tp

extern "C" {

tp_status tp_plan_create(tp_engine* e, const tp_plan_desc* d, tp_plan** out) {
    clear_error();
    if (!e || !d || !out) return fail(TP_E_INVALID, "tp_plan_create: NULL argument");
    *out = nullptr;
    const tp_table* f = d->fact;
    if (!f || f->eng != e) return fail(TP_E_INVALID, "plan: fact table missing or from another engine");
    if (d->filter.col != -1 && !valid_col(f, d->filter.col)) return fail(TP_E_INVALID, "plan: bad filter column");
    const bool join = d->join.fact_col >= 0;
    if (join) {
        if (!valid_col(f, d->join.fact_col)) return fail(TP_E_INVALID, "plan: bad join fact column");
        if (!d->dim || d->dim->eng != e || !valid_col(d->dim, d->join.dim_col))
            return fail(TP_E_INVALID, "plan: bad dimension table or key column");
    } else if (d->join.fact_col != -1) {
        return fail(TP_E_INVALID, "plan: bad join fact column");
    }
    if (d->dim_filter_on && (!join || !valid_col(d->dim, d->dim_filter.col)))
        return fail(TP_E_INVALID, "plan: bad dimension predicate column");
    if (d->lip < TP_LIP_AUTO || d->lip > TP_LIP_ON) return fail(TP_E_INVALID, "plan: bad lip mode");
    if (d->n_group < 0 || d->n_group > 4) return fail(TP_E_INVALID, "plan: 0..4 group fields");
    if (d->n_agg < 1 || d->n_agg > 8) return fail(TP_E_INVALID, "plan: 1..8 aggregates");
    if (d->join_many && (!join || d->join_partitions > 1))
        return fail(TP_E_INVALID, "plan: a fan-out join needs a join and is never partitioned");
    if (d->n_extra_dims < 0 || d->n_extra_dims > TP_MAX_EXTRA_DIMS || (d->n_extra_dims > 0 && !join))
        return fail(TP_E_INVALID, "plan: 0..%d further dimensions, after a first join", TP_MAX_EXTRA_DIMS);
    for (int j = 0; j < d->n_extra_dims; ++j) {
        const tp_table* x = d->extra_dim[j];
        if (!x || x->eng != e || !valid_col(f, d->extra_join[j].fact_col) || !valid_col(x, d->extra_join[j].dim_col))
            return fail(TP_E_INVALID, "plan: bad further dimension %d or its join columns", j);
        if (d->extra_dim_filter_on[j] && !valid_col(x, d->extra_dim_filter[j].col))
            return fail(TP_E_INVALID, "plan: bad predicate column of further dimension %d", j);
    }
    std::unique_ptr<tp_plan> p(new (std::nothrow) tp_plan());
    if (!p) return fail(TP_E_NOMEM, "plan: out of host memory");
    static std::atomic<uint64_t> next_serial{1};
    p->eng = e;
    p->serial = next_serial++;
    p->d = *d;
    if (!d->dim_filter_on) p->d.dim_filter.col = -1;   // internally: col < 0 = no predicate
    if (join) {   // every joined dimension in one list: the first, then the further ones
        p->n_dims = 1 + d->n_extra_dims;
        p->dims[0] = d->dim;
        p->joins[0] = d->join;
        p->dflt[0] = p->d.dim_filter;
        for (int j = 0; j < d->n_extra_dims; ++j) {
            p->dims[1 + j] = d->extra_dim[j];
            p->joins[1 + j] = d->extra_join[j];
            p->dflt[1 + j] = d->extra_dim_filter[j];
            if (!d->extra_dim_filter_on[j]) p->dflt[1 + j].col = -1;
        }
    }
    int key_bits = 0, dim_bits[4] = {0, 0, 0, 0};
    for (int g = 0; g < d->n_group; ++g) {
        const tp_group_field& gf = d->group[g];
        if (gf.bits < 1 || gf.bits > 64) return fail(TP_E_INVALID, "plan: group field %d needs 1..64 bits", g);
        key_bits += gf.bits;
        p->gdpos[g] = 0;
        p->gdim[g] = -1;
        if (gf.side == TP_SIDE_FACT) {
            if (!valid_col(f, gf.col)) return fail(TP_E_INVALID, "plan: bad group column %d", g);
        } else if (gf.side >= TP_SIDE_DIM && gf.side < TP_SIDE_DIM + p->n_dims) {
            const int k = gf.side - TP_SIDE_DIM;   // payload of dimension k
            if (!valid_col(p->dims[k], gf.col)) return fail(TP_E_INVALID, "plan: bad dimension group column %d", g);
            p->gdim[g] = k;
            p->gdpos[g] = dim_bits[k];
            dim_bits[k] += gf.bits;
        } else {
            return fail(TP_E_INVALID, "plan: bad group side %d", g);
        }
    }
    if (key_bits > 64) return fail(TP_E_INVALID, "plan: group key wider than 64 bits");
    for (int k = 0; k < 4; ++k)
        if (dim_bits[k] > tpk::MAX_DIM_BITS)
            return fail(TP_E_INVALID, "plan: group fields of one dimension wider than 31 bits");
    const int dim_bits0 = dim_bits[0];
    int ns = 0;
    for (int a = 0; a < d->n_agg; ++a) {
        const tp_agg& ag = d->aggs[a];
        p->sum_of_agg[a] = -1;
        switch (ag.kind) {
        case TP_AGG_COUNT: break;
        case TP_AGG_SUM_MUL_SUB:
            if (!valid_col(f, ag.col_b)) return fail(TP_E_INVALID, "plan: bad aggregate column");
            /* fallthrough */
        case TP_AGG_SUM:
        case TP_AGG_AVG:
            if (!valid_col(f, ag.col_a)) return fail(TP_E_INVALID, "plan: bad aggregate column");
            p->sum_of_agg[a] = ns++;
            break;
        default: return fail(TP_E_INVALID, "plan: bad aggregate kind");
        }
    }
    p->n_sum = ns;
    p->key_bits = key_bits;
    p->dim_bits = dim_bits0;
    p->load_factor = d->load_factor > 0 ? d->load_factor : e->cfg.load_factor;
    if (!(p->load_factor > 0.05f && p->load_factor <= 0.9f)) return fail(TP_E_INVALID, "plan: bad load factor");
    const int jp = d->join_partitions;
    if (jp < 0 || jp > 64 || (jp > 1 && (jp & (jp - 1)) != 0))
        return fail(TP_E_INVALID, "plan: join_partitions must be 0, 1 or a power of two up to 64");
    const int want = d->agg_strategy ? d->agg_strategy : e->cfg.agg_strategy;
    const bool fits_shared = key_bits <= 12 && tpk::agg_shared_smem_bytes(key_bits, ns) <= 160 * 1024;
    if (want == TP_AGG_SHARED && !fits_shared)
        return fail(TP_E_INVALID, "plan: shared-memory aggregation needs a key of at most 12 bits");
    if (want < TP_AGG_AUTO || want > TP_AGG_GLOBAL) return fail(TP_E_INVALID, "plan: bad strategy");
    p->strategy = (want == TP_AGG_GLOBAL || !fits_shared) ? TP_AGG_GLOBAL : TP_AGG_SHARED;
    *out = p.release();
    return TP_OK;
}

void tp_plan_destroy(tp_plan* p) { delete p; }

tp_status tp_execute(tp_plan* p, tp_result** out) {
    clear_error();
    if (!p || !out) return fail(TP_E_INVALID, "tp_execute: NULL argument");
    *out = nullptr;
    std::lock_guard<std::mutex> lk(p->eng->exec_mu);
    return execute_locked(p, &p->eng->lane0, nullptr, out);
}

// ----------------------------------------------------------------- results

uint64_t tp_result_groups(const tp_result* r) { return r ? r->n_groups : 0; }

static bool fetch(tp_result* r, void* dst, const void* src, uint64_t bytes) {
    if (bytes == 0) return true;
    if (cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        fail(TP_E_CUDA, "result copy failed");
        return false;
    }
    r->eng->d2h_bytes += bytes;
    return true;
}

const uint64_t* tp_result_keys(tp_result* r) {
    if (!r) return nullptr;
    std::lock_guard<std::mutex> lk(r->mu);
    if (!r->have_keys) {
        r->h_keys.resize(r->n_groups ? r->n_groups : 1);
        if (!fetch(r, r->h_keys.data(), r->d_keys, r->n_groups * 8)) return nullptr;
        r->have_keys = true;
    }
    return r->h_keys.data();
}

const int64_t* tp_result_count(tp_result* r) {
    if (!r) return nullptr;
    std::lock_guard<std::mutex> lk(r->mu);
    if (!r->have_counts) {
        r->h_counts.resize(r->n_groups ? r->n_groups : 1);
        if (!fetch(r, r->h_counts.data(), r->d_counts, r->n_groups * 8)) return nullptr;
        r->have_counts = true;
    }
    return r->h_counts.data();
}

const tp_i128* tp_result_sum(tp_result* r, int32_t agg) {
    if (!r || agg < 0 || agg >= r->n_agg || r->sum_of_agg[agg] < 0) return nullptr;
    const int si = r->sum_of_agg[agg];
    std::lock_guard<std::mutex> lk(r->mu);
    if (!r->have_sum[si]) {
        r->h_sums[si].resize(r->n_groups ? r->n_groups : 1);
        if (!fetch(r, r->h_sums[si].data(), r->d_sums[si], r->n_groups * 16)) return nullptr;
        r->have_sum[si] = true;
    }
    return r->h_sums[si].data();
}

const double* tp_result_avg(tp_result* r, int32_t agg) {
    if (!r || agg < 0 || agg >= r->n_agg || !r->is_avg[agg]) return nullptr;
    const int si = r->sum_of_agg[agg];
    std::lock_guard<std::mutex> lk(r->mu);
    if (!r->have_avg[si]) {
        r->h_avgs[si].resize(r->n_groups ? r->n_groups : 1);
        if (!fetch(r, r->h_avgs[si].data(), r->d_avgs[si], r->n_groups * 8)) return nullptr;
        r->have_avg[si] = true;
    }
    return r->h_avgs[si].data();
}

const void* tp_result_device_keys(const tp_result* r) { return r ? r->d_keys : nullptr; }
const void* tp_result_device_count(const tp_result* r) { return r ? r->d_counts : nullptr; }

const void* tp_result_device_sum(const tp_result* r, int32_t agg) {
    if (!r || agg < 0 || agg >= r->n_agg || r->sum_of_agg[agg] < 0) return nullptr;
    return r->d_sums[r->sum_of_agg[agg]];
}

const void* tp_result_device_avg(const tp_result* r, int32_t agg) {
    if (!r || agg < 0 || agg >= r->n_agg || !r->is_avg[agg]) return nullptr;
    return r->d_avgs[r->sum_of_agg[agg]];
}

void tp_result_free(tp_result* r) {
    if (!r) return;
    tp_engine* e = r->eng;
    if (r->dev) {
        cudaSetDevice(e->device);
        cudaStream_t rs = r->stream ? r->stream : e->compute;
        cudaStreamSynchronize(rs);
        dev_free(e, r->dev, rs);
    }
    if (r->reserved) release(e, r->reserved);
    delete r;
}

}  // extern "C"
