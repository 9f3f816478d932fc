// tp_execute_noalloc: the low-cardinality star query without any device
// allocation.
//
// Some callers cannot allocate GPU memory while they run a query: a host
// application that has handed all device memory to its own allocator (a
// database buffer pool, PyTorch's caching allocator) and forbids side
// allocations, or a latency-bound caller for whom cudaMalloc/cudaFree -- which
// may synchronise the device or fail under fragmentation -- is not
// acceptable in the middle of its work.  This entry point serves them: the
// caller passes device input columns and device output arrays, and every
// piece of scratch the kernels need (join hash table, per-group
// accumulators, status words) lives in one fixed, file-scope device array.
//
// The array is NOLOC_SCRATCH_BYTES long and is held by every GPU that loads
// this library until the process exits.  The first call made with a device
// current sets that device up: it looks up the array's device address and
// loads the kernels the call launches, which is when the CUDA driver places
// the array and the kernel code in device memory (with lazy module loading
// this would otherwise happen at a later first launch).  So make that first
// call at start-up, before handing the rest of device memory to another
// allocator, and before any stream capture; later calls allocate nothing.
// Every call shares the array and starts by clearing what must start at
// zero; calls whose work overlaps on the GPU (different streams, or different
// host threads) race on it and must be serialised by the caller.
#include <cmath>
#include <mutex>

#include "tp_internal.h"

namespace {

constexpr uint64_t NOLOC_MISC_BYTES = 256;                        // status words, join side cell
constexpr uint64_t NOLOC_ACC_BYTES = 4096ull * (1 + 2 * 8) * 8;   // 4096 groups x 8 sums (557,056 B)
constexpr uint64_t NOLOC_JOIN_BYTES = 8ull << 20;                 // 2^20 8-byte or 2^19 16-byte slots
constexpr uint64_t NOLOC_SCRATCH_BYTES = NOLOC_MISC_BYTES + NOLOC_ACC_BYTES + NOLOC_JOIN_BYTES;

}  // namespace

static __device__ __align__(256) unsigned char tp_noalloc_scratch[NOLOC_SCRATCH_BYTES];

namespace {

constexpr int NOLOC_MAX_DEVICES = 64;
std::mutex g_noloc_mu;
void* g_noloc_addr[NOLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set up once).
tp_status noloc_scratch(void** out) {
    int dev = 0;
    TP_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOLOC_MAX_DEVICES) return tp::fail(TP_E_INVALID, "tp_execute_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noloc_mu);
    if (!g_noloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, tp_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return tp::fail(TP_E_CUDA, "tp_execute_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        }
        e = tpk::load_plain_kernels();
        if (e != cudaSuccess) {
            cudaGetLastError();
            return tp::fail(TP_E_CUDA, "tp_execute_noalloc: loading its kernels failed: %s", cudaGetErrorString(e));
        }
        g_noloc_addr[dev] = p;
    }
    *out = g_noloc_addr[dev];
    return TP_OK;
}

bool col_ok(int32_t c, int32_t n) { return c >= 0 && c < n; }

uint64_t pow2_ge(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

tpk::DevCol dcol(const void* const* cols, const int32_t* types, int32_t c) {
    tpk::DevCol d{};
    d.ptr = cols[c];
    d.type = types[c];
    return d;
}

}  // namespace

extern "C" tp_status tp_execute_noalloc(const tp_plan_desc* d, const void* const* fact_cols,
                                        const int32_t* fact_types, int32_t n_fact_cols, uint64_t n_fact,
                                        const void* const* dim_cols, const int32_t* dim_types,
                                        int32_t n_dim_cols, uint64_t n_dim, uint64_t* keys, int64_t* counts,
                                        tp_i128* const* sums, double* const* avgs, uint64_t* n_groups,
                                        void* stream) {
    using tp::fail;
    tp::clear_error();
    if (!d || !fact_types || !keys || !counts || !n_groups || n_fact_cols < 1 || n_fact_cols > 32 ||
        (n_fact && !fact_cols))
        return fail(TP_E_INVALID, "tp_execute_noalloc: NULL or bad argument");
    const bool join = d->join.fact_col >= 0;
    for (int c = 0; c < n_fact_cols; ++c)
        if (tp::type_size(fact_types[c]) == 0 || (n_fact && (!fact_cols[c] || ((uintptr_t)fact_cols[c] & 15u))))
            return fail(TP_E_INVALID, "tp_execute_noalloc: fact column %d: bad type, NULL or not 16-byte aligned", c);
    if (join) {
        if (!dim_types || n_dim_cols < 1 || n_dim_cols > 32 || (n_dim && !dim_cols))
            return fail(TP_E_INVALID, "tp_execute_noalloc: bad dimension columns");
        for (int c = 0; c < n_dim_cols; ++c)
            if (tp::type_size(dim_types[c]) == 0 || (n_dim && !dim_cols[c]))
                return fail(TP_E_INVALID, "tp_execute_noalloc: dimension column %d: bad type or NULL", c);
        if (!col_ok(d->join.fact_col, n_fact_cols) || !col_ok(d->join.dim_col, n_dim_cols))
            return fail(TP_E_INVALID, "tp_execute_noalloc: bad join columns");
    }
    if (d->filter.col != -1 && !col_ok(d->filter.col, n_fact_cols))
        return fail(TP_E_INVALID, "tp_execute_noalloc: bad filter column");
    if (d->dim_filter_on && (!join || !col_ok(d->dim_filter.col, n_dim_cols)))
        return fail(TP_E_INVALID, "tp_execute_noalloc: bad dimension predicate column");
    if (d->n_extra_dims != 0) return fail(TP_E_INVALID, "tp_execute_noalloc: one dimension at most");
    if (d->join_many) return fail(TP_E_INVALID, "tp_execute_noalloc: no fan-out joins");
    if (d->n_group < 0 || d->n_group > 4 || d->n_agg < 1 || d->n_agg > 8)
        return fail(TP_E_INVALID, "tp_execute_noalloc: 0..4 group fields and 1..8 aggregates");
    tpk::QueryDev q{};
    tpk::BuildDev b{};
    if (d->dim_filter_on) {   // only admitted dimension rows are inserted
        b.has_filter = 1;
        b.flo = d->dim_filter.lo;
        b.fhi = d->dim_filter.hi;
        if (n_dim) b.fcol = dcol(dim_cols, dim_types, d->dim_filter.col);
    }
    int key_bits = 0, dim_bits = 0, nf = 0;
    for (int g = 0; g < d->n_group; ++g) {
        const tp_group_field& gf = d->group[g];
        if (gf.bits < 1 || gf.bits > 64) return fail(TP_E_INVALID, "tp_execute_noalloc: bad group width");
        key_bits += gf.bits;
        q.gside[g] = gf.side;
        q.gbits[g] = gf.bits;
        if (gf.side == TP_SIDE_FACT) {
            if (!col_ok(gf.col, n_fact_cols)) return fail(TP_E_INVALID, "tp_execute_noalloc: bad group column");
            if (n_fact) q.gcol[g] = dcol(fact_cols, fact_types, gf.col);
        } else if (gf.side == TP_SIDE_DIM && join && col_ok(gf.col, n_dim_cols)) {
            q.gdpos[g] = dim_bits;
            b.dbits[nf] = gf.bits;
            b.dpos[nf] = dim_bits;
            if (n_dim) b.dcol[nf] = dcol(dim_cols, dim_types, gf.col);
            ++nf;
            dim_bits += gf.bits;
        } else {
            return fail(TP_E_INVALID, "tp_execute_noalloc: bad dimension group field");
        }
    }
    // limits of the fixed scratch array
    if (key_bits > 12)
        return fail(TP_E_INVALID, "tp_execute_noalloc: group key of %d bits; at most 12 bits (4096 groups) fit the "
                    "fixed scratch", key_bits);
    if (dim_bits > tpk::MAX_DIM_BITS) return fail(TP_E_INVALID, "tp_execute_noalloc: dimension fields over 31 bits");
    int ns = 0;
    int sum_of_agg[8];
    for (int a = 0; a < d->n_agg; ++a) {
        const tp_agg& ag = d->aggs[a];
        sum_of_agg[a] = -1;
        if (ag.kind == TP_AGG_COUNT) continue;
        if (ag.kind != TP_AGG_SUM && ag.kind != TP_AGG_AVG && ag.kind != TP_AGG_SUM_MUL_SUB)
            return fail(TP_E_INVALID, "tp_execute_noalloc: bad aggregate kind");
        if (!col_ok(ag.col_a, n_fact_cols) || (ag.kind == TP_AGG_SUM_MUL_SUB && !col_ok(ag.col_b, n_fact_cols)))
            return fail(TP_E_INVALID, "tp_execute_noalloc: bad aggregate column");
        if (!sums || !sums[a] || (ag.kind == TP_AGG_AVG && (!avgs || !avgs[a])))
            return fail(TP_E_INVALID, "tp_execute_noalloc: missing output array for aggregate %d", a);
        sum_of_agg[a] = ns;
        if (n_fact) q.sa[ns] = dcol(fact_cols, fact_types, ag.col_a);
        if (ag.kind == TP_AGG_SUM_MUL_SUB) {
            q.skind[ns] = tpk::S_MUL_SUB;
            if (n_fact) q.sb[ns] = dcol(fact_cols, fact_types, ag.col_b);
            q.sk[ns] = ag.k;
        }
        ++ns;
    }
    const float lf = d->load_factor > 0 ? d->load_factor : 0.5f;
    if (!(lf > 0.05f && lf <= 0.9f)) return fail(TP_E_INVALID, "tp_execute_noalloc: bad load factor");
    const bool key64 = join && dim_types[d->join.dim_col] == TP_I64;
    const uint64_t slot_bytes = key64 ? 16 : 8;
    uint64_t want = (uint64_t)std::ceil(n_dim / lf);
    if (want < 64) want = 64;
    const uint64_t join_cap = join ? pow2_ge(want) : 0;
    if (join_cap * slot_bytes > NOLOC_JOIN_BYTES)
        return fail(TP_E_INVALID, "tp_execute_noalloc: %llu dimension rows need a %llu-slot join table; the fixed "
                    "scratch holds %llu slots", (unsigned long long)n_dim, (unsigned long long)join_cap,
                    (unsigned long long)(NOLOC_JOIN_BYTES / slot_bytes));

    void* base = nullptr;
    tp_status s = noloc_scratch(&base);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    TP_TRY_CUDA(cudaGetDevice(&dev));
    TP_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    unsigned char* misc = (unsigned char*)base;
    uint32_t* err = (uint32_t*)misc;
    unsigned long long* groups_dev = (unsigned long long*)(misc + 64);
    uint64_t* gacc = (uint64_t*)(misc + NOLOC_MISC_BYTES);
    uint64_t* jslots = (uint64_t*)(misc + NOLOC_MISC_BYTES + NOLOC_ACC_BYTES);
    const uint32_t G = 1u << key_bits;
    // the array keeps the previous call's contents: clear what starts at zero
    TP_TRY_CUDA(cudaMemsetAsync(misc, 0, NOLOC_MISC_BYTES, st));
    TP_TRY_CUDA(cudaMemsetAsync(gacc, 0, (uint64_t)G * (1 + 2 * ns) * 8, st));
    if (join) {
        TP_TRY_CUDA(cudaMemsetAsync(jslots, 0xFF, join_cap * slot_bytes, st));
        q.jt.slots = jslots;
        q.jt.mask = join_cap - 1;
        q.jt.side = (uint32_t*)(misc + 128);
        q.jt.key64 = key64 ? 1 : 0;
        b.jt = q.jt;
        b.err = err;
        b.n_dfield = nf;
        if (n_dim) {
            b.key = dcol(dim_cols, dim_types, d->join.dim_col);
            TP_TRY_CUDA(tpk::launch_build(b, n_dim, sms, st));
        }
    }
    q.has_filter = d->filter.col >= 0;
    if (q.has_filter && n_fact) {
        q.fcol = dcol(fact_cols, fact_types, d->filter.col);
        q.flo = d->filter.lo;
        q.fhi = d->filter.hi;
    }
    q.has_join = join ? 1 : 0;
    if (join && n_fact) q.fk = dcol(fact_cols, fact_types, d->join.fact_col);
    q.n_group = d->n_group;
    q.n_sum = ns;
    q.eager = 1;
    q.err = err;
    if (n_fact) {
        const int grid = tpk::agg_shared_grid(key_bits, ns, sms);
        TP_TRY_CUDA(tpk::launch_agg_shared(q, n_fact, gacc, key_bits, grid, st));
    }
    tpk::OutDev od{};
    od.keys = keys;
    od.counts = counts;
    for (int a = 0; a < d->n_agg; ++a) {
        const int si = sum_of_agg[a];
        if (si < 0) continue;
        od.sums[si] = (uint64_t*)sums[a];
        if (d->aggs[a].kind == TP_AGG_AVG) {
            od.avgs[si] = avgs[a];
            od.has_avg[si] = 1;
        }
    }
    od.n_groups = groups_dev;
    TP_TRY_CUDA(tpk::launch_final_dense(gacc, key_bits, ns, od, st));
    uint64_t words[2] = {0, 0};
    TP_TRY_CUDA(cudaMemcpyAsync(&words[0], err, 4, cudaMemcpyDeviceToHost, st));
    TP_TRY_CUDA(cudaMemcpyAsync(&words[1], groups_dev, 8, cudaMemcpyDeviceToHost, st));
    TP_TRY_CUDA(cudaStreamSynchronize(st));
    const uint32_t e = (uint32_t)words[0];
    if (e & tpk::ERR_DUP) return fail(TP_E_DUP_KEY, "join build side holds a duplicate key");
    if (e & tpk::ERR_RANGE) return fail(TP_E_RANGE, "a group field value does not fit its bit width");
    if (e & tpk::ERR_INTERNAL) return fail(TP_E_INTERNAL, "device consistency check failed");
    *n_groups = words[1];
    return TP_OK;
}
