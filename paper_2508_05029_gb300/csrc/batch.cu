// Batched execution: many queries in one persistent kernel, one CUDA graph.
//
// Paper basis: Section 3.1 (operators spawn tasks over batches; tasks run on
// the GPU asynchronously), Section 3.3.1 (the Compute Executor drains a task
// queue).  Here the queue lives on the device: the host lays out every task of
// every query -- build chunks first, then probe tiles, then one finalisation
// per query -- and resident CTAs claim them in order with one atomic counter.
// A probe tile of query q waits until all of q's build chunks are done, a
// finalisation until all of q's probe tiles are done.  Every waited-on task
// has a smaller index, so it was claimed earlier by a CTA that is running and
// never waits on a later task: the queue cannot deadlock.  Waits are bounded
// by wait_ns of %globaltimer; on expiry the CTA records ERR_TIMEOUT and drops
// the task, so the host reports TP_E_TIMEOUT instead of hanging.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <string>

#include "tp_internal.h"
#include "device.cuh"

namespace tpk {

__device__ __forceinline__ uint64_t batch_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0 waits until *ctr reaches want; the CTA learns the outcome.
__device__ __forceinline__ bool cta_wait_count(unsigned* ctr, unsigned want, uint64_t wait_ns, uint32_t* err,
                                               int* flag) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint64_t t0 = batch_ns();
        while (*(volatile unsigned*)ctr < want) {
            if (batch_ns() - t0 > wait_ns) {
                atomicOr(err, ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(256);
        }
        __threadfence();
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

// Probe tile [r0, r1) of one query: warp tiles of 128 rows, plain loads; the
// join table was written earlier in this launch, so it is read at L2.
__device__ void batch_probe(const BatchQuery& B, uint64_t r0, uint64_t r1, unsigned char* smem) {
    const QueryDev& q = B.q;
    const uint32_t G = 1u << B.key_bits;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t* cnt = (uint32_t*)smem;
    if (B.smem) {
        uint32_t words = 1;
        for (int s = 0; s < q.n_sum; ++s) words += (uint32_t)B.sum_mode[s];
        for (uint32_t i = threadIdx.x; i < words * G; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
    }
    for (uint64_t t0 = r0 + (uint64_t)warp * 128; t0 < r1; t0 += (uint64_t)nwarps * 128) {
        bool pass[4];
        uint64_t key[4];
        const bool full = t0 + 128 <= r1;
        const bool any = full ? eval_keys<true, false>(q, t0, r1, lane, pass, key)
                              : eval_keys<false, false>(q, t0, r1, lane, pass, key);
        if (!any) continue;
        uint32_t g[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            g[i] = (uint32_t)key[i];
            if (!pass[i]) continue;
            if (B.smem) atomicAdd(&cnt[g[i]], 1u);
            else atomicAdd((unsigned long long*)&B.acc[g[i]], 1ull);
        }
        uint32_t word = 1;
        for (int s = 0; s < q.n_sum; ++s) {
            I128 tm[4];
            if (full) eval_terms<true>(q, s, t0, r1, lane, pass, tm);
            else eval_terms<false>(q, s, t0, r1, lane, pass, tm);
            if (B.smem) {
                uint32_t* lo = cnt + (uint64_t)word * G;
                const int64_t off = B.sum_off[s];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (!pass[i]) continue;
                    const uint64_t t = (uint64_t)((int64_t)tm[i].lo - off);
                    const uint32_t old = atomicAdd(lo + g[i], (uint32_t)t);
                    if (B.sum_mode[s] == 2) {
                        const uint32_t h = (uint32_t)(t >> 32) + ((old + (uint32_t)t) < old ? 1u : 0u);
                        if (h) atomicAdd(lo + G + g[i], h);
                    }
                }
                word += (uint32_t)B.sum_mode[s];
            } else {
                uint64_t* lo = B.acc + (uint64_t)G * (1 + 2 * s);
                uint64_t* hi = B.acc + (uint64_t)G * (2 + 2 * s);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (!pass[i]) continue;
                    if (B.fast) atomicAdd((unsigned long long*)(lo + g[i]), (unsigned long long)tm[i].lo);
                    else atomic_add_i128(lo + g[i], hi + g[i], tm[i]);
                }
            }
        }
    }
    if (B.smem) {
        __syncthreads();
        for (uint32_t gi = threadIdx.x; gi < G; gi += blockDim.x) {
            const uint64_t c = cnt[gi];
            if (!c) continue;
            atomicAdd((unsigned long long*)&B.acc[gi], (unsigned long long)c);
            uint32_t word = 1;
            for (int s = 0; s < q.n_sum; ++s) {
                const uint32_t* w = cnt + (uint64_t)word * G;
                uint64_t v = w[gi];
                if (B.sum_mode[s] == 2) v += (uint64_t)w[G + gi] << 32;
                v += c * (uint64_t)B.sum_off[s];
                atomicAdd((unsigned long long*)&B.acc[(uint64_t)G * (1 + 2 * s) + gi], (unsigned long long)v);
                word += (uint32_t)B.sum_mode[s];
            }
        }
    }
}

__global__ void __launch_bounds__(BATCH_THREADS) k_batch(const BatchQuery* __restrict__ qs,
                                                        const BatchItem* __restrict__ items, uint32_t n_items,
                                                        uint32_t n_q, unsigned* ctr, uint32_t* err,
                                                        const uint64_t* __restrict__ wait) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint64_t wait_ns = *wait;   // device word, so a captured graph can be given another limit
    __shared__ uint32_t cur;
    __shared__ int flag;
    __shared__ uint64_t first_row;
    unsigned* build_done = ctr + 1;
    unsigned* probe_done = ctr + 1 + n_q;
    for (;;) {
        if (threadIdx.x == 0) cur = atomicAdd(ctr, 1u);
        __syncthreads();
        const uint32_t i = cur;
        __syncthreads();
        if (i >= n_items) return;
        const BatchItem it = items[i];
        const BatchQuery& B = qs[it.q];
        const uint64_t t_claim = B.task_ns ? batch_ns() : 0;
        if (it.kind == BI_BUILD) {
            for (uint64_t r = it.r0 + threadIdx.x; r < it.r1; r += blockDim.x) build_insert(B.b, r);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&build_done[it.q], 1u);
            }
        } else if (it.kind == BI_PROBE) {
            if (B.q.has_join && !cta_wait_count(&build_done[it.q], B.build_items, wait_ns, err, &flag)) continue;
            batch_probe(B, it.r0, it.r1, smem);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&probe_done[it.q], 1u);
            }
        } else {
            if (!cta_wait_count(&probe_done[it.q], B.probe_items, wait_ns, err, &flag)) continue;
            // groups [r0, r1): count them, wait for the ranges before to publish
            // where their rows end, publish this range's end, write the rows
            const uint32_t G = 1u << B.key_bits;
            const uint32_t g0 = (uint32_t)it.r0, g1 = (uint32_t)it.r1, k = g0 / FINAL_CHUNK;
            const uint32_t cnt = dense_range_count(B.acc, g0, g1);
            if (!cta_wait_count(B.final_done, k, wait_ns, err, &flag)) continue;
            if (threadIdx.x == 0) {
                const uint64_t first = k ? *(volatile unsigned long long*)B.final_end : 0ull;
                first_row = first;
                *(volatile unsigned long long*)B.final_end = first + cnt;
                __threadfence();
                atomicAdd(B.final_done, 1u);
                if (g1 == G) *B.out.n_groups = first + cnt;
            }
            __syncthreads();
            dense_range_emit(B.acc, G, g0, g1, B.q.n_sum, B.out, B.fast != 0, first_row);
        }
        __syncthreads();
        if (B.task_ns && threadIdx.x == 0) atomicAdd(B.task_ns, (unsigned long long)(batch_ns() - t_claim));
    }
}

int batch_grid(uint32_t smem_bytes, int num_sms) {
    ensure_smem_limit((const void*)k_batch, (int)smem_bytes);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, BATCH_THREADS, smem_bytes) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return per_sm * num_sms;
}

cudaError_t launch_batch(const BatchQuery* qs, const BatchItem* items, uint32_t n_items, uint32_t n_q,
                         unsigned* ctr, uint32_t* err, const uint64_t* wait_ns, uint32_t smem_bytes, int grid,
                         cudaStream_t st) {
    k_batch<<<grid, BATCH_THREADS, smem_bytes, st>>>(qs, items, n_items, n_q, ctr, err, wait_ns);
    return cudaGetLastError();
}

}  // namespace tpk

// ===================================================================== host

namespace {

using namespace tp;

#ifndef TP_BATCH_SMEM_MAX
#define TP_BATCH_SMEM_MAX (96 * 1024)
#endif
#ifndef TP_BATCH_SMEM_BITS
#define TP_BATCH_SMEM_BITS 12
#endif
// queries whose 32-bit group table fits this many bytes of shared memory
// (and keys of at most SMEM_TABLE_BITS bits) accumulate per tile in shared
// memory; the others add straight into device memory
constexpr uint32_t SMEM_TABLE_MAX = TP_BATCH_SMEM_MAX;
constexpr int SMEM_TABLE_BITS = TP_BATCH_SMEM_BITS;

struct Tune {
    float lf;              // join load factor (0: the plan's)
    uint32_t rows_per_warp;
    int agg;               // TP_AGG_AUTO / SHARED / GLOBAL
};

int ilog2(uint64_t x) {
    int b = 0;
    while (x > 1) {
        x >>= 1;
        ++b;
    }
    return b;
}

// Query class: buckets of fact size, group-key width and dimension size.
int query_class(const tp_plan* p) {
    const uint64_t nf = p->d.fact->rows;
    const uint64_t nd = p->d.join.fact_col >= 0 ? p->d.dim->rows : 0;
    return (ilog2(nf + 1) / 2) * 10000 + (p->key_bits / 4) * 100 + ilog2(nd + 1) / 2;
}

std::map<int, Tune> load_tuning(const char* path) {
    std::map<int, Tune> t;
    if (!path) return t;
    FILE* f = fopen(path, "r");
    if (!f) return t;
    char line[256];
    while (fgets(line, sizeof(line), f)) {
        int cls, agg;
        float lf;
        unsigned rpw;
        if (line[0] == '#') continue;
        if (sscanf(line, "%d %f %u %d", &cls, &lf, &rpw, &agg) == 4) t[cls] = Tune{lf, rpw, agg};
    }
    fclose(f);
    return t;
}

Tune tune_for(const std::map<int, Tune>& t, const tp_plan* p) {
    auto it = t.find(query_class(p));
    if (it != t.end()) return it->second;
    return Tune{0.0f, 1024, TP_AGG_AUTO};
}

uint64_t a256(uint64_t x) { return (x + 255) & ~255ull; }

uint64_t p2(uint64_t x) {
    uint64_t r = 1;
    while (r < x) r <<= 1;
    return r;
}

}  // namespace

struct tp_batch {
    tp_engine* e = nullptr;
    std::vector<tp_plan*> plans;
    void* dev = nullptr;
    uint64_t reserved = 0;
    tpk::BatchQuery* d_q = nullptr;
    tpk::BatchItem* d_items = nullptr;
    uint32_t n_items = 0;
    unsigned* d_ctr = nullptr;
    uint32_t* d_err = nullptr;
    unsigned long long* d_groups = nullptr;
    unsigned long long* d_task_ns = nullptr;   // per query: CTA nanoseconds of its tasks (last run)
    unsigned char* ff_base = nullptr;
    uint64_t ff_bytes = 0;
    unsigned char* zero_base = nullptr;
    uint64_t zero_bytes = 0;
    uint32_t smem = 0;
    int grid = 0;
    uint64_t* d_wait = nullptr;          // limit of every dependency wait, ns (device word)
    bool jit = false;                    // the run-time compiled kernel runs the queue
    std::vector<uint32_t> probe_items;   // per query, as laid out (tp_debug_batch_stall restores it)
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double last_ms = 0;
    std::vector<tpk::OutDev> outs;
};

static constexpr uint64_t BATCH_WAIT_NS = 2000000000ull;   // 2 s

// Resident CTAs of the run-time compiled queue kernel: every SM, as many as fit.
static int jit_batch_grid(const void* k, uint32_t smem_bytes, int num_sms) {
    tpk::ensure_smem_limit(k, (int)smem_bytes);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, tpk::BATCH_THREADS, smem_bytes) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * num_sms;
}

static void batch_free(tp_batch* b) {
    if (!b) return;
    tp_engine* e = b->e;
    cudaSetDevice(e->device);
    cudaStreamSynchronize(e->compute);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->dev) dev_free(e, b->dev, e->compute);
    cudaStreamSynchronize(e->compute);
    if (b->reserved) release(e, b->reserved);
    delete b;
}

namespace tp {

tp_status batch_check_plan(const tp_engine* e, const tp_plan* p, int i) {
    if (!p || p->eng != e) return fail(TP_E_INVALID, "plan %d missing or from another engine", i);
    if (p->d.fact->placement == PL_PAGES || (p->d.join.fact_col >= 0 && p->d.dim->placement == PL_PAGES))
        return fail(TP_E_INVALID, "plan %d reads a table in host pages", i);
    if (p->n_dims > 1) return fail(TP_E_INVALID, "plan %d is a star join (one dimension here)", i);
    if (p->d.join_many) return fail(TP_E_INVALID, "plan %d has a fan-out join", i);
    if (p->key_bits > 20) return fail(TP_E_INVALID, "plan %d has a %d-bit group key (at most 20)", i, p->key_bits);
    return TP_OK;
}

void batch_prep(const tp_engine* e, const tp_plan* p, float lf_tuned, uint32_t rows_per_warp, int agg,
                BatchPrep* out) {
    BatchPrep& x = *out;
    x = BatchPrep{};
    const float lf = lf_tuned > 0 ? lf_tuned : p->load_factor;
    x.join = p->d.join.fact_col >= 0;
    x.key64 = x.join && p->d.dim->types[p->d.join.dim_col] == TP_I64;
    x.direct = x.join && !(e->cfg.flags & TP_FLAG_NO_DIRECT_JOIN) && direct_join_range(p->d.dim, p->d.join.dim_col,
                                                                                        &x.range);
    x.join_cap = x.join && !x.direct ? p2(std::max<uint64_t>(64, (uint64_t)std::ceil(p->d.dim->rows / lf))) : 0;
    x.join_bytes = x.direct ? a256(x.range * 4) : a256(x.join_cap * (x.key64 ? 16 : 8));
    const uint64_t G = 1ull << p->key_bits;
    x.acc_bytes = a256(G * 8 * (1 + 2 * (uint64_t)p->n_sum));
    int n_avg = 0;
    for (int a = 0; a < p->d.n_agg; ++a) n_avg += p->d.aggs[a].kind == TP_AGG_AVG;
    x.out_bytes = a256(G * 8) * 2 + a256(G * 16) * p->n_sum + a256(G * 8) * n_avg;
    x.tile = (uint64_t)std::min<uint32_t>(std::max<uint32_t>(rows_per_warp, 128), 1u << 16) / 128 * 128 *
             (tpk::BATCH_THREADS / 32);
    x.fast = !(e->cfg.flags & TP_FLAG_EXACT_ONLY) && sums_fit_int64(p, p->d.fact);
    // shared-memory tables: 32-bit words, per tile; needs 64-bit safety
    if (x.fast && agg != TP_AGG_GLOBAL && p->key_bits <= SMEM_TABLE_BITS) {
        term_bounds(p, p->d.fact, x.bounds);
        uint32_t words = 1;
        bool ok = true;
        for (int s = 0; s < p->n_sum; ++s) {
            const unsigned __int128 r = x.tile;
            if (r * x.bounds[s].span <= 0xFFFFFFFFull) x.mode[s] = 1;
            else if (r * ((x.bounds[s].span >> 32) + 1) <= 0xFFFFFFFFull) x.mode[s] = 2;
            else ok = false;
            words += ok ? (uint32_t)x.mode[s] : 0;
        }
        const uint64_t bytes = 4 * G * words;
        if (ok && bytes <= SMEM_TABLE_MAX) {
            x.smem = true;
            x.smem_bytes = (uint32_t)bytes;
        }
    }
    if (!x.smem)
        for (int s = 0; s < tpk::MAX_SUM; ++s) x.mode[s] = 0;
    x.build_items = x.join ? (p->d.dim->rows + BATCH_BUILD_CHUNK - 1) / BATCH_BUILD_CHUNK : 0;
    x.probe_items = (p->d.fact->rows + x.tile - 1) / x.tile;
    x.final_items = (G + tpk::FINAL_CHUNK - 1) / tpk::FINAL_CHUNK;
}

void batch_query_desc(const tp_plan* p, const BatchPrep& x, void* join_slots, uint32_t* side, uint64_t* acc,
                      uint32_t* err, const tpk::OutDev& out, tpk::BatchQuery* Bp, unsigned* final_done,
                      unsigned long long* final_end) {
    const tp_plan_desc& d = p->d;
    tpk::BatchQuery& B = *Bp;
    memset(&B, 0, sizeof(B));
    tpk::JoinTable jt{};
    if (x.join) {
        jt.slots = (uint64_t*)join_slots;
        jt.mask = x.join_cap ? x.join_cap - 1 : 0;
        jt.key64 = x.key64 ? 1 : 0;
        jt.side = side;
        jt.direct = x.direct ? 1 : 0;
        jt.kmin = x.direct ? d.dim->cmin[d.join.dim_col] : 0;
        jt.range = x.direct ? x.range : 0;
    }
    std::vector<const void*> colptr(d.fact->types.size(), nullptr);
    for (size_t c = 0; c < colptr.size(); ++c) colptr[c] = d.fact->dev_cols[c];
    B.q = plan_query_dev(p, colptr, jt, err, true);
    B.acc = acc;
    B.key_bits = (uint32_t)p->key_bits;
    B.smem = x.smem ? 1 : 0;
    B.fast = x.fast ? 1 : 0;
    for (int t = 0; t < p->n_sum; ++t) {
        B.sum_mode[t] = x.smem ? x.mode[t] : 0;
        B.sum_off[t] = x.smem ? x.bounds[t].lo : 0;
    }
    if (x.join) {
        B.b.key.ptr = d.dim->dev_cols[d.join.dim_col];
        B.b.key.type = d.dim->types[d.join.dim_col];
        int nf = 0;
        for (int g = 0; g < d.n_group; ++g) {
            if (d.group[g].side != TP_SIDE_DIM) continue;
            B.b.dcol[nf].ptr = d.dim->dev_cols[d.group[g].col];
            B.b.dcol[nf].type = d.dim->types[d.group[g].col];
            B.b.dbits[nf] = d.group[g].bits;
            B.b.dpos[nf] = p->gdpos[g];
            ++nf;
        }
        B.b.n_dfield = nf;
        B.b.jt = jt;
        B.b.err = err;
        if (d.dim_filter.col >= 0) {   // the dimension predicate gates the build
            B.b.has_filter = 1;
            B.b.fcol.ptr = d.dim->dev_cols[d.dim_filter.col];
            B.b.fcol.type = d.dim->types[d.dim_filter.col];
            B.b.flo = d.dim_filter.lo;
            B.b.fhi = d.dim_filter.hi;
        }
    }
    B.out = out;
    B.build_items = (uint32_t)x.build_items;
    B.probe_items = (uint32_t)x.probe_items;
    B.final_done = final_done;
    B.final_end = final_end;
}

void batch_items(const tp_plan* p, const BatchPrep& x, uint32_t qi, int kind, std::vector<tpk::BatchItem>* items) {
    if (kind == tpk::BI_BUILD) {
        for (uint64_t k = 0; k < x.build_items; ++k)
            items->push_back(tpk::BatchItem{qi, tpk::BI_BUILD, k * BATCH_BUILD_CHUNK,
                                            std::min<uint64_t>(p->d.dim->rows, (k + 1) * BATCH_BUILD_CHUNK), 0});
    } else if (kind == tpk::BI_PROBE) {
        const uint64_t rows = p->d.fact->rows;
        for (uint64_t k = 0; k < x.probe_items; ++k)
            items->push_back(tpk::BatchItem{qi, tpk::BI_PROBE, k * x.tile, std::min(rows, (k + 1) * x.tile), 0});
    } else {
        const uint64_t G = 1ull << p->key_bits;
        for (uint64_t k = 0; k < x.final_items; ++k)
            items->push_back(tpk::BatchItem{qi, tpk::BI_FINAL, k * tpk::FINAL_CHUNK,
                                            std::min<uint64_t>(G, (k + 1) * tpk::FINAL_CHUNK), 0});
    }
}

std::string batch_shape(const tp_plan* p, const tpk::BatchQuery& B, const BatchPrep& x, const std::string& name) {
    int narrow[tpk::MAX_SUM] = {};
    narrow_products(p, p->d.fact, narrow);
    return shape_struct(name, B.q, x.mode, x.smem, x.fast, narrow);
}

std::string batch_kernel_source(const std::vector<std::string>& shapes) {
    std::string src;
    for (size_t k = 0; k < shapes.size(); ++k) src += shapes[k];
    src += "#include \"jit_batch.cuh\"\n"
           "__device__ void tpj::dispatch_probe(const tpk::BatchQuery& B, uint64_t r0, uint64_t r1, "
           "unsigned char* smem) {\n    switch (B.shape) {\n";
    for (size_t k = 0; k < shapes.size(); ++k)
        src += "    case " + std::to_string(k) + ": probe_tile<JS_" + std::to_string(k) + ">(B, r0, r1, smem); break;\n";
    src += "    default: break;\n    }\n}\n";
    return src;
}

int batch_kernel_grid(const void* jit_kernel_or_null, uint32_t smem_bytes, int num_sms) {
    return jit_kernel_or_null ? jit_batch_grid(jit_kernel_or_null, smem_bytes, num_sms)
                              : tpk::batch_grid(smem_bytes, num_sms);
}

}  // namespace tp

static tp_status batch_create_impl(tp_engine* e, tp_plan* const* plans, int32_t n, const std::map<int, Tune>& tune,
                                   tp_batch** out) {
    if (!e || !plans || n < 1 || !out) return fail(TP_E_INVALID, "tp_batch_create: bad arguments");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        tp_status s = batch_check_plan(e, plans[i], i);
        if (s) {
            const std::string why = tp_last_error();
            return fail(s, "tp_batch_create: %s", why.c_str());
        }
    }
    TP_TRY_CUDA(cudaSetDevice(e->device));
    std::unique_ptr<tp_batch, void (*)(tp_batch*)> b(new (std::nothrow) tp_batch(), batch_free);
    if (!b) return fail(TP_E_NOMEM, "tp_batch_create: out of host memory");
    b->e = e;
    b->plans.assign(plans, plans + n);
    // ---- per query sizes and choices
    std::vector<BatchPrep> qs(n);
    // zeroed every run: counters, error word, group counts, join side cells, accumulators
    uint64_t ff = 0, zero = a256((1 + 2 * (uint64_t)n) * 4) + 256 + a256(8 * (uint64_t)n) * 5, outb = 0;
    uint32_t smem_max = 16;
    uint64_t n_items = 0;
    for (int i = 0; i < n; ++i) {
        const Tune t = tune_for(tune, plans[i]);
        BatchPrep& x = qs[i];
        batch_prep(e, plans[i], t.lf, t.rows_per_warp, t.agg, &x);
        if (x.smem) smem_max = std::max(smem_max, x.smem_bytes);
        ff += x.join_bytes;
        zero += x.acc_bytes;
        outb += x.out_bytes;
        n_items += x.build_items + x.probe_items + x.final_items;
    }
    if (n_items >= (1ull << 32)) return fail(TP_E_INVALID, "tp_batch_create: too many tasks");
    const uint64_t qbytes = a256(sizeof(tpk::BatchQuery) * n);
    const uint64_t ibytes = a256(sizeof(tpk::BatchItem) * n_items);
    const uint64_t total = ff + zero + qbytes + ibytes + outb + 256;   // + the wait-limit word
    tp_status s = reserve(e, total);
    if (s) return s;
    b->reserved = total;
    if ((s = dev_alloc(e, &b->dev, total, e->compute))) return s;
    unsigned char* base = (unsigned char*)b->dev;
    b->ff_base = base;
    b->ff_bytes = ff;
    b->zero_base = base + ff;
    b->zero_bytes = zero;
    unsigned char* zp = b->zero_base;
    b->d_ctr = (unsigned*)zp;
    zp += a256((1 + 2 * (uint64_t)n) * 4);
    b->d_err = (uint32_t*)zp;
    zp += 256;
    b->d_groups = (unsigned long long*)zp;
    zp += a256(8 * (uint64_t)n);
    uint32_t* sides = (uint32_t*)zp;   // two words per query: present flag, payload
    zp += a256(8 * (uint64_t)n);
    b->d_task_ns = (unsigned long long*)zp;
    zp += a256(8 * (uint64_t)n);
    unsigned* final_done = (unsigned*)zp;
    zp += a256(8 * (uint64_t)n);
    unsigned long long* final_end = (unsigned long long*)zp;
    zp += a256(8 * (uint64_t)n);
    unsigned char* accp = zp;
    unsigned char* qp = b->zero_base + zero;
    b->d_q = (tpk::BatchQuery*)qp;
    b->d_items = (tpk::BatchItem*)(qp + qbytes);
    unsigned char* op = qp + qbytes + ibytes;
    b->d_wait = (uint64_t*)(base + total - 256);
    // ---- descriptors and tasks on the host: every query's build chunks,
    // then every query's probe tiles, then one finalisation per query
    std::vector<tpk::BatchQuery> hq(n);
    std::vector<tpk::BatchItem> items;
    items.reserve(n_items);
    unsigned char* jp = b->ff_base;
    b->outs.resize(n);
    for (int i = 0; i < n; ++i) {
        const tp_plan* p = plans[i];
        const BatchPrep& x = qs[i];
        // outputs
        const uint64_t G = 1ull << p->key_bits;
        tpk::OutDev& o = b->outs[i];
        memset(&o, 0, sizeof(o));
        o.keys = (uint64_t*)op;
        op += a256(G * 8);
        o.counts = (int64_t*)op;
        op += a256(G * 8);
        for (int t = 0; t < p->n_sum; ++t) {
            o.sums[t] = (uint64_t*)op;
            op += a256(G * 16);
        }
        for (int a = 0; a < p->d.n_agg; ++a) {
            if (p->d.aggs[a].kind != TP_AGG_AVG) continue;
            const int t = p->sum_of_agg[a];
            o.avgs[t] = (double*)op;
            o.has_avg[t] = 1;
            op += a256(G * 8);
        }
        o.n_groups = b->d_groups + i;
        batch_query_desc(p, x, jp, sides + 2 * i, (uint64_t*)accp, b->d_err, o, &hq[i], final_done + 2 * i,
                         final_end + i);
        hq[i].task_ns = b->d_task_ns + i;
        jp += x.join_bytes;
        accp += x.acc_bytes;
        batch_items(p, x, (uint32_t)i, tpk::BI_BUILD, &items);
    }
    for (int i = 0; i < n; ++i) batch_items(plans[i], qs[i], (uint32_t)i, tpk::BI_PROBE, &items);
    for (int i = 0; i < n; ++i) batch_items(plans[i], qs[i], (uint32_t)i, tpk::BI_FINAL, &items);
    b->n_items = (uint32_t)items.size();
    // run-time compiled probe tasks: one shape struct per distinct query shape
    const void* jk = nullptr;
    if (!(e->cfg.flags & TP_FLAG_NO_JIT)) {
        std::map<std::string, int> ids;
        std::vector<std::string> shapes;
        for (int i = 0; i < n; ++i) {
            const std::string key = batch_shape(plans[i], hq[i], qs[i], "JS_");
            auto it = ids.find(key);
            if (it == ids.end()) {
                const int id = (int)ids.size();
                it = ids.emplace(key, id).first;
                shapes.push_back(batch_shape(plans[i], hq[i], qs[i], "JS_" + std::to_string(id)));
            }
            hq[i].shape = it->second;
        }
        std::string why;
        jk = jit_kernel(e, batch_kernel_source(shapes), "tpj_batch", &why);
    }
    b->jit = jk != nullptr;
    b->probe_items.resize(n);
    for (int i = 0; i < n; ++i) b->probe_items[i] = hq[i].probe_items;
    TP_TRY_CUDA(cudaMemcpyAsync(b->d_wait, &BATCH_WAIT_NS, 8, cudaMemcpyHostToDevice, e->compute));
    TP_TRY_CUDA(cudaMemcpyAsync(b->d_q, hq.data(), sizeof(tpk::BatchQuery) * n, cudaMemcpyHostToDevice, e->compute));
    TP_TRY_CUDA(cudaMemcpyAsync(b->d_items, items.data(), sizeof(tpk::BatchItem) * items.size(),
                                cudaMemcpyHostToDevice, e->compute));
    TP_TRY_CUDA(cudaStreamSynchronize(e->compute));
    b->smem = smem_max;
    b->grid = batch_kernel_grid(jk, b->smem, e->num_sms);
    // ---- capture: reset tables and counters, run the queue
    cudaGraph_t graph = nullptr;
    TP_TRY_CUDA(cudaStreamBeginCapture(e->compute, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaMemsetAsync(b->ff_base, 0xFF, b->ff_bytes, e->compute);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(b->zero_base, 0, b->zero_bytes, e->compute);
    if (ce == cudaSuccess && jk) {
        const tpk::BatchQuery* a_q = b->d_q;
        const tpk::BatchItem* a_items = b->d_items;
        uint32_t a_n = b->n_items, a_nq = (uint32_t)n;
        unsigned* a_ctr = b->d_ctr;
        uint32_t* a_err = b->d_err;
        const uint64_t* a_wait = b->d_wait;
        void* args[] = {&a_q, &a_items, &a_n, &a_nq, &a_ctr, &a_err, &a_wait};
        ce = cudaLaunchKernel(jk, dim3(b->grid), dim3(tpk::BATCH_THREADS), args, b->smem, e->compute);
    } else if (ce == cudaSuccess) {
        ce = tpk::launch_batch(b->d_q, b->d_items, b->n_items, (uint32_t)n, b->d_ctr, b->d_err, b->d_wait, b->smem,
                               b->grid, e->compute);
    }
    cudaError_t ce2 = cudaStreamEndCapture(e->compute, &graph);
    if (ce != cudaSuccess || ce2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(TP_E_CUDA, "tp_batch_create: graph capture failed: %s",
                    cudaGetErrorString(ce != cudaSuccess ? ce : ce2));
    }
    ce = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(TP_E_CUDA, "tp_batch_create: graph instantiation failed: %s", cudaGetErrorString(ce));
    TP_TRY_CUDA(cudaEventCreate(&b->ev0));
    TP_TRY_CUDA(cudaEventCreate(&b->ev1));
    *out = b.release();
    return TP_OK;
}

static tp_status batch_run(tp_batch* b, std::vector<tp_result*>* results) {
    tp_engine* e = b->e;
    TP_TRY_CUDA(cudaSetDevice(e->device));
    const int n = (int)b->plans.size();
    TP_TRY_CUDA(cudaEventRecord(b->ev0, e->compute));
    TP_TRY_CUDA(cudaGraphLaunch(b->exec, e->compute));
    TP_TRY_CUDA(cudaEventRecord(b->ev1, e->compute));
    e->launches += 1;
    if (b->jit) e->jit_launches++;
    std::vector<unsigned long long> groups(n);
    uint32_t err = 0;
    TP_TRY_CUDA(cudaMemcpyAsync(groups.data(), b->d_groups, 8ull * n, cudaMemcpyDeviceToHost, e->compute));
    TP_TRY_CUDA(cudaMemcpyAsync(&err, b->d_err, 4, cudaMemcpyDeviceToHost, e->compute));
    TP_TRY_CUDA(cudaStreamSynchronize(e->compute));
    float ms = 0;
    cudaEventElapsedTime(&ms, b->ev0, b->ev1);
    b->last_ms = ms;
    e->d2h_bytes += 8ull * n + 4;
    if (err & tpk::ERR_DUP) return fail(TP_E_DUP_KEY, "a join build side holds a duplicate key");
    if (err & tpk::ERR_RANGE) return fail(TP_E_RANGE, "a group field value does not fit its bit width");
    if (err & tpk::ERR_TIMEOUT) return fail(TP_E_TIMEOUT, "a bounded wait of the batch expired");
    if (err & tpk::ERR_INTERNAL) return fail(TP_E_INTERNAL, "device consistency check failed");
    if (!results) return TP_OK;
    results->assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
        const tp_plan* p = b->plans[i];
        tp_result* r = new (std::nothrow) tp_result();
        if (!r) {
            for (tp_result* x : *results) delete x;
            return fail(TP_E_NOMEM, "tp_batch_execute: out of host memory");
        }
        const tpk::OutDev& o = b->outs[i];
        r->eng = e;
        r->n_groups = groups[i];
        r->n_agg = p->d.n_agg;
        r->n_sum = p->n_sum;
        r->d_keys = o.keys;
        r->d_counts = o.counts;
        for (int a = 0; a < p->d.n_agg; ++a) {
            r->sum_of_agg[a] = p->sum_of_agg[a];
            r->is_avg[a] = p->d.aggs[a].kind == TP_AGG_AVG;
        }
        for (int t = 0; t < p->n_sum; ++t) {
            r->d_sums[t] = o.sums[t];
            r->d_avgs[t] = o.avgs[t];
        }
        r->have_sum.assign(8, false);
        r->have_avg.assign(8, false);
        r->h_sums.resize(8);
        r->h_avgs.resize(8);
        (*results)[i] = r;
    }
    return TP_OK;
}

extern "C" {

tp_status tp_batch_create(tp_engine* e, tp_plan* const* plans, int32_t n, const char* tuning_path,
                          tp_batch** out) {
    clear_error();
    if (!e) return fail(TP_E_INVALID, "tp_batch_create: NULL engine");
    std::lock_guard<std::mutex> lk(e->exec_mu);
    return batch_create_impl(e, plans, n, load_tuning(tuning_path), out);
}

tp_status tp_batch_execute(tp_batch* b, tp_result** results) {
    clear_error();
    if (!b || !results) return fail(TP_E_INVALID, "tp_batch_execute: NULL argument");
    std::lock_guard<std::mutex> lk(b->e->exec_mu);
    std::vector<tp_result*> rs;
    tp_status s = batch_run(b, &rs);
    if (s) return s;
    for (size_t i = 0; i < rs.size(); ++i) results[i] = rs[i];
    return TP_OK;
}

double tp_batch_last_ms(const tp_batch* b) { return b ? b->last_ms : 0.0; }

tp_status tp_debug_batch_stall(tp_batch* b, int32_t query, uint64_t wait_ns) {
    clear_error();
    if (!b || query >= (int32_t)b->plans.size() || (query >= 0 && wait_ns == 0))
        return fail(TP_E_INVALID, "tp_debug_batch_stall: bad arguments");
    std::lock_guard<std::mutex> lk(b->e->exec_mu);
    TP_TRY_CUDA(cudaSetDevice(b->e->device));
    const uint64_t w = query >= 0 ? wait_ns : BATCH_WAIT_NS;
    TP_TRY_CUDA(cudaMemcpy(b->d_wait, &w, 8, cudaMemcpyHostToDevice));
    for (int i = 0; i < (int)b->plans.size(); ++i) {
        // the stalled query's finalisation waits for one probe tile more than exists
        const uint32_t want = b->probe_items[i] + (i == query ? 1u : 0u);
        TP_TRY_CUDA(cudaMemcpy(&b->d_q[i].probe_items, &want, 4, cudaMemcpyHostToDevice));
    }
    return TP_OK;
}

void tp_batch_destroy(tp_batch* b) { batch_free(b); }

tp_status tp_autotune(tp_engine* e, tp_plan* const* plans, int32_t n, const char* path) {
    clear_error();
    if (!e || !plans || n < 1 || !path) return fail(TP_E_INVALID, "tp_autotune: bad arguments");
    std::lock_guard<std::mutex> lk(e->exec_mu);
    // every class is tuned in the same runs of the whole set: a candidate
    // value of one knob is tried for every class at once, and each class
    // keeps it when its own queries' CTA time (summed over their tasks, read
    // from the device) fell by 2% or more
    std::vector<int> cls(n);
    std::map<int, Tune> table;
    for (int i = 0; i < n; ++i) {
        cls[i] = query_class(plans[i]);
        table[cls[i]] = Tune{0.5f, 1024, TP_AGG_AUTO};
    }
    auto class_cost = [&](const std::map<int, Tune>& t, std::map<int, double>* cost) -> tp_status {
        tp_batch* b = nullptr;
        tp_status s = batch_create_impl(e, plans, n, t, &b);
        if (s) return s;
        cost->clear();
        std::vector<unsigned long long> ns(n);
        for (int rep = 0; rep < 3 && s == TP_OK; ++rep) {   // the best of three runs per query
            s = batch_run(b, nullptr);
            if (s) break;
            cudaError_t ce = cudaMemcpy(ns.data(), b->d_task_ns, 8ull * n, cudaMemcpyDeviceToHost);
            if (ce != cudaSuccess) {
                s = fail(TP_E_CUDA, "tp_autotune: %s", cudaGetErrorString(ce));
                break;
            }
            std::map<int, double> c;
            for (int i = 0; i < n; ++i) c[cls[i]] += (double)ns[i];
            for (auto& kv : c) {
                auto it = cost->find(kv.first);
                if (it == cost->end() || kv.second < it->second) (*cost)[kv.first] = kv.second;
            }
        }
        batch_free(b);
        return s;
    };
    std::map<int, double> best;
    tp_status s = class_cost(table, &best);
    if (s) return s;
    const uint32_t rpw[] = {128, 256, 512, 1024};
    const int aggs[] = {TP_AGG_AUTO, TP_AGG_GLOBAL};
    const float lfs[] = {0.5f, 0.7f};
    for (int knob = 0; knob < 3; ++knob) {
        const int nv = knob == 0 ? 4 : 2;
        for (int v = 0; v < nv; ++v) {
            std::map<int, Tune> cand = table;
            bool differs = false;
            for (auto& kv : cand) {
                Tune t = kv.second;
                if (knob == 0) t.rows_per_warp = rpw[v];
                if (knob == 1) t.agg = aggs[v];
                if (knob == 2) t.lf = lfs[v];
                differs = differs || memcmp(&t, &kv.second, sizeof(Tune)) != 0;
                kv.second = t;
            }
            if (!differs) continue;
            std::map<int, double> cost;
            if ((s = class_cost(cand, &cost))) return s;
            for (auto& kv : cost) {
                if (kv.second < best[kv.first] * 0.98) {
                    best[kv.first] = kv.second;
                    table[kv.first] = cand[kv.first];
                }
            }
        }
    }
    FILE* f = fopen(path, "w");
    if (!f) return fail(TP_E_INVALID, "tp_autotune: cannot write %s", path);
    fprintf(f, "# theseus-gb autotune: class load_factor rows_per_warp agg(0 auto, 2 device memory)\n");
    for (auto& kv : table)
        fprintf(f, "%d %.2f %u %d\n", kv.first, kv.second.lf, kv.second.rows_per_warp, kv.second.agg);
    fclose(f);
    return TP_OK;
}

}  // extern "C"
