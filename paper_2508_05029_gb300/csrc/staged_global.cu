// Staged fused filter -> probe -> aggregate kernel for many groups: the
// bulk-copy pipeline of pipeline.cuh feeding one open-addressing aggregation
// table in device memory.
//
// Paper basis: Section 3.1 (operators over batches of equal-length columns),
// Section 3.2 (join), Section 4 (decimals held as 128-bit integers).  Design
// choices of this library:
//
//  * Late materialisation.  When the filter is selective the layout stages
//    only the filter column; every other column is read from global memory
//    for the surviving rows only, so a 1%-selective scan moves little more
//    than the filter column.
//  * Warp aggregation.  Lanes whose rows carry the same group key find each
//    other with __match_any_sync; the lowest lane of each set adds the
//    others' count and terms (shuffles) and updates the table once, so a key
//    repeated within a warp's rows costs one table update, not one per row.
//  * Bulk occupancy counting.  New slots of a hashed table are counted per
//    lane and added to the table's counter once per CTA.
//  * 64-bit updates.  When column bounds prove every sum stays in int64
//    (FAST), counts and sums are fire-and-forget 64-bit global reductions on
//    the low words; the high words are filled in by sign extension when the
//    groups are gathered.  Otherwise each row adds an exact 128-bit term with
//    carry propagation.
#include <algorithm>

#include "agg_warp.cuh"
#include "pipeline.cuh"

namespace tpk {

// bytes in front of the ring: the CTA's claimed-slot counter (keeps the
// stages 128-byte aligned)
constexpr uint32_t GLOBAL_RING_OFFSET = 128;

// Filter, probe and pack the 64-bit group keys of this lane's rows; returns
// the mask of surviving rows (no early exit: callers use warp shuffles).
__device__ __forceinline__ uint32_t eval_keys64(const QueryDev& q, const StageLayout& L,
                                                const unsigned char* stage, uint64_t row0, uint32_t r0,
                                                uint64_t key[ST_RPL]) {
    uint32_t pm = (1u << ST_RPL) - 1u;
    int64_t v[ST_RPL];
#pragma unroll
    for (int j = 0; j < ST_RPL; ++j) key[j] = 0;
    if (q.has_filter) {
        load_rows(col_src(L, SL_FILTER, q.fcol, stage, row0), r0, pm, v);
        uint32_t keep = 0;
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) keep |= (uint32_t)(v[j] >= q.flo && v[j] <= q.fhi) << j;
        pm = keep;
    }
    uint32_t pay[ST_RPL];
#pragma unroll
    for (int j = 0; j < ST_RPL; ++j) pay[j] = 0;
    if (q.has_join && pm) {
        load_rows(col_src(L, SL_FK, q.fk, stage, row0), r0, pm, v);
        probe_rows(q.jt, v, pm, pay, q.err);
        uint32_t bad = 0;
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) bad |= (uint32_t)((pay[j] & PAYLOAD_BAD) != 0) << j;
        if (bad & pm) {
            atomicOr(q.err, ERR_RANGE);
            pm &= ~bad;
        }
    }
#pragma unroll
    for (int f = 0; f < MAX_GROUP; ++f) {
        if (f >= q.n_group || !pm) break;
        const int bits = q.gbits[f];
        if (q.gside[f] == 0) {
            load_rows(col_src(L, SL_GROUP + f, q.gcol[f], stage, row0), r0, pm, v);
            uint32_t bad = 0;
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                if (bits < 64) {
                    bad |= (uint32_t)(((uint64_t)v[j] >> bits) != 0) << j;
                    key[j] = (key[j] << bits) | (uint64_t)v[j];
                } else {
                    key[j] = (uint64_t)v[j];
                }
            }
            if (bad & pm) {
                atomicOr(q.err, ERR_RANGE);
                pm &= ~bad;
            }
        } else {
            const uint32_t mask = (1u << bits) - 1u;
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) key[j] = (key[j] << bits) | ((pay[j] >> q.gdpos[f]) & mask);
        }
    }
    return pm;
}

// Terms of sum s for this lane's rows (64-bit; FAST only).
__device__ __forceinline__ void eval_terms64(const QueryDev& q, const StageLayout& L, int s,
                                             const unsigned char* stage, uint64_t row0, uint32_t r0, uint32_t pm,
                                             int64_t t[ST_RPL]) {
    load_rows(col_src(L, SL_SA + s, q.sa[s], stage, row0), r0, pm, t);
    if (q.skind[s] == S_MUL_SUB) {
        int64_t b[ST_RPL];
        load_rows(col_src(L, SL_SB + s, q.sb[s], stage, row0), r0, pm, b);
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) t[j] *= (q.sk[s] - b[j]);
    }
}

template <int NS, bool FAST>
__device__ __forceinline__ void consume_global(const QueryDev& q, const StageLayout& L, const AggTable& tab,
                                               const unsigned char* stage, uint64_t row0, uint32_t r0,
                                               uint32_t& claims) {
    uint64_t key[ST_RPL];
    const uint32_t pm = eval_keys64(q, L, stage, row0, r0, key);
    if (__ballot_sync(0xffffffffu, pm != 0) == 0) return;   // warp-uniform exit
    int64_t t[NS > 0 ? NS : 1][ST_RPL];
    I128 tm[NS > 0 ? NS : 1][ST_RPL];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if (s >= q.n_sum) break;
        if constexpr (FAST) {
            eval_terms64(q, L, s, stage, row0, r0, pm, t[s]);
        } else {
            int64_t a[ST_RPL];
            load_rows(col_src(L, SL_SA + s, q.sa[s], stage, row0), r0, pm, a);
            if (q.skind[s] == S_MUL_SUB) {
                int64_t b[ST_RPL];
                load_rows(col_src(L, SL_SB + s, q.sb[s], stage, row0), r0, pm, b);
#pragma unroll
                for (int j = 0; j < ST_RPL; ++j) tm[s][j] = mul_sub(a[j], q.sk[s], b[j]);
            } else {
#pragma unroll
                for (int j = 0; j < ST_RPL; ++j) tm[s][j] = i128_from_i64(a[j]);
            }
        }
    }
    bool valid[ST_RPL];
#pragma unroll
    for (int j = 0; j < ST_RPL; ++j) valid[j] = (pm >> j) & 1u;
    agg_warp_rows<NS, FAST, ST_RPL>(tab, q.err, q.n_sum, valid, key, t, tm, claims);
}

template <int NS, bool FAST>
__global__ void __launch_bounds__(ST_THREADS, ST_CTAS)
    k_agg_global_staged(const __grid_constant__ QueryDev q, const __grid_constant__ StageLayout L, uint64_t n,
                        const __grid_constant__ AggTable tab) {
    extern __shared__ __align__(128) unsigned char smem[];
    // the CTA's claimed-slot count sits in front of the ring
    unsigned int* cta_claims = (unsigned int*)smem;
    if (threadIdx.x == 0) *cta_claims = 0;
    uint32_t claims = 0;
    run_pipeline(q, L, n, smem + GLOBAL_RING_OFFSET, [&](const unsigned char* stage, uint64_t row0, uint32_t r0) {
        consume_global<NS, FAST>(q, L, tab, stage, row0, r0, claims);
    });
    if (threadIdx.x >= 32) {
        const uint32_t w = __reduce_add_sync(0xffffffffu, claims);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(cta_claims, w);
    }
    __syncthreads();
    if (threadIdx.x == 0) agg_add_claims(tab, q.err, *cta_claims);
}

// ------------------------------------------------------------------- host

static uint32_t align128g(uint64_t x) { return (uint32_t)((x + 127) & ~127ull); }

bool staged_layout_global(const QueryDev& q, bool stage_all, StageLayout* L) {
    memset(L, 0, sizeof(*L));
    for (int i = 0; i < SL_COUNT; ++i) L->col_of_slot[i] = -1;
    auto esz = [](int type) { return type == T_I64 ? 8 : (type == T_I32 ? 4 : 1); };
    auto add = [&](int slot, const DevCol& c) -> bool {
        if (((uintptr_t)c.ptr & 15u) != 0) return false;
        for (int k = 0; k < L->n_cols; ++k)
            if (L->src[k] == c.ptr && L->esize[k] == esz(c.type)) {
                L->col_of_slot[slot] = (int8_t)k;
                return true;
            }
        if (L->n_cols >= ST_MAX_COLS) return false;
        const int k = L->n_cols++;
        L->src[k] = c.ptr;
        L->esize[k] = esz(c.type);
        L->col_of_slot[slot] = (int8_t)k;
        return true;
    };
    bool ok = true;
    if (q.has_filter) ok = ok && add(SL_FILTER, q.fcol);
    if (stage_all || !q.has_filter) {
        if (q.has_join) ok = ok && add(SL_FK, q.fk);
        for (int g = 0; g < q.n_group; ++g)
            if (q.gside[g] == 0) ok = ok && add(SL_GROUP + g, q.gcol[g]);
        for (int s = 0; s < q.n_sum; ++s) {
            ok = ok && add(SL_SA + s, q.sa[s]);
            if (q.skind[s] == S_MUL_SUB) ok = ok && add(SL_SB + s, q.sb[s]);
        }
    }
    if (!ok || L->n_cols == 0) return false;
    uint32_t off = 0;
    for (int k = 0; k < L->n_cols; ++k) {
        L->off[k] = off;
        L->tile_bytes += (uint32_t)ST_TILE * L->esize[k];
        off = align128g(off + (uint64_t)ST_TILE * L->esize[k]);
    }
    L->stage_bytes = off;
    L->table_bytes = 0;
    int dev = 0, optin = 0, per_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
        return false;
    const uint64_t budget = std::min<uint64_t>((uint64_t)optin, (uint64_t)per_sm / ST_CTAS - 1024);
    const uint64_t fixed = GLOBAL_RING_OFFSET + 2 * ST_MAX_STAGES * sizeof(uint64_t);
    int stages = (int)((budget - fixed) / L->stage_bytes);
    if (stages > ST_MAX_STAGES) stages = ST_MAX_STAGES;
    if (stages < 2) return false;
    L->n_stages = stages;
    L->smem_bytes = (uint32_t)(fixed + (uint64_t)stages * L->stage_bytes);
    L->wait_ns = 2000000000ull;
    return true;
}

template <int NS, bool FAST>
static cudaError_t launch_global_t(const QueryDev& q, const StageLayout& L, uint64_t n, const AggTable& t,
                                   int grid, cudaStream_t st) {
    auto fn = k_agg_global_staged<NS, FAST>;
    cudaError_t e = ensure_smem_limit((const void*)fn, (int)L.smem_bytes);
    if (e != cudaSuccess) return e;
    fn<<<grid, ST_THREADS, L.smem_bytes, st>>>(q, L, n, t);
    return cudaGetLastError();
}

cudaError_t launch_agg_global_staged(const QueryDev& q, const StageLayout& L, uint64_t n, const AggTable& t,
                                     bool fast, int num_sms, cudaStream_t st) {
    if (n < (uint64_t)ST_TILE) return cudaSuccess;
    const uint64_t tiles = n / ST_TILE;
    const uint64_t slots = (uint64_t)num_sms * ST_CTAS;
    const int grid = (int)(tiles < slots ? tiles : slots);
    const int ns = q.n_sum;
    if (fast) {
        if (ns <= 1) return launch_global_t<1, true>(q, L, n, t, grid, st);
        if (ns <= 2) return launch_global_t<2, true>(q, L, n, t, grid, st);
        if (ns <= 4) return launch_global_t<4, true>(q, L, n, t, grid, st);
        return launch_global_t<8, true>(q, L, n, t, grid, st);
    }
    if (ns <= 1) return launch_global_t<1, false>(q, L, n, t, grid, st);
    if (ns <= 2) return launch_global_t<2, false>(q, L, n, t, grid, st);
    if (ns <= 4) return launch_global_t<4, false>(q, L, n, t, grid, st);
    return launch_global_t<8, false>(q, L, n, t, grid, st);
}

}  // namespace tpk
