// Staged fused filter -> probe -> aggregate kernel (few groups).
//
// Paper basis: Section 3.1 (operators run GPU kernels over batches of
// equal-length columns), Section 3.2 (join), Section 4 (decimals held as
// 128-bit integers).  The pipeline itself is this library's design for
// sm_103a:
//
//   warp 0 (one lane)  : for every tile of ST_TILE rows this CTA owns, waits
//                        until the consumers have released a stage, then
//                        issues one 1-D bulk copy (cp.async.bulk) per column
//                        the query reads into that stage; the copies signal
//                        the stage's "full" mbarrier with their byte count.
//                        Streaming copies carry an L2 evict-first policy so
//                        the join table stays resident in L2.
//   warps 1..C         : wait for a full stage, each evaluates 32 * ST_RPL
//                        rows of it (lane l taking rows l, l+32, ...: every
//                        shared-memory load is conflict-free), then arrive on
//                        the stage's "empty" mbarrier.
//
// Several CTAs share an SM (ST_CTAS), so many consumer warps keep hash probes
// and shared-memory atomics in flight.  Groups accumulate in a per-CTA dense
// table in shared memory.  With `FAST` (the host proved from column bounds
// that no sum can leave int64) the table holds only 32-bit words -- 32-bit
// shared-memory atomics are about 12x the throughput of 64-bit ones on this
// part -- each term offset by its proven minimum so it is non-negative, with a
// carry word where a per-CTA sum can pass 2^32.  Otherwise the table holds
// exact 128-bit sums updated with 64-bit atomics and carry propagation.
//
// The kernel takes whole tiles only; the host runs the rows after the last
// whole tile through the plain-load kernel.  Every mbarrier wait is bounded by
// L.wait_ns of %globaltimer time; on expiry the kernel records ERR_TIMEOUT and
// the CTA winds down.
#include <algorithm>

#include "pipeline.cuh"

namespace tpk {

// Shared-memory dense table of one CTA.
//   FAST (narrow): 32-bit words only -- shared-memory atomics on 32-bit words
//   are an order of magnitude faster than on 64-bit ones.  count[G], then per
//   sum s a block of low words at L.sum_word[s] and, in mode 2, the next
//   block of carry words.
//   Exact: count[G] (u64) then lo[s][G], hi[s][G] with 128-bit carries.
template <bool FAST>
struct DenseTable {
    unsigned char* base;
    uint32_t G;
    __device__ __forceinline__ void add_count(uint32_t g) const {
        if constexpr (FAST) atomicAdd((unsigned int*)base + g, 1u);
        else atomicAdd((unsigned long long*)base + g, 1ull);
    }
    __device__ __forceinline__ uint32_t* words(uint32_t block) const { return (uint32_t*)base + (uint64_t)block * G; }
    __device__ __forceinline__ uint64_t* lo(int s) const { return (uint64_t*)base + (uint64_t)G * (1 + 2 * s); }
    __device__ __forceinline__ uint64_t* hi(int s) const { return (uint64_t*)base + (uint64_t)G * (2 + 2 * s); }
};

template <bool FAST>
__device__ __forceinline__ uint32_t G_of(const DenseTable<FAST>& t) { return t.G; }

// Full tile in shared memory: every load is in bounds, so loads are issued
// for all 8 rows and the pass mask only guards probes and side effects.
template <int NS, bool FAST>
__device__ __forceinline__ void consume_dense_full(const QueryDev& q, const StageLayout& L,
                                                   const unsigned char* stage, uint32_t r0,
                                                   const DenseTable<FAST>& tab) {
    uint32_t pm = 0xFFu;
    int64_t v[ST_RPL];
    if (q.has_filter) {
        load8_smem(stage + L.off[L.col_of_slot[SL_FILTER]], q.fcol.type, r0, v);
        uint32_t keep = 0;
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) keep |= (uint32_t)(v[j] >= q.flo && v[j] <= q.fhi) << j;
        pm = keep;
        if (!pm) return;
    }
    uint32_t pay[ST_RPL];
    if (q.has_join) {
        load8_smem(stage + L.off[L.col_of_slot[SL_FK]], q.fk.type, r0, v);
        probe_rows(q.jt, v, pm, pay, q.err);
        uint32_t bad = 0;
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) bad |= (uint32_t)((pay[j] & PAYLOAD_BAD) != 0) << j;
        if (bad & pm) {
            atomicOr(q.err, ERR_RANGE);
            pm &= ~bad;
        }
        if (!pm) return;
    }
    uint32_t g[ST_RPL];
#pragma unroll
    for (int j = 0; j < ST_RPL; ++j) g[j] = 0;
#pragma unroll
    for (int f = 0; f < MAX_GROUP; ++f) {
        if (f >= q.n_group) break;
        const int bits = q.gbits[f];
        if (q.gside[f] == 0) {
            load8_smem(stage + L.off[L.col_of_slot[SL_GROUP + f]], q.gcol[f].type, r0, v);
            uint32_t bad = 0;
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                bad |= (uint32_t)(((uint64_t)v[j] >> bits) != 0) << j;
                g[j] = (g[j] << bits) | (uint32_t)v[j];
            }
            if (bad & pm) {
                atomicOr(q.err, ERR_RANGE);
                pm &= ~bad;
            }
        } else {
            const uint32_t mask = (1u << bits) - 1u;
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) g[j] = (g[j] << bits) | ((pay[j] >> q.gdpos[f]) & mask);
        }
    }
    if (!pm) return;
#pragma unroll
    for (int j = 0; j < ST_RPL; ++j)
        if (pm & (1u << j)) tab.add_count(g[j]);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if (s >= q.n_sum) break;
        load8_smem(stage + L.off[L.col_of_slot[SL_SA + s]], q.sa[s].type, r0, v);
        const bool ms = q.skind[s] == S_MUL_SUB;
        if constexpr (FAST) {
            if (ms) {
                int64_t b[ST_RPL];
                load8_smem(stage + L.off[L.col_of_slot[SL_SB + s]], q.sb[s].type, r0, b);
                const int64_t k = q.sk[s];
#pragma unroll
                for (int j = 0; j < ST_RPL; ++j) v[j] *= (k - b[j]);
            }
            const int64_t off = L.sum_off[s];
            uint32_t* lo = tab.words(L.sum_word[s]);
            if (L.sum_mode[s] == 1) {
#pragma unroll
                for (int j = 0; j < ST_RPL; ++j)
                    if (pm & (1u << j)) atomicAdd(lo + g[j], (uint32_t)(uint64_t)(v[j] - off));
            } else {
                uint32_t old[ST_RPL];
#pragma unroll
                for (int j = 0; j < ST_RPL; ++j)
                    old[j] = (pm & (1u << j)) ? atomicAdd(lo + g[j], (uint32_t)(uint64_t)(v[j] - off)) : 0u;
                uint32_t* hi = lo + G_of(tab);
#pragma unroll
                for (int j = 0; j < ST_RPL; ++j) {
                    const uint64_t t = (uint64_t)(v[j] - off);
                    const uint32_t h = (uint32_t)(t >> 32) + ((old[j] + (uint32_t)t) < old[j] ? 1u : 0u);
                    if ((pm & (1u << j)) && h) atomicAdd(hi + g[j], h);
                }
            }
        } else {
            uint64_t* lo = tab.lo(s);
            uint64_t* hi = tab.hi(s);
            if (ms) {
                int64_t b[ST_RPL];
                load8_smem(stage + L.off[L.col_of_slot[SL_SB + s]], q.sb[s].type, r0, b);
#pragma unroll
                for (int j = 0; j < ST_RPL; ++j)
                    if (pm & (1u << j)) atomic_add_i128(lo + g[j], hi + g[j], mul_sub(v[j], q.sk[s], b[j]));
            } else {
#pragma unroll
                for (int j = 0; j < ST_RPL; ++j)
                    if (pm & (1u << j)) atomic_add_i128(lo + g[j], hi + g[j], i128_from_i64(v[j]));
            }
        }
    }
}

template <int NS, bool FAST>
__global__ void __launch_bounds__(ST_THREADS, ST_CTAS)
    k_agg_shared_staged(const __grid_constant__ QueryDev q, const __grid_constant__ StageLayout L, uint64_t n,
                        uint64_t* __restrict__ gacc, uint32_t G) {
    extern __shared__ __align__(128) unsigned char smem[];
    DenseTable<FAST> tab{smem, G};
    for (uint32_t i = threadIdx.x; i < L.table_bytes / 8; i += blockDim.x) ((uint64_t*)smem)[i] = 0;
    run_pipeline(q, L, n, smem + L.table_bytes, [&](const unsigned char* stage, uint64_t, uint32_t r0) {
        consume_dense_full<NS, FAST>(q, L, stage, r0, tab);
    });
    __syncthreads();
    // fold this CTA's table into the global dense table (count[G], lo/hi[s][G])
    for (uint32_t gi = threadIdx.x; gi < G; gi += blockDim.x) {
        uint64_t c;
        if constexpr (FAST) c = ((const unsigned int*)smem)[gi];
        else c = ((const uint64_t*)smem)[gi];
        if (c == 0) continue;
        atomicAdd((unsigned long long*)&gacc[gi], (unsigned long long)c);
        for (int s = 0; s < q.n_sum; ++s) {
            if constexpr (FAST) {
                // sum = carry words * 2^32 + low words + count * offset, exact
                // modulo 2^64 and, by the bounds, inside int64
                const uint32_t* w = tab.words(L.sum_word[s]);
                uint64_t v = w[gi];
                if (L.sum_mode[s] == 2) v += (uint64_t)w[G + gi] << 32;
                v += c * (uint64_t)L.sum_off[s];
                atomicAdd((unsigned long long*)&gacc[(uint64_t)G * (1 + 2 * s) + gi], (unsigned long long)v);
            } else {
                I128 v{tab.lo(s)[gi], tab.hi(s)[gi]};
                atomic_add_i128(&gacc[(uint64_t)G * (1 + 2 * s) + gi], &gacc[(uint64_t)G * (2 + 2 * s) + gi], v);
            }
        }
    }
}

// ------------------------------------------------------------------- host

static uint32_t align128(uint64_t x) { return (uint32_t)((x + 127) & ~127ull); }

static int esize_host(int type) { return type == T_I64 ? 8 : (type == T_I32 ? 4 : 1); }

bool staged_layout_shared(const QueryDev& q, uint32_t key_bits, bool fast, const TermBounds* bounds,
                          uint64_t rows, int num_sms, const StageGeom& geom, int max_stages, StageLayout* L) {
    memset(L, 0, sizeof(*L));
    for (int i = 0; i < SL_COUNT; ++i) L->col_of_slot[i] = -1;
    auto add = [&](int slot, const DevCol& c) -> bool {
        if (((uintptr_t)c.ptr & 15u) != 0) return false;
        for (int k = 0; k < L->n_cols; ++k)
            if (L->src[k] == c.ptr && L->esize[k] == esize_host(c.type)) {
                L->col_of_slot[slot] = (int8_t)k;
                return true;
            }
        if (L->n_cols >= ST_MAX_COLS) return false;
        const int k = L->n_cols++;
        L->src[k] = c.ptr;
        L->esize[k] = esize_host(c.type);
        L->col_of_slot[slot] = (int8_t)k;
        return true;
    };
    bool ok = true;
    if (q.has_filter) ok = ok && add(SL_FILTER, q.fcol);
    if (q.has_join) ok = ok && add(SL_FK, q.fk);
    for (int j = 0; j < q.n_xjoin; ++j) ok = ok && add(SL_FKX + j, q.fkx[j]);   // run-time compiled kernel only
    for (int g = 0; g < q.n_group; ++g)
        if (q.gside[g] == 0) ok = ok && add(SL_GROUP + g, q.gcol[g]);
    for (int s = 0; s < q.n_sum; ++s) {
        ok = ok && add(SL_SA + s, q.sa[s]);
        if (q.skind[s] == S_MUL_SUB) ok = ok && add(SL_SB + s, q.sb[s]);
    }
    if (!ok) return false;
    const uint32_t tile = (uint32_t)geom.consumers * 32u * (uint32_t)geom.rpl;
    L->tile = (int32_t)tile;
    L->threads = 32 * (1 + geom.consumers);
    L->ctas = geom.ctas;
    uint32_t off = 0;
    for (int k = 0; k < L->n_cols; ++k) {
        L->off[k] = off;
        L->tile_bytes += tile * L->esize[k];
        off = align128(off + (uint64_t)tile * L->esize[k]);
    }
    L->stage_bytes = off ? off : 128;
    const uint64_t G = 1ull << key_bits;
    if (fast) {
        // rows one CTA can see in this launch bound every 32-bit word: its
        // share of the whole tiles plus, for the run-time compiled kernel, the
        // rows after the last whole tile, which CTA (tiles % grid) evaluates
        // too -- CTA 0, holding a full share, when tiles is a multiple of grid
        const uint64_t tiles = rows / tile;
        const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(tiles, (uint64_t)num_sms * geom.ctas));
        const uint64_t r_cta = (tiles + grid - 1) / grid * (uint64_t)tile + (rows - tiles * (uint64_t)tile);
        if (r_cta >= (1ull << 32)) return false;
        uint32_t block = 1;   // block 0: counts
        for (int s = 0; s < q.n_sum; ++s) {
            const unsigned __int128 rs = (unsigned __int128)r_cta;
            const uint64_t span = bounds[s].span;
            if (rs * span <= 0xFFFFFFFFull) {
                L->sum_mode[s] = 1;
            } else if (rs * ((span >> 32) + 1) <= 0xFFFFFFFFull) {
                L->sum_mode[s] = 2;
            } else {
                return false;
            }
            L->sum_off[s] = bounds[s].lo;
            L->sum_word[s] = block;
            block += (uint32_t)L->sum_mode[s];
        }
        L->table_bytes = align128(G * 4 * block);
    } else {
        L->table_bytes = align128(G * 8 * (1 + 2 * (uint64_t)q.n_sum));
    }
    int dev = 0, optin = 0, per_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
        return false;
    // each of the resident CTAs gets its share (1 KB per CTA stays reserved by the runtime)
    const uint64_t budget = std::min<uint64_t>((uint64_t)optin, (uint64_t)per_sm / geom.ctas - 1024);
    const uint64_t fixed = L->table_bytes + 2 * ST_MAX_STAGES * sizeof(uint64_t);
    if (budget <= fixed) return false;
    int stages = (int)((budget - fixed) / L->stage_bytes);
    if (stages > max_stages) stages = max_stages;
    if (stages > ST_MAX_STAGES) stages = ST_MAX_STAGES;
    if (stages < 2) return false;
    L->n_stages = stages;
    L->smem_bytes = (uint32_t)(fixed + (uint64_t)stages * L->stage_bytes);
    L->wait_ns = 2000000000ull;
    return true;
}

template <int NS, bool FAST>
static cudaError_t launch_staged_t(const QueryDev& q, const StageLayout& L, uint64_t n, uint64_t* gacc,
                                   uint32_t G, int grid, cudaStream_t st) {
    auto fn = k_agg_shared_staged<NS, FAST>;
    cudaError_t e = ensure_smem_limit((const void*)fn, (int)L.smem_bytes);
    if (e != cudaSuccess) return e;
    fn<<<grid, ST_THREADS, L.smem_bytes, st>>>(q, L, n, gacc, G);
    return cudaGetLastError();
}

cudaError_t launch_agg_shared_staged(const QueryDev& q, const StageLayout& L, uint64_t n, uint64_t* gacc,
                                     uint32_t key_bits, bool fast, int num_sms, cudaStream_t st) {
    if (n < (uint64_t)ST_TILE) return cudaSuccess;
    const uint64_t tiles = n / ST_TILE;
    const uint64_t slots = (uint64_t)num_sms * ST_CTAS;
    const int grid = (int)(tiles < slots ? tiles : slots);
    const uint32_t G = 1u << key_bits;
    const int ns = q.n_sum;
    if (fast) {
        if (ns <= 1) return launch_staged_t<1, true>(q, L, n, gacc, G, grid, st);
        if (ns <= 2) return launch_staged_t<2, true>(q, L, n, gacc, G, grid, st);
        if (ns <= 4) return launch_staged_t<4, true>(q, L, n, gacc, G, grid, st);
        return launch_staged_t<8, true>(q, L, n, gacc, G, grid, st);
    }
    if (ns <= 1) return launch_staged_t<1, false>(q, L, n, gacc, G, grid, st);
    if (ns <= 2) return launch_staged_t<2, false>(q, L, n, gacc, G, grid, st);
    if (ns <= 4) return launch_staged_t<4, false>(q, L, n, gacc, G, grid, st);
    return launch_staged_t<8, false>(q, L, n, gacc, G, grid, st);
}

cudaError_t launch_agg_shared_staged_jit(const void* kernel, const QueryDev& q, const StageLayout& L, uint64_t n,
                                         uint64_t* gacc, uint32_t key_bits, int num_sms, cudaStream_t st) {
    if (n < (uint64_t)L.tile) return cudaSuccess;
    const uint64_t tiles = n / (uint64_t)L.tile;
    const uint64_t slots = (uint64_t)num_sms * L.ctas;
    const int grid = (int)(tiles < slots ? tiles : slots);
    uint32_t G = 1u << key_bits;
    cudaError_t e = ensure_smem_limit(kernel, (int)L.smem_bytes);
    if (e != cudaSuccess) return e;
    QueryDev qa = q;
    StageLayout la = L;
    void* args[] = {&qa, &la, &n, &gacc, &G};
    return cudaLaunchKernel(kernel, dim3(grid), dim3(L.threads), args, L.smem_bytes, st);
}

}  // namespace tpk
