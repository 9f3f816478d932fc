// Radix partitioning for the out-of-core (hybrid) hash join.
//
// Paper basis: Section 3.1 (Batch Holders move data to a larger memory tier
// when the GPU's is scarce), Section 3.3.2 (the Memory Executor spills data
// that is not needed soon), Section 3.2 (the exchange hash-partitions both
// join sides).  On one GPU both sides of the join are split into P = 2^k
// partitions by the top k bits of fmix64(key).  Partitions whose hash table
// fits the device budget stay resident and are probed while the fact table
// streams; the build and fact rows of the other partitions are written out
// (these kernels) and spilled to pinned host pages, then joined one partition
// at a time.
#include "device.cuh"

namespace tpk {

__device__ __forceinline__ uint32_t part_of(int64_t key, int shift) {
    return (uint32_t)(fmix64((uint64_t)key) >> shift);
}

// Per-block shared histogram of the admitted build rows, merged into counts.
__global__ void k_part_hist(const __grid_constant__ BuildDev b, uint64_t n, int shift, unsigned long long* counts) {
    __shared__ unsigned h[256];
    const uint32_t P = 1u << (64 - shift);
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        if (dim_row_admitted(b, i)) atomicAdd(&h[part_of(ld1(b.key, i), shift)], 1u);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x)
        if (h[i]) atomicAdd(&counts[i], (unsigned long long)h[i]);
}

cudaError_t launch_part_hist(const BuildDev& b, uint64_t n, int shift, unsigned long long* counts, int num_sms,
                             cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (shift < 56 || shift > 63) return cudaErrorInvalidValue;   // 2..256 partitions
    uint64_t blocks = (n + 255) / 256;
    if (blocks > (uint64_t)num_sms * 4) blocks = (uint64_t)num_sms * 4;
    k_part_hist<<<(unsigned)blocks, 256, 0, st>>>(b, n, shift, counts);
    return cudaGetLastError();
}

__device__ __forceinline__ bool fact_row_passes(const QueryDev& q, uint64_t i) {
    if (!q.has_filter) return true;
    const int64_t v = ld1(q.fcol, i);
    return v >= q.flo && v <= q.fhi;
}

// Fact rows that pass the filter and the lookahead filter and fall in a
// spilled partition, per partition.
__global__ void k_part_hist_fact(const __grid_constant__ QueryDev q, uint64_t n, int shift, uint64_t spill_mask,
                                 unsigned long long* counts) {
    __shared__ unsigned h[256];
    const uint32_t P = 1u << (64 - shift);
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (!fact_row_passes(q, i)) continue;
        const int64_t key = ld1(q.fk, i);
        const uint32_t p = part_of(key, shift);
        if (((spill_mask >> p) & 1ull) && (q.jt.lip == nullptr || lip_test(q.jt, key))) atomicAdd(&h[p], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x)
        if (h[i]) atomicAdd(&counts[i], (unsigned long long)h[i]);
}

cudaError_t launch_part_hist_fact(const QueryDev& q, uint64_t n, int shift, uint64_t spill_mask,
                                  unsigned long long* counts, int num_sms, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (shift < 58 || shift > 63) return cudaErrorInvalidValue;   // masks cover at most 64 partitions
    uint64_t blocks = (n + 255) / 256;
    if (blocks > (uint64_t)num_sms * 4) blocks = (uint64_t)num_sms * 4;
    k_part_hist_fact<<<(unsigned)blocks, 256, 0, st>>>(q, n, shift, spill_mask, counts);
    return cudaGetLastError();
}

// Scatter kernels place rows of spilled partitions with one global cursor
// atomic per (tile, partition): a tile of SP_TILE rows counts its rows per
// partition in shared memory, reserves each partition's range at once, and
// every row takes its rank inside its partition's range, so the rows of a
// partition from one tile land next to each other.
constexpr int SP_THREADS = 512;
constexpr int SP_RPT = 4;                          // rows per thread per tile
constexpr int SP_TILE = SP_THREADS * SP_RPT;

// Admitted build rows: insert the resident partitions, spill the others as
// pairs; every admitted key enters the lookahead filter.
__global__ void __launch_bounds__(SP_THREADS)
    k_build_part(const __grid_constant__ BuildDev b, uint64_t n, const unsigned long long* base,
                 unsigned long long* cursor, int64_t* keys, uint32_t* pays) {
    __shared__ unsigned cnt[64];
    __shared__ unsigned long long at0[64];
    const JoinTable& jt = b.jt;
    for (uint64_t t0 = (uint64_t)blockIdx.x * SP_TILE; t0 < n; t0 += (uint64_t)gridDim.x * SP_TILE) {
        if (threadIdx.x < 64) cnt[threadIdx.x] = 0;
        __syncthreads();
        uint32_t part[SP_RPT], rank[SP_RPT];
        bool spill[SP_RPT];
#pragma unroll
        for (int k = 0; k < SP_RPT; ++k) {
            const uint64_t i = t0 + (uint64_t)k * SP_THREADS + threadIdx.x;
            spill[k] = false;
            if (i >= n || !dim_row_admitted(b, i)) continue;
            const int64_t key = ld1(b.key, i);
            part[k] = part_of(key, jt.part_shift);
            if ((jt.part_mask >> part[k]) & 1ull) {
                build_insert(b, i);
            } else {
                if (jt.lip != nullptr) lip_insert(jt, key);
                spill[k] = true;
                rank[k] = atomicAdd(&cnt[part[k]], 1u);
            }
        }
        __syncthreads();
        if (threadIdx.x < 64 && cnt[threadIdx.x])
            at0[threadIdx.x] = base[threadIdx.x] + atomicAdd(&cursor[threadIdx.x], (unsigned long long)cnt[threadIdx.x]);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < SP_RPT; ++k) {
            if (!spill[k]) continue;
            const uint64_t i = t0 + (uint64_t)k * SP_THREADS + threadIdx.x;
            uint32_t payload = 0;
            for (int f = 0; f < b.n_dfield; ++f) {
                const int64_t v = ld1(b.dcol[f], i);
                if (v < 0 || ((uint64_t)v >> b.dbits[f]) != 0) payload |= PAYLOAD_BAD;
                else payload |= (uint32_t)((uint64_t)v << b.dpos[f]);
            }
            const uint64_t at = at0[part[k]] + rank[k];
            keys[at] = ld1(b.key, i);
            pays[at] = payload;
        }
        __syncthreads();
    }
}

cudaError_t launch_build_part(const BuildDev& b, uint64_t n, const unsigned long long* base,
                              unsigned long long* cursor, int64_t* keys, uint32_t* pays, int num_sms,
                              cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + SP_TILE - 1) / SP_TILE;
    if (blocks > (uint64_t)num_sms * 4) blocks = (uint64_t)num_sms * 4;
    k_build_part<<<(unsigned)blocks, SP_THREADS, 0, st>>>(b, n, base, cursor, keys, pays);
    return cudaGetLastError();
}

// Insert spilled (key, payload) pairs: the same table layout build_insert makes.
__global__ void k_build_pairs(const __grid_constant__ JoinTable jt, const int64_t* keys, const uint32_t* pays,
                              uint64_t n, uint32_t* err) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        // the payload is already packed: the same table logic as build_insert
        const int64_t key = keys[i];
        const uint32_t payload = pays[i];
        if (jt.direct) {
            const uint32_t v = (payload & PAYLOAD_BAD) ? PAYLOAD_BAD : payload;
            const uint64_t idx = (uint64_t)key - (uint64_t)jt.kmin;
            if (idx >= jt.range) { atomicOr(err, ERR_INTERNAL); continue; }
            if (atomicCAS((unsigned int*)jt.slots + idx, EMPTY32, v) != EMPTY32) atomicOr(err, ERR_DUP);
            continue;
        }
        const bool special = jt.key64 ? (uint64_t)key == EMPTY64 : (uint32_t)key == EMPTY32;
        if (special) {
            if (atomicCAS(jt.side, 0u, 1u) != 0u) atomicOr(err, ERR_DUP);
            else jt.side[1] = payload;
            continue;
        }
        uint64_t s = join_hash(jt, key) & jt.mask;
        bool placed = false;
        for (uint64_t it = 0; it <= jt.mask; ++it) {
            if (!jt.key64) {
                const unsigned long long want = ((unsigned long long)payload << 32) | (uint32_t)key;
                const unsigned long long prev =
                    atomicCAS((unsigned long long*)jt.slots + s, (unsigned long long)EMPTY64, want);
                if (prev == EMPTY64) { placed = true; break; }
                if ((uint32_t)prev == (uint32_t)key) { atomicOr(err, ERR_DUP); placed = true; break; }
            } else {
                const unsigned long long prev = atomicCAS((unsigned long long*)jt.slots + 2 * s,
                                                          (unsigned long long)EMPTY64, (unsigned long long)key);
                if (prev == EMPTY64) {
                    jt.slots[2 * s + 1] = payload;
                    placed = true;
                    break;
                }
                if (prev == (unsigned long long)key) { atomicOr(err, ERR_DUP); placed = true; break; }
            }
            s = (s + 1) & jt.mask;
        }
        if (!placed) atomicOr(err, ERR_INTERNAL);
    }
}

cudaError_t launch_build_pairs(const JoinTable& jt, const int64_t* keys, const uint32_t* pays, uint64_t n,
                               uint32_t* err, int num_sms, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > (uint64_t)num_sms * 8) blocks = (uint64_t)num_sms * 8;
    k_build_pairs<<<(unsigned)blocks, 256, 0, st>>>(jt, keys, pays, n, err);
    return cudaGetLastError();
}

// Fact rows of spilled partitions: copy every requested column to its
// partition's run in the staging columns, narrow where cols says so
// (tile-aggregated cursors, as above).
__global__ void __launch_bounds__(SP_THREADS)
    k_fact_spill(const __grid_constant__ QueryDev q, uint64_t n, uint64_t spill_mask,
                 const __grid_constant__ SpillCols cols, const unsigned long long* base, unsigned long long* cursor) {
    __shared__ unsigned cnt[64];
    __shared__ unsigned long long at0[64];
    const int shift = q.jt.part_shift;
    for (uint64_t t0 = (uint64_t)blockIdx.x * SP_TILE; t0 < n; t0 += (uint64_t)gridDim.x * SP_TILE) {
        if (threadIdx.x < 64) cnt[threadIdx.x] = 0;
        __syncthreads();
        uint32_t part[SP_RPT], rank[SP_RPT];
        bool spill[SP_RPT];
#pragma unroll
        for (int k = 0; k < SP_RPT; ++k) {
            const uint64_t i = t0 + (uint64_t)k * SP_THREADS + threadIdx.x;
            spill[k] = false;
            if (i >= n || !fact_row_passes(q, i)) continue;
            const int64_t key = ld1(q.fk, i);
            part[k] = part_of(key, shift);
            if (!((spill_mask >> part[k]) & 1ull)) continue;
            if (q.jt.lip != nullptr && !lip_test(q.jt, key)) continue;   // cannot join: not spilled
            spill[k] = true;
            rank[k] = atomicAdd(&cnt[part[k]], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 64 && cnt[threadIdx.x])
            at0[threadIdx.x] = base[threadIdx.x] + atomicAdd(&cursor[threadIdx.x], (unsigned long long)cnt[threadIdx.x]);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < SP_RPT; ++k) {
            if (!spill[k]) continue;
            const uint64_t i = t0 + (uint64_t)k * SP_THREADS + threadIdx.x;
            const uint64_t at = at0[part[k]] + rank[k];
            for (int c = 0; c < cols.n; ++c) {
                int64_t v;
                switch (cols.esize[c]) {
                case 8: v = ((const int64_t*)cols.src[c])[i]; break;
                case 4: v = ((const int32_t*)cols.src[c])[i]; break;
                default: v = ((const uint8_t*)cols.src[c])[i]; break;
                }
                const uint64_t d = cols.w[c] < cols.esize[c] ? (uint64_t)v - (uint64_t)cols.base[c] : (uint64_t)v;
                switch (cols.w[c]) {
                case 8: ((uint64_t*)cols.dst[c])[at] = d; break;
                case 4: ((uint32_t*)cols.dst[c])[at] = (uint32_t)d; break;
                case 2: ((uint16_t*)cols.dst[c])[at] = (uint16_t)d; break;
                default: ((uint8_t*)cols.dst[c])[at] = (uint8_t)d; break;
                }
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_fact_spill(const QueryDev& q, uint64_t n, uint64_t spill_mask, const SpillCols& cols,
                              const unsigned long long* base, unsigned long long* cursor, int num_sms,
                              cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + SP_TILE - 1) / SP_TILE;
    if (blocks > (uint64_t)num_sms * 4) blocks = (uint64_t)num_sms * 4;
    k_fact_spill<<<(unsigned)blocks, SP_THREADS, 0, st>>>(q, n, spill_mask, cols, base, cursor);
    return cudaGetLastError();
}

// ------------------------------------------------------- fan-out build

__global__ void k_many_collect(const __grid_constant__ BuildDev b, uint64_t n, uint64_t* __restrict__ keys,
                               uint32_t* __restrict__ pays, unsigned long long* ctr) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (!dim_row_admitted(b, i)) continue;
        const int64_t key = ld1(b.key, i);
        if (b.jt.lip != nullptr) lip_insert(b.jt, key);
        uint32_t payload = 0;
        for (int f = 0; f < b.n_dfield; ++f) {
            const int64_t v = ld1(b.dcol[f], i);
            if (v < 0 || ((uint64_t)v >> b.dbits[f]) != 0) payload |= PAYLOAD_BAD;
            else payload |= (uint32_t)((uint64_t)v << b.dpos[f]);
        }
        const unsigned long long at = atomicAdd(ctr, 1ull);
        keys[at] = (uint64_t)key;
        pays[at] = payload;
    }
}

cudaError_t launch_many_collect(const BuildDev& b, uint64_t n, uint64_t* keys, uint32_t* pays,
                                unsigned long long* ctr, int num_sms, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > (uint64_t)num_sms * 8) blocks = (uint64_t)num_sms * 8;
    k_many_collect<<<(unsigned)blocks, 256, 0, st>>>(b, n, keys, pays, ctr);
    return cudaGetLastError();
}

__global__ void k_many_heads(const uint64_t* __restrict__ keys, uint64_t n, int64_t* __restrict__ hkeys,
                             uint32_t* __restrict__ hidx, unsigned long long* ctr) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (i > 0 && keys[i] == keys[i - 1]) continue;
        const unsigned long long at = atomicAdd(ctr, 1ull);
        hkeys[at] = (int64_t)keys[i];
        hidx[at] = (uint32_t)i;
    }
}

cudaError_t launch_many_heads(const uint64_t* keys, uint64_t n, int64_t* hkeys, uint32_t* hidx,
                              unsigned long long* ctr, int num_sms, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > (uint64_t)num_sms * 8) blocks = (uint64_t)num_sms * 8;
    k_many_heads<<<(unsigned)blocks, 256, 0, st>>>(keys, n, hkeys, hidx, ctr);
    return cudaGetLastError();
}

}  // namespace tpk
