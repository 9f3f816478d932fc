// Operator kernels of the per-batch pipeline: hash build, fused
// filter -> probe -> aggregate (shared-memory or global table), and the
// finalisation that turns accumulators into sorted result rows.
//
// Paper basis: Section 3.1 (operators run GPU kernels over batches of
// equal-length columns; Filter and Join), Section 4 (decimal values held as
// 128-bit integers).  The kernel designs are this library's own.
//
// Row layout inside a warp tile: a warp owns 128 consecutive rows.  Lane l
// holds rows {2l, 2l+1, 64+2l, 64+2l+1}, so every column is read with two
// fully coalesced vector loads per lane whatever its width (8-bit: 2 bytes,
// 32-bit: 8 bytes, 64-bit: 16 bytes per load).
#include <algorithm>
#include <map>
#include <mutex>

#include "device.cuh"

namespace tpk {

// ------------------------------------------------------ launch attributes

cudaError_t ensure_smem_limit(const void* fn, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int> limit;   // (device, kernel) -> bytes set
    int dev = 0;
    cudaError_t g = cudaGetDevice(&dev);
    if (g != cudaSuccess) return g;
    std::lock_guard<std::mutex> lk(mu);
    int& cur = limit[{dev, fn}];
    if (bytes <= cur) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// --------------------------------------------------------------------- fill

__global__ void k_fill_u64(uint64_t* p, uint64_t n, uint64_t v) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

cudaError_t launch_fill_u64(uint64_t* p, uint64_t n, uint64_t v, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_fill_u64<<<(unsigned)blocks, 256, 0, st>>>(p, n, v);
    return cudaGetLastError();
}

__global__ void k_init_agg(uint64_t* slots, uint64_t n_words, uint32_t words) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_words;
         i += (uint64_t)gridDim.x * blockDim.x)
        slots[i] = (i % words == 0) ? EMPTY64 : 0ull;
}

cudaError_t launch_init_agg(uint64_t* slots, uint64_t n_slots, uint32_t words, cudaStream_t st) {
    const uint64_t n = n_slots * words;
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    k_init_agg<<<(unsigned)blocks, 256, 0, st>>>(slots, n, words);
    return cudaGetLastError();
}

// -------------------------------------------------------------------- build

__global__ void __launch_bounds__(256) k_build(const __grid_constant__ BuildDev b, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        build_insert(b, i);
}

cudaError_t launch_build(const BuildDev& b, uint64_t n, int num_sms, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    uint64_t cap = (uint64_t)num_sms * 8;
    if (blocks > cap) blocks = cap;
    k_build<<<(unsigned)blocks, 256, 0, st>>>(b, n);
    return cudaGetLastError();
}

// ------------------------------------------------- shared-memory aggregation
//
// Few groups (packed key of at most 12 bits): every CTA keeps a private dense
// table in shared memory indexed by the key itself -- count[G], then lo[G],
// hi[G] per sum -- updated with shared-memory atomics, and merges it into the
// global dense table (same layout) once at the end.

constexpr int AGG_THREADS = 512;

template <int NS>
__global__ void __launch_bounds__(AGG_THREADS) k_agg_shared(const __grid_constant__ QueryDev q,
                                                           uint64_t n, uint64_t* __restrict__ gacc,
                                                           uint32_t G) {
    extern __shared__ uint64_t sm[];
    const uint32_t words = G * (1 + 2 * NS);
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) sm[i] = 0;
    __syncthreads();
    uint64_t* cnt = sm;
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = blockDim.x >> 5;
    const uint64_t ntiles = (n + 127) / 128;
    const uint64_t nfull = n / 128;
    for (uint64_t t = blockIdx.x * nwarps + (threadIdx.x >> 5); t < ntiles; t += gridDim.x * nwarps) {
        const bool full = t < nfull;
        // fan-out joins pair a row with each partner in turn (m); otherwise one pass
        for (uint32_t m = 0;; ++m) {
            bool pass[4];
            uint64_t key[4];
            const bool any = full ? eval_keys<true>(q, t * 128, n, lane, pass, key, m)
                                  : eval_keys<false>(q, t * 128, n, lane, pass, key, m);
            if (!any) break;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (pass[i]) atomicAdd((unsigned long long*)&cnt[(uint32_t)key[i]], 1ull);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                I128 tm[4];
                if (full) eval_terms<true>(q, s, t * 128, n, lane, pass, tm);
                else eval_terms<false>(q, s, t * 128, n, lane, pass, tm);
                uint64_t* lo = sm + G * (1 + 2 * s);
                uint64_t* hi = sm + G * (2 + 2 * s);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (pass[i]) atomic_add_i128(lo + (uint32_t)key[i], hi + (uint32_t)key[i], tm[i]);
            }
            if (!q.jt.many) break;
        }
    }
    __syncthreads();
    for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) {
        const uint64_t c = cnt[g];
        if (c == 0) continue;
        atomicAdd((unsigned long long*)&gacc[g], (unsigned long long)c);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            I128 v{sm[G * (1 + 2 * s) + g], sm[G * (2 + 2 * s) + g]};
            atomic_add_i128(&gacc[G * (1 + 2 * s) + g], &gacc[G * (2 + 2 * s) + g], v);
        }
    }
}

size_t agg_shared_smem_bytes(uint32_t key_bits, int n_sum) {
    return (size_t)(1u << key_bits) * (1 + 2 * (size_t)n_sum) * sizeof(uint64_t);
}

template <int NS>
static void* agg_shared_fn() { return (void*)k_agg_shared<NS>; }

static void* agg_shared_kernel(int n_sum) {
    switch (n_sum) {
    case 0: return agg_shared_fn<0>();
    case 1: return agg_shared_fn<1>();
    case 2: return agg_shared_fn<2>();
    case 3: return agg_shared_fn<3>();
    case 4: return agg_shared_fn<4>();
    case 5: return agg_shared_fn<5>();
    case 6: return agg_shared_fn<6>();
    case 7: return agg_shared_fn<7>();
    default: return agg_shared_fn<8>();
    }
}

int agg_shared_grid(uint32_t key_bits, int n_sum, int num_sms) {
    size_t smem = agg_shared_smem_bytes(key_bits, n_sum);
    void* fn = agg_shared_kernel(n_sum);
    ensure_smem_limit(fn, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, AGG_THREADS, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return per_sm * num_sms;
}

cudaError_t launch_agg_shared(const QueryDev& q, uint64_t n, uint64_t* gacc, uint32_t key_bits,
                              int grid, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const uint32_t G = 1u << key_bits;
    const size_t smem = agg_shared_smem_bytes(key_bits, q.n_sum);
    uint64_t tiles = (n + 127) / 128;
    uint64_t need = (tiles + (AGG_THREADS / 32) - 1) / (AGG_THREADS / 32);
    unsigned blocks = (unsigned)(need < (uint64_t)grid ? need : (uint64_t)grid);
    switch (q.n_sum) {
#define TPK_CASE(K) \
    case K: k_agg_shared<K><<<blocks, AGG_THREADS, smem, st>>>(q, n, gacc, G); break;
    TPK_CASE(0) TPK_CASE(1) TPK_CASE(2) TPK_CASE(3) TPK_CASE(4) TPK_CASE(5) TPK_CASE(6) TPK_CASE(7) TPK_CASE(8)
#undef TPK_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------- global aggregation
//
// Many groups: one open-addressing table in device memory.  A lane merges its
// two pairs of adjacent rows first when their keys agree (clustered keys such
// as an order key repeated over consecutive line items), then claims or finds
// the slot and adds count and sums with 64-bit atomics.

template <int NS>
__global__ void __launch_bounds__(256) k_agg_global(const __grid_constant__ QueryDev q, uint64_t n,
                                                   const __grid_constant__ AggTable t) {
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = blockDim.x >> 5;
    const uint64_t ntiles = (n + 127) / 128;
    const uint64_t nfull = n / 128;
    uint32_t claims = 0;   // fresh slots this lane took, added to the table once per warp at the end
    for (uint64_t tt = blockIdx.x * nwarps + (threadIdx.x >> 5); tt < ntiles; tt += gridDim.x * nwarps) {
        const bool full = tt < nfull;
        // fan-out joins pair a row with each partner in turn (m); otherwise one pass
        for (uint32_t m = 0;; ++m) {
            bool pass[4];
            uint64_t key[4];
            const bool any = full ? eval_keys<true>(q, tt * 128, n, lane, pass, key, m)
                                  : eval_keys<false>(q, tt * 128, n, lane, pass, key, m);
            if (!any) break;
            // rows (0,1) and (2,3) are adjacent: fold the second into the first
            // when their keys agree
            bool fold[2];
            uint64_t* slot[4];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                fold[j] = pass[2 * j] && pass[2 * j + 1] && key[2 * j] == key[2 * j + 1];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                slot[i] = nullptr;
                if (!pass[i] || ((i & 1) && fold[i >> 1])) continue;
                bool claimed;
                slot[i] = agg_slot_any(t, key[i], q.err, claimed);
                claims += claimed ? 1u : 0u;
                if (slot[i])
                    atomicAdd((unsigned long long*)(slot[i] + 1), (i & 1) == 0 && fold[i >> 1] ? 2ull : 1ull);
            }
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                I128 tm[4];
                if (full) eval_terms<true>(q, s, tt * 128, n, lane, pass, tm);
                else eval_terms<false>(q, s, tt * 128, n, lane, pass, tm);
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    if (fold[j]) tm[2 * j] = i128_add(tm[2 * j], tm[2 * j + 1]);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (slot[i]) atomic_add_i128(slot[i] + 2 + 2 * s, slot[i] + 3 + 2 * s, tm[i]);
            }
            if (!q.jt.many) break;
        }
    }
    agg_add_claims_warp(t, q.err, claims);
}

cudaError_t launch_agg_global(const QueryDev& q, uint64_t n, const AggTable& t, int num_sms,
                              cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    uint64_t tiles = (n + 127) / 128;
    uint64_t need = (tiles + 7) / 8;
    uint64_t cap = (uint64_t)num_sms * 8;
    unsigned blocks = (unsigned)(need < cap ? need : cap);
    switch (q.n_sum) {
#define TPK_CASE(K) \
    case K: k_agg_global<K><<<blocks, 256, 0, st>>>(q, n, t); break;
    TPK_CASE(0) TPK_CASE(1) TPK_CASE(2) TPK_CASE(3) TPK_CASE(4) TPK_CASE(5) TPK_CASE(6) TPK_CASE(7) TPK_CASE(8)
#undef TPK_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- finalise

// One CTA walks the dense table in key order, so the output is sorted.
__global__ void __launch_bounds__(1024) k_final_dense(const uint64_t* __restrict__ gacc, uint32_t G,
                                                     int n_sum, const __grid_constant__ OutDev o, int lo_only) {
    final_dense_block(gacc, G, n_sum, o, lo_only != 0);
}

cudaError_t launch_final_dense(const uint64_t* gacc, uint32_t key_bits, int n_sum, const OutDev& o,
                               cudaStream_t st, bool lo_only) {
    k_final_dense<<<1, 1024, 0, st>>>(gacc, 1u << key_bits, n_sum, o, lo_only ? 1 : 0);
    return cudaGetLastError();
}

// Occupied slots of the global table -> (key, slot index); also the max key.
// ------------------------------------------------------------ narrow pages

__device__ __forceinline__ void store_widened(void* dst, int out, uint64_t i, uint64_t v) {
    if (out == 8) ((int64_t*)dst)[i] = (int64_t)v;
    else if (out == 4) ((int32_t*)dst)[i] = (int32_t)(uint32_t)v;
    else ((uint8_t*)dst)[i] = (uint8_t)v;
}

// Each thread widens DECODE_PER rows per round (rows i, i + T, ... for T
// threads in the grid, so every load and store stays coalesced), with all of
// their loads issued before the first store.
constexpr int DECODE_PER = 4;

template <typename U>
__device__ __forceinline__ void decode_col(const U* __restrict__ src, int64_t base, void* dst, int out,
                                           uint64_t rows) {
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < rows; i0 += DECODE_PER * T) {
        U v[DECODE_PER];
#pragma unroll
        for (int k = 0; k < DECODE_PER; ++k)
            if (i0 + k * T < rows) v[k] = __ldcs(src + i0 + k * T);
#pragma unroll
        for (int k = 0; k < DECODE_PER; ++k)
            if (i0 + k * T < rows) store_widened(dst, out, i0 + k * T, (uint64_t)base + (uint64_t)v[k]);
    }
}

// Row i's value sits at bit bit0 + i * bits of the word stream starting at
// the 4-byte-aligned address at or below src (bit0 = 8 * the misalignment);
// the word after the value's first is read only when the value reaches into
// it, so no word beyond the stream's last is touched.
__device__ __forceinline__ void decode_bits(const uint8_t* src, int bits, int64_t base, void* dst, int out,
                                            uint64_t rows) {
    const uint32_t* w = (const uint32_t*)((uintptr_t)src & ~(uintptr_t)3);
    const uint64_t bit0 = 8 * ((uintptr_t)src & 3);
    const uint32_t mask = (1u << bits) - 1u;   // bits <= 31
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < rows; i0 += DECODE_PER * T) {
        uint32_t lo[DECODE_PER], hi[DECODE_PER], sh[DECODE_PER];
#pragma unroll
        for (int r = 0; r < DECODE_PER; ++r) {
            const uint64_t i = i0 + r * T;
            lo[r] = hi[r] = sh[r] = 0;
            if (i >= rows) continue;
            const uint64_t at = bit0 + i * (uint64_t)bits;
            const uint64_t k = at >> 5;
            sh[r] = (uint32_t)(at & 31);
            lo[r] = __ldg(w + k);
            if (sh[r] + (uint32_t)bits > 32) hi[r] = __ldg(w + k + 1);
        }
#pragma unroll
        for (int r = 0; r < DECODE_PER; ++r) {
            const uint64_t i = i0 + r * T;
            if (i >= rows) continue;
            uint32_t v = lo[r] >> sh[r];
            if (sh[r] + (uint32_t)bits > 32) v |= hi[r] << (32 - sh[r]);
            store_widened(dst, out, i, (uint64_t)base + (uint64_t)(v & mask));
        }
    }
}

__global__ void k_decode(const __grid_constant__ DecodeCols d) {
    for (int c = 0; c < d.n; ++c) {
        if (d.bits[c]) {
            decode_bits((const uint8_t*)d.src[c], d.bits[c], d.base[c], d.dst[c], d.out[c], d.rows[c]);
            continue;
        }
        switch (d.w[c]) {
        case 1: decode_col((const uint8_t*)d.src[c], d.base[c], d.dst[c], d.out[c], d.rows[c]); break;
        case 2: decode_col((const uint16_t*)d.src[c], d.base[c], d.dst[c], d.out[c], d.rows[c]); break;
        default: decode_col((const uint32_t*)d.src[c], d.base[c], d.dst[c], d.out[c], d.rows[c]); break;
        }
    }
}

cudaError_t launch_decode(const DecodeCols& d, int num_sms, cudaStream_t st) {
    uint64_t rows = 0;
    for (int c = 0; c < d.n; ++c) rows = std::max<uint64_t>(rows, d.rows[c]);
    if (rows == 0) return cudaSuccess;
    const uint64_t blocks = std::min<uint64_t>((rows + 255) / 256, (uint64_t)num_sms * 4);
    k_decode<<<(unsigned)blocks, 256, 0, st>>>(d);
    return cudaGetLastError();
}

// ------------------------------------------------------------ direct tables

// Occupied slots (count word non-zero) of each chunk of DIRECT_CHUNK slots.
__global__ void k_direct_count(const __grid_constant__ AggTable t, uint64_t n_slots, uint32_t* __restrict__ counts) {
    __shared__ uint32_t warp_sum[32];
    const uint64_t n_chunks = (n_slots + DIRECT_CHUNK - 1) / DIRECT_CHUNK;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        uint32_t n = 0;
        for (uint32_t i = threadIdx.x; i < DIRECT_CHUNK; i += blockDim.x) {
            const uint64_t s = c * DIRECT_CHUNK + i;
            if (s < n_slots && t.slots[s * t.words + 1] != 0) ++n;
        }
        for (int off = 16; off > 0; off >>= 1) n += __shfl_xor_sync(0xffffffffu, n, off);
        if (lane == 0) warp_sum[warp] = n;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += warp_sum[w];
            counts[c] = tot;
        }
        __syncthreads();
    }
}

cudaError_t launch_direct_count(const AggTable& t, uint64_t n_slots, uint32_t* counts, int num_sms,
                                cudaStream_t st) {
    if (n_slots == 0) return cudaSuccess;
    const uint64_t n_chunks = (n_slots + DIRECT_CHUNK - 1) / DIRECT_CHUNK;
    const uint64_t blocks = std::min<uint64_t>(n_chunks, (uint64_t)num_sms * 8);
    k_direct_count<<<(unsigned)blocks, 256, 0, st>>>(t, n_slots, counts);
    return cudaGetLastError();
}

// Exclusive scan of the chunk counts by one CTA; offsets[n_chunks] = total.
__global__ void k_direct_scan(const uint32_t* __restrict__ counts, uint64_t n_chunks,
                              unsigned long long* __restrict__ offsets) {
    __shared__ unsigned long long part[1024];
    const uint64_t per = (n_chunks + blockDim.x - 1) / blockDim.x;
    const uint64_t b = threadIdx.x * per, e = b + per < n_chunks ? b + per : n_chunks;
    unsigned long long sum = 0;
    for (uint64_t i = b; i < e; ++i) sum += counts[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (uint32_t i = 0; i < blockDim.x; ++i) {
            const unsigned long long v = part[i];
            part[i] = run;
            run += v;
        }
        offsets[n_chunks] = run;
    }
    __syncthreads();
    unsigned long long run = part[threadIdx.x];
    for (uint64_t i = b; i < e; ++i) {
        offsets[i] = run;
        run += counts[i];
    }
}

cudaError_t launch_direct_scan(const uint32_t* counts, uint64_t n_chunks, unsigned long long* offsets,
                               cudaStream_t st) {
    k_direct_scan<<<1, 1024, 0, st>>>(counts, n_chunks, offsets);
    return cudaGetLastError();
}

// Each chunk writes its occupied slots in slot (= key) order at its offset.
__global__ void k_direct_emit(const __grid_constant__ AggTable t, uint64_t n_slots,
                              const unsigned long long* __restrict__ offsets, int n_sum,
                              const __grid_constant__ OutDev o, int lo_only) {
    __shared__ uint32_t warp_tot[32];
    __shared__ unsigned long long base;
    const uint64_t n_chunks = (n_slots + DIRECT_CHUNK - 1) / DIRECT_CHUNK;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (uint64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        if (threadIdx.x == 0) base = offsets[c];
        __syncthreads();
        for (uint32_t i0 = 0; i0 < DIRECT_CHUNK; i0 += blockDim.x) {
            const uint64_t s = c * DIRECT_CHUNK + i0 + threadIdx.x;
            const uint64_t* p = t.slots + s * t.words;
            const bool has = s < n_slots && p[1] != 0;
            const unsigned m = __ballot_sync(0xffffffffu, has);
            if (lane == 0) warp_tot[warp] = __popc(m);
            __syncthreads();
            uint32_t before = 0, total = 0;
            for (int w = 0; w < nwarps; ++w) {
                if (w < warp) before += warp_tot[w];
                total += warp_tot[w];
            }
            if (has) {
                uint64_t lh[2 * MAX_SUM];
                for (int x = 0; x < n_sum; ++x) {
                    lh[2 * x] = p[2 + 2 * x];
                    lh[2 * x + 1] = lo_only ? (uint64_t)((int64_t)lh[2 * x] >> 63) : p[3 + 2 * x];
                }
                write_row(o, base + before + __popc(m & ((1u << lane) - 1u)), s + t.kmin, p[1], lh, n_sum);
            }
            __syncthreads();
            if (threadIdx.x == 0) base += total;
            __syncthreads();
        }
    }
}

cudaError_t launch_direct_emit(const AggTable& t, uint64_t n_slots, const unsigned long long* offsets, int n_sum,
                               const OutDev& o, bool lo_only, int num_sms, cudaStream_t st) {
    if (n_slots == 0) return cudaSuccess;
    const uint64_t n_chunks = (n_slots + DIRECT_CHUNK - 1) / DIRECT_CHUNK;
    const uint64_t blocks = std::min<uint64_t>(n_chunks, (uint64_t)num_sms * 8);
    k_direct_emit<<<(unsigned)blocks, 256, 0, st>>>(t, n_slots, offsets, n_sum, o, lo_only ? 1 : 0);
    return cudaGetLastError();
}

// Occupied slots of a hashed global table as (key, slot) pairs, in no
// particular order (a sort by key follows), plus the largest key.  A CTA
// takes COMPACT_PER * 256 slots at a time (slot = chunk + i * 256 + thread,
// coalesced), ranks its occupied ones with a block scan and reserves their
// output range with one atomic, so the shared counter sees one update per
// chunk instead of one per warp.
constexpr int COMPACT_PER = 8;

__global__ void __launch_bounds__(256) k_compact_global(const __grid_constant__ AggTable t, uint64_t cap_with_side,
                                                        uint64_t* __restrict__ keys, uint32_t* __restrict__ idx,
                                                        unsigned long long* count, unsigned long long* maxkey) {
    __shared__ uint32_t warp_sums[8];
    __shared__ unsigned long long base_s;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long local_max = 0;
    const uint64_t per_chunk = (uint64_t)COMPACT_PER * 256;
    const uint64_t n_chunks = (cap_with_side + per_chunk - 1) / per_chunk;
    for (uint64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        uint32_t occ = 0;
        uint64_t key[COMPACT_PER];
        ulonglong2 kc[COMPACT_PER];   // {key, count} of each slot, all loads in flight at once
#pragma unroll
        for (int i = 0; i < COMPACT_PER; ++i) {
            const uint64_t s = ch * per_chunk + (uint64_t)i * 256 + threadIdx.x;
            kc[i] = s < cap_with_side ? __ldcs((const ulonglong2*)(t.slots + s * t.words)) : make_ulonglong2(0, 0);
        }
#pragma unroll
        for (int i = 0; i < COMPACT_PER; ++i) {
            const uint64_t s = ch * per_chunk + (uint64_t)i * 256 + threadIdx.x;
            key[i] = 0;
            if (kc[i].y != 0) {
                occ |= 1u << i;
                key[i] = (s == cap_with_side - 1) ? EMPTY64 : kc[i].x;
            }
        }
        // block-wide exclusive scan of the occupied counts
        const uint32_t c = (uint32_t)__popc(occ);
        uint32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) warp_sums[w] = inc;
        __syncthreads();
        uint32_t before = 0, all = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            before += k < w ? warp_sums[k] : 0u;
            all += warp_sums[k];
        }
        if (threadIdx.x == 0) base_s = all ? atomicAdd(count, (unsigned long long)all) : 0ull;
        __syncthreads();
        uint64_t pos = base_s + before + inc - c;
#pragma unroll
        for (int i = 0; i < COMPACT_PER; ++i) {
            if (!(occ >> i & 1u)) continue;
            keys[pos] = key[i];
            idx[pos] = (uint32_t)(ch * per_chunk + (uint64_t)i * 256 + threadIdx.x);
            ++pos;
            if (key[i] > local_max) local_max = key[i];
        }
        __syncthreads();   // warp_sums and base_s are reused by the next chunk
    }
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, local_max, off);
        if (o > local_max) local_max = o;
    }
    if (lane == 0 && local_max) atomicMax(maxkey, local_max);
}

cudaError_t launch_compact_global(const AggTable& t, uint64_t cap_with_side, uint64_t* keys,
                                  uint32_t* idx, unsigned long long* count,
                                  unsigned long long* maxkey, int num_sms, cudaStream_t st) {
    // as many CTAs as are resident at once: each takes a fixed share of the
    // chunks, so a second, partial wave would leave SMs idle at the end
    static const int per_sm = [] {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void*)k_compact_global, 256, 0) != cudaSuccess ||
            n < 1) {
            cudaGetLastError();
            n = 1;
        }
        return n;
    }();
    uint64_t blocks = (cap_with_side + COMPACT_PER * 256 - 1) / (COMPACT_PER * 256);
    const uint64_t cap = (uint64_t)num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    k_compact_global<<<(unsigned)blocks, 256, 0, st>>>(t, cap_with_side, keys, idx, count, maxkey);
    return cudaGetLastError();
}

// Rows of the sorted output: GATHER_PER rows per thread, every index and key
// load, then every slot load, in flight before the first row is written.  A
// 32-byte slot (one sum) is read with one 256-bit load (sm_100 and later):
// a random slot then costs one L1 lookup per lane instead of three.
constexpr int GATHER_PER = 4;

__device__ __forceinline__ void ld_slot4(const uint64_t* p, uint64_t (&w)[4]) {
    asm("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(w[0]), "=l"(w[1]), "=l"(w[2]), "=l"(w[3]) : "l"(p));
}

__global__ void __launch_bounds__(256) k_gather_global(const __grid_constant__ AggTable t,
                                                       const uint64_t* __restrict__ skeys,
                                                       const uint32_t* __restrict__ sidx, uint64_t n, int n_sum,
                                                       const __grid_constant__ OutDev o, int lo_only) {
    const bool v4 = t.words == 4 && ((uintptr_t)t.slots & 31u) == 0;
    const uint64_t per = (uint64_t)GATHER_PER * blockDim.x;
    for (uint64_t b = blockIdx.x * per; b < n; b += (uint64_t)gridDim.x * per) {
        uint64_t key[GATHER_PER];
        uint32_t at[GATHER_PER];
#pragma unroll
        for (int r = 0; r < GATHER_PER; ++r) {
            const uint64_t i = b + (uint64_t)r * blockDim.x + threadIdx.x;
            at[r] = 0;
            key[r] = 0;
            if (i < n) {
                at[r] = sidx[i];
                key[r] = skeys[i];
            }
        }
        if (v4) {
            uint64_t w[GATHER_PER][4];
#pragma unroll
            for (int r = 0; r < GATHER_PER; ++r)
                if (b + (uint64_t)r * blockDim.x + threadIdx.x < n) ld_slot4(t.slots + (uint64_t)at[r] * 4, w[r]);
#pragma unroll
            for (int r = 0; r < GATHER_PER; ++r) {
                const uint64_t i = b + (uint64_t)r * blockDim.x + threadIdx.x;
                if (i >= n) continue;
                const uint64_t lh[2] = {w[r][2], lo_only ? (uint64_t)((int64_t)w[r][2] >> 63) : w[r][3]};
                write_row(o, i, key[r], w[r][1], lh, 1);
            }
        } else {
#pragma unroll
            for (int r = 0; r < GATHER_PER; ++r) {
                const uint64_t i = b + (uint64_t)r * blockDim.x + threadIdx.x;
                if (i >= n) continue;
                const uint64_t* p = t.slots + (uint64_t)at[r] * t.words;
                uint64_t lh[2 * MAX_SUM];
                for (int s = 0; s < n_sum; ++s) {
                    lh[2 * s] = p[2 + 2 * s];
                    lh[2 * s + 1] = lo_only ? (uint64_t)((int64_t)lh[2 * s] >> 63) : p[3 + 2 * s];
                }
                write_row(o, i, key[r], p[1], lh, n_sum);
            }
        }
    }
}

cudaError_t launch_gather_global(const AggTable& t, const uint64_t* sorted_keys,
                                 const uint32_t* sorted_idx, uint64_t n, int n_sum, const OutDev& o,
                                 int num_sms, cudaStream_t st, bool lo_only) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + GATHER_PER * 256 - 1) / (GATHER_PER * 256);
    uint64_t cap = (uint64_t)num_sms * 8;
    if (blocks > cap) blocks = cap;
    k_gather_global<<<(unsigned)blocks, 256, 0, st>>>(t, sorted_keys, sorted_idx, n, n_sum, o, lo_only ? 1 : 0);
    return cudaGetLastError();
}

// --------------------------------------------------- selectivity sampling

__global__ void k_sample_filter(const __grid_constant__ QueryDev q, uint64_t n, uint32_t samples,
                                unsigned long long* out) {
    unsigned local = 0;
    for (uint32_t j = threadIdx.x; j < samples; j += blockDim.x) {
        const uint64_t row = (uint64_t)(((unsigned __int128)j * n) / samples);
        const int64_t v = ld1(q.fcol, row);
        local += (v >= q.flo && v <= q.fhi) ? 1u : 0u;
    }
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(out, (unsigned long long)local);
}

cudaError_t launch_sample_filter(const QueryDev& q, uint64_t n, uint32_t samples,
                                 unsigned long long* out, cudaStream_t st) {
    if (n == 0 || samples == 0) return cudaSuccess;
    k_sample_filter<<<1, 256, 0, st>>>(q, n, samples, out);
    return cudaGetLastError();
}

// ------------------------------------------------------- column statistics

__global__ void k_minmax(const __grid_constant__ DevCol c, uint64_t n, long long* out) {
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const long long v = ld1(c, i);
        lo = v < lo ? v : lo;
        hi = v > hi ? v : hi;
    }
    for (int off = 16; off > 0; off >>= 1) {
        const long long a = __shfl_xor_sync(0xffffffffu, lo, off);
        const long long b = __shfl_xor_sync(0xffffffffu, hi, off);
        lo = a < lo ? a : lo;
        hi = b > hi ? b : hi;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(out, lo);
        atomicMax(out + 1, hi);
    }
}

cudaError_t launch_minmax(const DevCol& c, uint64_t n, long long* out, int num_sms, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    const uint64_t cap = (uint64_t)num_sms * 4;
    if (blocks > cap) blocks = cap;
    k_minmax<<<(unsigned)blocks, 256, 0, st>>>(c, n, out);
    return cudaGetLastError();
}

cudaError_t load_plain_kernels() {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_build);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_final_dense);
#define TPK_LOAD(K) \
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_agg_shared<K>);
    TPK_LOAD(0) TPK_LOAD(1) TPK_LOAD(2) TPK_LOAD(3) TPK_LOAD(4) TPK_LOAD(5) TPK_LOAD(6) TPK_LOAD(7) TPK_LOAD(8)
#undef TPK_LOAD
    return e;
}

}  // namespace tpk
