// Many-group aggregation under a selective filter: a selection pass, then a
// gather pass over the selected rows only.
//
// Paper basis: Section 3.1 (operators run GPU kernels over batches of
// equal-length columns), Section 3.2 (join), Section 4 (decimals held as
// 128-bit integers).  The split is this library's design for GB300.  Fused
// into one scan, a 1%-selective query leaves most lanes idle while the few
// surviving rows wait on their dependent loads (foreign key, join table,
// group key, aggregation slot), and the filter column streams only as fast as
// those chains complete.  Here:
//
//  * k_select streams the filter column alone with 16-byte vector loads at
//    HBM rate and writes the batch-relative indices of the passing rows to a
//    selection vector.  A chunk's passing rows get their output range from
//    one atomic per CTA-chunk and stay in ascending row order inside it.
//  * k_agg_selected gives every lane SEL_RPL selected rows, so all lanes issue
//    their gathers, probes and table updates together; equal keys among a
//    warp's rows (consecutive rows of one order key) are combined first
//    (agg_warp.cuh), and hashed-table claims are counted once per warp.  The
//    join probe (probe4) takes exactly four rows, so SEL_RPL is four.
#include <algorithm>
#include <type_traits>

#include "agg_warp.cuh"

namespace tpk {

constexpr int SEL_THREADS = 256;
constexpr int SEL_LOADS = 4;   // 16-byte loads per thread per chunk

template <int T>
struct SelVec;
template <>
struct SelVec<T_I32> {
    typedef int4 V;
    static constexpr int N = 4;
    __device__ static uint32_t at(const V& v, int k) {
        return (uint32_t)(k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w);
    }
};
template <>
struct SelVec<T_I64> {
    typedef longlong2 V;
    static constexpr int N = 2;
    __device__ static uint64_t at(const V& v, int k) { return (uint64_t)(k == 0 ? v.x : v.y); }
};
template <>
struct SelVec<T_U8> {
    typedef uint4 V;
    static constexpr int N = 16;
    __device__ static uint32_t at(const V& v, int k) {
        const uint32_t w = k < 4 ? v.x : k < 8 ? v.y : k < 12 ? v.z : v.w;
        return (w >> (8 * (k & 3))) & 0xFFu;
    }
};

// lo <= x <= hi as one unsigned compare: x - lo (mod 2^bits) <= hi - lo, for
// bounds already clamped to the column type's range with lo <= hi.
template <int T>
struct SelRange {
    typedef typename std::conditional<T == T_I64, uint64_t, uint32_t>::type W;
    W lo, span;
    bool none;   // no value of the type lies in [lo, hi]
    __device__ SelRange(int64_t flo, int64_t fhi) {
        const int64_t tmin = T == T_I64 ? INT64_MIN : (T == T_I32 ? (int64_t)INT32_MIN : 0);
        const int64_t tmax = T == T_I64 ? INT64_MAX : (T == T_I32 ? (int64_t)INT32_MAX : 255);
        const int64_t l = flo < tmin ? tmin : flo, h = fhi > tmax ? tmax : fhi;
        none = flo > fhi || l > h;
        lo = (W)(uint64_t)l;
        span = none ? (W)0 : (W)((uint64_t)h - (uint64_t)l);
    }
    __device__ bool in(W x) const { return !none && (W)(x - lo) <= span; }
};

// Block-wide exclusive scan of x (every thread of the CTA calls it); *total
// gets the sum over the CTA.  Fields packed in x add independently as long as
// none overflows.
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t x, uint64_t* total, uint64_t* warp_sums) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    uint64_t before = 0, all = 0;
#pragma unroll
    for (int i = 0; i < SEL_THREADS / 32; ++i) {
        const uint64_t v = warp_sums[i];
        before += i < w ? v : 0;
        all += v;
    }
    *total = all;
    return before + inc - x;
}

// Indices (batch-relative) of the rows of [0, n) whose filter value lies in
// [lo, hi], appended at sel[*cursor]; the caller sized sel for n rows.
// A chunk is SEL_LOADS vectors per thread: row (i * SEL_THREADS + t) * N + k
// is element k of thread t's i-th vector, so (i, t, k) order is row order.
template <int T>
__global__ void __launch_bounds__(SEL_THREADS) k_select(const __grid_constant__ DevCol c, int64_t lo, int64_t hi,
                                                        uint64_t n, uint32_t* __restrict__ sel,
                                                        unsigned long long* cursor) {
    typedef SelVec<T> SV;
    constexpr int N = SV::N;
    constexpr uint64_t CH = (uint64_t)SEL_LOADS * SEL_THREADS * N;
    __shared__ uint64_t warp_sums[SEL_THREADS / 32];
    __shared__ unsigned long long base_s;
    const typename SV::V* src = (const typename SV::V*)c.ptr;
    const SelRange<T> rg(lo, hi);
    const uint64_t n_chunks = (n + CH - 1) / CH;
    const uint64_t n_full = n / CH;
    // the next whole chunk's vectors are loaded while this one is ranked and
    // written, so a CTA keeps a chunk of loads in flight throughout
    typename SV::V nxt[SEL_LOADS];
    auto load_chunk = [&](uint64_t ch) {
#pragma unroll
        for (int i = 0; i < SEL_LOADS; ++i) nxt[i] = __ldcs(src + ch * CH / N + (uint64_t)i * SEL_THREADS + threadIdx.x);
    };
    if (blockIdx.x < n_full) load_chunk(blockIdx.x);
    for (uint64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const uint64_t r0 = ch * CH;
        uint32_t m[SEL_LOADS];   // pass bits of each vector
        if (ch < n_full) {
            typename SV::V v[SEL_LOADS];
#pragma unroll
            for (int i = 0; i < SEL_LOADS; ++i) v[i] = nxt[i];
            if (ch + gridDim.x < n_full) load_chunk(ch + gridDim.x);
#pragma unroll
            for (int i = 0; i < SEL_LOADS; ++i) {
                m[i] = 0;
#pragma unroll
                for (int k = 0; k < N; ++k) m[i] |= (uint32_t)rg.in(SV::at(v[i], k)) << k;
            }
        } else {   // the last, partial chunk
#pragma unroll
            for (int i = 0; i < SEL_LOADS; ++i) {
                m[i] = 0;
                const uint64_t rb = r0 + ((uint64_t)i * SEL_THREADS + threadIdx.x) * N;
                for (int k = 0; k < N; ++k) {
                    if (rb + k >= n) break;
                    m[i] |= (uint32_t)rg.in((typename SelRange<T>::W)(uint64_t)ld1(c, rb + k)) << k;
                }
            }
        }
        // per-vector counts in 16-bit fields (each field sums to at most CH / SEL_LOADS)
        uint64_t packed = 0;
#pragma unroll
        for (int i = 0; i < SEL_LOADS; ++i) packed |= (uint64_t)__popc(m[i]) << (16 * i);
        uint64_t tot;
        const uint64_t ex = block_excl_scan(packed, &tot, warp_sums);
        if (threadIdx.x == 0) {
            uint64_t all = 0;
#pragma unroll
            for (int i = 0; i < SEL_LOADS; ++i) all += (tot >> (16 * i)) & 0xFFFFu;
            base_s = all ? atomicAdd(cursor, (unsigned long long)all) : 0ull;
        }
        __syncthreads();
        uint64_t off = base_s;
#pragma unroll
        for (int i = 0; i < SEL_LOADS; ++i) {
            uint64_t o = off + ((ex >> (16 * i)) & 0xFFFFu);
            uint32_t bits = m[i];
            const uint64_t rb = r0 + ((uint64_t)i * SEL_THREADS + threadIdx.x) * N;
            while (bits) {
                const int k = __ffs(bits) - 1;
                bits &= bits - 1u;
                sel[o++] = (uint32_t)(rb + k);
            }
            off += (tot >> (16 * i)) & 0xFFFFu;
        }
        __syncthreads();   // warp_sums and base_s are reused by the next chunk
    }
}

// The selected rows' join, group key and terms, SEL_RPL rows per lane
// (entries e0 + 32 j + lane of the selection vector), then warp-aggregated
// table updates.  *count selected rows; the filter is not evaluated again.
constexpr int SEL_RPL = 4;
template <int NS, bool FAST>
__global__ void __launch_bounds__(256, 2) k_agg_selected(const __grid_constant__ QueryDev q,
                                                      const uint32_t* __restrict__ sel,
                                                      const unsigned long long* count,
                                                      const __grid_constant__ AggTable tab) {
    constexpr int R = SEL_RPL;
    static_assert(R == 4, "probe4 probes exactly four rows per lane");
    constexpr int NSX = NS > 0 ? NS : 1;
    const uint64_t cnt = *count;
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t claims = 0;
    for (uint64_t e0 = gw * 32 * R; e0 < cnt; e0 += nw * 32 * R) {
        bool pass[R];
        uint64_t row[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const uint64_t e = e0 + 32 * j + lane;
            pass[j] = e < cnt;
            row[j] = pass[j] ? (uint64_t)__ldcs(sel + e) : 0;
        }
        // every column of the selected rows in flight at once: the rows
        // passed the filter, so all of them are needed unless the join drops
        // the row
        // fact-side group fields go straight to their bit positions of the
        // packed key (first field highest); dimension fields follow the probe
        int64_t fk[R], a[NSX][R], b[NSX][R];
        uint64_t key[R];
        bool bad[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            key[j] = 0;
            bad[j] = false;
        }
#pragma unroll
        for (int j = 0; j < R; ++j) fk[j] = (q.has_join && pass[j]) ? ld1(q.fk, row[j]) : 0;
        {
            int shift = 0;
            for (int g = q.n_group - 1; g >= 0; --g) {
                const int bits = q.gbits[g];
                if (q.gside[g] == 0) {
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        const uint64_t f = pass[j] ? (uint64_t)ld1(q.gcol[g], row[j]) : 0;
                        if (bits < 64) {
                            bad[j] = bad[j] || (f >> bits) != 0;
                            key[j] |= f << shift;
                        } else {
                            key[j] = f;
                        }
                    }
                }
                shift += bits;
            }
        }
#pragma unroll
        for (int s = 0; s < NSX; ++s) {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const bool on = s < q.n_sum && pass[j];
                a[s][j] = on ? ld1(q.sa[s], row[j]) : 0;
                b[s][j] = (on && q.skind[s] == S_MUL_SUB) ? ld1(q.sb[s], row[j]) : 0;
            }
        }
        uint32_t pay[R];
#pragma unroll
        for (int j = 0; j < R; ++j) pay[j] = 0;
        if (q.has_join) {
            probe4<true>(q.jt, fk, pass, pay, q.err);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (pass[j] && (pay[j] & PAYLOAD_BAD)) {
                    atomicOr(q.err, ERR_RANGE);
                    pass[j] = false;
                }
            }
        }
        {
            int shift = 0;
            for (int g = q.n_group - 1; g >= 0; --g) {
                const int bits = q.gbits[g];
                if (q.gside[g] != 0) {   // dimension fields fit their bits by construction of the payload
#pragma unroll
                    for (int j = 0; j < R; ++j) key[j] |= ((uint64_t)(pay[j] >> q.gdpos[g]) & ((1ull << bits) - 1ull))
                                                          << shift;
                }
                shift += bits;
            }
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (pass[j] && bad[j]) {
                atomicOr(q.err, ERR_RANGE);
                pass[j] = false;
            }
        }
        int64_t t[NSX][R];
        I128 tm[NSX][R];
#pragma unroll
        for (int s = 0; s < NSX; ++s) {
            const bool ms = q.skind[s] == S_MUL_SUB;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if constexpr (FAST) t[s][j] = ms ? a[s][j] * (q.sk[s] - b[s][j]) : a[s][j];
                else tm[s][j] = ms ? mul_sub(a[s][j], q.sk[s], b[s][j]) : i128_from_i64(a[s][j]);
            }
        }
        agg_warp_rows<NS, FAST, R>(tab, q.err, q.n_sum, pass, key, t, tm, claims);
    }
    agg_add_claims_warp(tab, q.err, claims);
}

// ------------------------------------------------------------------- host

bool select_usable(const QueryDev& q, uint64_t n) {
    return q.has_filter && q.n_xjoin == 0 && !q.jt.many && n < (1ull << 32) &&
           ((uintptr_t)q.fcol.ptr & 15u) == 0;
}

// CTAs of `fn` (block of `threads`, no dynamic shared memory) resident on
// one SM at once; a grid of at most that many per SM runs in one wave, so no
// CTA starts its fixed share of the chunks only after others finished theirs.
static int resident_ctas(const void* fn, int threads) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

template <int T>
static void select_t(const QueryDev& q, uint64_t n, uint32_t* sel, unsigned long long* cursor, uint64_t chunks,
                     int num_sms, cudaStream_t st) {
    static const int per_sm = resident_ctas((const void*)k_select<T>, SEL_THREADS);
    const unsigned grid = (unsigned)std::min<uint64_t>(chunks, (uint64_t)num_sms * per_sm);
    k_select<T><<<grid, SEL_THREADS, 0, st>>>(q.fcol, q.flo, q.fhi, n, sel, cursor);
}

cudaError_t launch_select(const QueryDev& q, uint64_t n, uint32_t* sel, unsigned long long* cursor, int num_sms,
                          cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int per = q.fcol.type == T_I32 ? 4 : (q.fcol.type == T_I64 ? 2 : 16);
    const uint64_t ch = (uint64_t)SEL_LOADS * SEL_THREADS * per;
    const uint64_t chunks = (n + ch - 1) / ch;
    switch (q.fcol.type) {
    case T_I32: select_t<T_I32>(q, n, sel, cursor, chunks, num_sms, st); break;
    case T_I64: select_t<T_I64>(q, n, sel, cursor, chunks, num_sms, st); break;
    default: select_t<T_U8>(q, n, sel, cursor, chunks, num_sms, st); break;
    }
    return cudaGetLastError();
}

template <int NS, bool FAST>
static cudaError_t launch_selected_t(const QueryDev& q, const uint32_t* sel, const unsigned long long* count,
                                     const AggTable& t, unsigned grid, cudaStream_t st) {
    k_agg_selected<NS, FAST><<<grid, 256, 0, st>>>(q, sel, count, t);
    return cudaGetLastError();
}

cudaError_t launch_agg_selected(const QueryDev& q, const uint32_t* sel, const unsigned long long* count,
                                uint64_t max_rows, const AggTable& t, bool fast, int num_sms, cudaStream_t st) {
    if (max_rows == 0) return cudaSuccess;
    // one warp per 32 * SEL_RPL selected rows at most, at most 8 CTAs per SM
    const uint64_t warps = (max_rows + 32 * SEL_RPL - 1) / (32 * SEL_RPL);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((warps + 7) / 8, (uint64_t)num_sms * 8));
    const int ns = q.n_sum;
    if (fast) {
        if (ns <= 1) return launch_selected_t<1, true>(q, sel, count, t, grid, st);
        if (ns <= 2) return launch_selected_t<2, true>(q, sel, count, t, grid, st);
        if (ns <= 4) return launch_selected_t<4, true>(q, sel, count, t, grid, st);
        return launch_selected_t<8, true>(q, sel, count, t, grid, st);
    }
    if (ns <= 1) return launch_selected_t<1, false>(q, sel, count, t, grid, st);
    if (ns <= 2) return launch_selected_t<2, false>(q, sel, count, t, grid, st);
    if (ns <= 4) return launch_selected_t<4, false>(q, sel, count, t, grid, st);
    return launch_selected_t<8, false>(q, sel, count, t, grid, st);
}

}  // namespace tpk
