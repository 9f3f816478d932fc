// Plan-specialised staged dense aggregation, compiled at run time (NVRTC).
//
// Paper basis: Section 3.1 (operators run GPU kernels over batches of
// equal-length columns), Section 3.2 (join), Section 4 (decimals held as
// 128-bit integers).  The pipeline is the one of the ahead-of-time staged
// kernel: one producer lane streams each tile's columns into an mbarrier ring
// with bulk copies, consumer warps evaluate 32 * ST_RPL rows of a stage each,
// groups accumulate in a per-CTA dense table in shared memory, and the table
// is folded into the global dense table at the end.  What differs: the plan's
// shape is a compile-time constant here, so a row costs only the loads,
// compares and atomics its query needs -- no type switches, no loops over
// runtime field counts, 32-bit arithmetic where only a low word is kept --
// and the rows after the last whole tile are evaluated in the same launch.
//
// The host prepends a generated struct JS describing the shape:
//   filter, ftype            filter present; its column type (T_*)
//   join, ktype              J_NONE / J_DIRECT / J_HASH32 / J_HASH64; fk type
//   part                     partition filter on the join (hybrid join)
//   ng, gside[], gtype[], gbits[]   group fields, first field highest
//   ns, skind[], atype[], btype[]   sums: S_SUM / S_MUL_SUB and column types
//   mode[]                   1: low word, 2: low + carry word (fast), 0: exact
//   narrow[]                 mode 2 MUL_SUB operands proved to fit in int32
//   fast                     32-bit shared-memory table (column bounds proved
//                            every sum stays inside int64)
// and every runtime value (column offsets in a stage, filter bounds, join
// table, term offsets, multiplier constants) still comes from the launch's
// QueryDev / StageLayout, so one compiled kernel serves every plan and batch
// of the same shape.
#pragma once
#include "pipeline.cuh"

namespace tpj {
using namespace tpk;

enum : int { J_NONE = 0, J_DIRECT = 1, J_HASH32 = 2, J_HASH64 = 3 };

template <int T> struct ColT;
template <> struct ColT<T_I32> { using type = int32_t; using utype = uint32_t; };
template <> struct ColT<T_I64> { using type = int64_t; using utype = uint64_t; };
template <> struct ColT<T_U8> { using type = uint8_t; using utype = uint8_t; };

template <int T>
__device__ __forceinline__ typename ColT<T>::type lds(const unsigned char* col, uint32_t r) {
    return ((const typename ColT<T>::type*)col)[r];
}

// Low 32 bits of row r of a column (of an int64 column: its low word).
template <int T>
__device__ __forceinline__ uint32_t lds_lo(const unsigned char* col, uint32_t r) {
    if constexpr (T == T_I64) return ((const uint32_t*)col)[2 * r];
    else return (uint32_t)lds<T>(col, r);
}

// Per-CTA constants of the shape, hoisted out of the tile loop.
struct Ctx {
    uint32_t off_f, off_k;
    uint32_t off_g[MAX_GROUP];
    uint32_t off_a[MAX_SUM], off_b[MAX_SUM];
    int64_t flo, fhi;
    int32_t flo32, fhi32;   // the bounds clamped to int32 (1 > 0 when nothing passes)
    unsigned char* tab;   // shared-memory dense table
    uint32_t G;
};

// Group field F (compile-time recursion over the fields).
template <int F>
__device__ __forceinline__ void group_fields(const QueryDev& q, const Ctx& c, const unsigned char* stage,
                                             uint32_t r0, const uint32_t pay[ST_RPL], uint32_t g[ST_RPL],
                                             uint32_t& pm) {
    if constexpr (F < JS::ng) {
        constexpr int bits = JS::gbits[F];
        if constexpr (JS::gside[F] == 0) {
            constexpr int T = JS::gtype[F];
            using U = typename ColT<T>::utype;
            uint32_t bad = 0;
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                const U v = (U)lds<T>(stage + c.off_g[F], r0 + 32 * j);
                if constexpr (bits < 8 * (int)sizeof(U)) bad |= (uint32_t)((v >> bits) != 0) << j;
                else if constexpr (T != T_U8) bad |= (uint32_t)((typename ColT<T>::type)v < 0) << j;
                g[j] = (g[j] << bits) | (uint32_t)v;
            }
            if (bad & pm) {
                atomicOr(q.err, ERR_RANGE);
                pm &= ~bad;
            }
        } else {
            const uint32_t mask = (bits >= 32) ? ~0u : ((1u << bits) - 1u);
            const int pos = q.gdpos[F];
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) g[j] = (g[j] << bits) | ((pay[j] >> pos) & mask);
        }
        group_fields<F + 1>(q, c, stage, r0, pay, g, pm);
    }
}

// Sum S of the rows in pm (compile-time recursion over the sums).
template <int S>
__device__ __forceinline__ void sums(const QueryDev& q, const StageLayout& L, const Ctx& c,
                                     const unsigned char* stage, uint32_t r0, const uint32_t g[ST_RPL],
                                     uint32_t pm) {
    if constexpr (S < JS::ns) {
        constexpr int TA = JS::atype[S];
        constexpr int TB = JS::btype[S];
        constexpr bool MS = JS::skind[S] == S_MUL_SUB;
        const unsigned char* ca = stage + c.off_a[S];
        const unsigned char* cb = stage + c.off_b[S];
        if constexpr (JS::fast && JS::mode[S] == 1) {
            // the per-CTA sums of (term - offset) fit in 32 bits: only the low
            // word of every term matters, and it is exact mod 2^32
            uint32_t* lo = (uint32_t*)c.tab + (uint64_t)L.sum_word[S] * c.G;
            const uint32_t off = (uint32_t)(uint64_t)L.sum_off[S];
            const uint32_t k = (uint32_t)(uint64_t)q.sk[S];
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                uint32_t t = lds_lo<TA>(ca, r0 + 32 * j);
                if constexpr (MS) t *= k - lds_lo<TB>(cb, r0 + 32 * j);
                if (pm >> j & 1u) atomicAdd(lo + g[j], t - off);
            }
        } else if constexpr (JS::fast) {
            uint32_t* lo = (uint32_t*)c.tab + (uint64_t)L.sum_word[S] * c.G;
            uint32_t* hi = lo + c.G;
            const int64_t off = L.sum_off[S];
            const int64_t k = q.sk[S];
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                int64_t v = (int64_t)lds<TA>(ca, r0 + 32 * j);
                if constexpr (MS) {
                    const int64_t d = k - (int64_t)lds<TB>(cb, r0 + 32 * j);
                    if constexpr (JS::narrow[S]) v = (int64_t)(int32_t)v * (int64_t)(int32_t)d;
                    else v *= d;
                }
                const uint64_t t = (uint64_t)(v - off);
                if (pm >> j & 1u) {
                    const uint32_t old = atomicAdd(lo + g[j], (uint32_t)t);
                    const uint32_t h = (uint32_t)(t >> 32) + ((old + (uint32_t)t) < old ? 1u : 0u);
                    if (h) atomicAdd(hi + g[j], h);
                }
            }
        } else {
            uint64_t* lo = (uint64_t*)c.tab + (uint64_t)c.G * (1 + 2 * S);
            uint64_t* hi = (uint64_t*)c.tab + (uint64_t)c.G * (2 + 2 * S);
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                if (!(pm >> j & 1u)) continue;
                const int64_t a = (int64_t)lds<TA>(ca, r0 + 32 * j);
                if constexpr (MS) atomic_add_i128(lo + g[j], hi + g[j], mul_sub(a, q.sk[S], (int64_t)lds<TB>(cb, r0 + 32 * j)));
                else atomic_add_i128(lo + g[j], hi + g[j], i128_from_i64(a));
            }
        }
        sums<S + 1>(q, L, c, stage, r0, g, pm);
    }
}

// One consumer warp's rows of a full stage: filter -> probe -> group key ->
// count and sums.
__device__ __forceinline__ void consume(const QueryDev& q, const StageLayout& L, const Ctx& c,
                                        const unsigned char* stage, uint32_t r0, uint32_t valid) {
    uint32_t pm = valid;
    if constexpr (JS::filter) {
        pm = 0;
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) {
            if constexpr (JS::ftype == T_I64) {
                const int64_t v = lds<T_I64>(stage + c.off_f, r0 + 32 * j);
                pm |= (uint32_t)(v >= c.flo && v <= c.fhi) << j;
            } else {
                const int32_t v = (int32_t)lds<JS::ftype>(stage + c.off_f, r0 + 32 * j);
                pm |= (uint32_t)(v >= c.flo32 && v <= c.fhi32) << j;
            }
        }
        pm &= valid;
        if (!pm) return;
    }
    uint32_t pay[ST_RPL];
#pragma unroll
    for (int j = 0; j < ST_RPL; ++j) pay[j] = 0;
    if constexpr (JS::join == J_DIRECT) {
        const unsigned int* dt = (const unsigned int*)q.jt.slots;
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) {
            const uint64_t idx = (uint64_t)((int64_t)lds<JS::ktype>(stage + c.off_k, r0 + 32 * j) - q.jt.kmin);
            pay[j] = ((pm >> j) & 1u) && idx < q.jt.range ? __ldg(dt + idx) : EMPTY32;
        }
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j)
            if (pay[j] == EMPTY32) pm &= ~(1u << j);
    } else if constexpr (JS::join == J_HASH32 || JS::join == J_HASH64) {
        int64_t key[ST_RPL];
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) key[j] = (int64_t)lds<JS::ktype>(stage + c.off_k, r0 + 32 * j);
        if constexpr (JS::part) {
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j)
                if (!part_resident(q.jt, key[j])) pm &= ~(1u << j);
        }
        if constexpr (JS::join == J_HASH32) probe_rows_k32(q.jt, key, pm, pay, q.err);
        else probe_rows_k64(q.jt, key, pm, pay, q.err);
    }
    if constexpr (JS::join != J_NONE) {
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
    group_fields<0>(q, c, stage, r0, pay, g, pm);
    if (!pm) return;
#pragma unroll
    for (int j = 0; j < ST_RPL; ++j) {
        if (!(pm >> j & 1u)) continue;
        if constexpr (JS::fast) atomicAdd((unsigned int*)c.tab + g[j], 1u);
        else atomicAdd((unsigned long long*)c.tab + g[j], 1ull);
    }
    sums<0>(q, L, c, stage, r0, g, pm);
}

// Stage offsets of the group-field (F) and sum (S) columns, by compile-time
// recursion: the shape arrays are only ever indexed by constants.
template <int F, int S>
__device__ __forceinline__ void stage_offsets(const StageLayout& L, Ctx& c) {
    if constexpr (F < JS::ng) {
        if constexpr (JS::gside[F] == 0) c.off_g[F] = L.off[L.col_of_slot[SL_GROUP + F]];
        stage_offsets<F + 1, S>(L, c);
    } else if constexpr (S < JS::ns) {
        c.off_a[S] = L.off[L.col_of_slot[SL_SA + S]];
        if constexpr (JS::skind[S] == S_MUL_SUB) c.off_b[S] = L.off[L.col_of_slot[SL_SB + S]];
        stage_offsets<F, S + 1>(L, c);
    }
}

// Adds sum S (and the following ones) of group gi of this CTA's table to the
// global dense table.
template <int S>
__device__ __forceinline__ void fold_sums(const StageLayout& L, const unsigned char* smem, uint64_t* gacc,
                                          uint32_t G, uint32_t gi, uint64_t cnt) {
    if constexpr (S < JS::ns) {
        if constexpr (JS::fast) {
            // sum = carry words * 2^32 + low words + count * offset: exact
            // modulo 2^64 and, by the bounds, inside int64
            const uint32_t* w = (const uint32_t*)smem + (uint64_t)L.sum_word[S] * G;
            uint64_t v = w[gi];
            if constexpr (JS::mode[S] == 2) v += (uint64_t)w[G + gi] << 32;
            v += cnt * (uint64_t)L.sum_off[S];
            atomicAdd((unsigned long long*)&gacc[(uint64_t)G * (1 + 2 * S) + gi], (unsigned long long)v);
        } else {
            I128 v{((const uint64_t*)smem)[(uint64_t)G * (1 + 2 * S) + gi],
                   ((const uint64_t*)smem)[(uint64_t)G * (2 + 2 * S) + gi]};
            atomic_add_i128(&gacc[(uint64_t)G * (1 + 2 * S) + gi], &gacc[(uint64_t)G * (2 + 2 * S) + gi], v);
        }
        fold_sums<S + 1>(L, smem, gacc, G, gi, cnt);
    }
}

}  // namespace tpj

extern "C" __global__ void __launch_bounds__(tpk::ST_THREADS, tpk::ST_CTAS)
    tpj_dense(const __grid_constant__ tpk::QueryDev q, const __grid_constant__ tpk::StageLayout L, uint64_t n,
              uint64_t* __restrict__ gacc, uint32_t G) {
    using namespace tpk;
    using namespace tpj;
    extern __shared__ __align__(128) unsigned char smem[];
    for (uint32_t i = threadIdx.x; i < L.table_bytes / 8; i += blockDim.x) ((uint64_t*)smem)[i] = 0;
    Ctx c{};
    c.tab = smem;
    c.G = G;
    c.flo = q.flo;
    c.fhi = q.fhi;
    if (q.flo > q.fhi || q.flo > INT32_MAX || q.fhi < INT32_MIN) {
        c.flo32 = 1;
        c.fhi32 = 0;
    } else {
        c.flo32 = (int32_t)(q.flo < INT32_MIN ? (int64_t)INT32_MIN : q.flo);
        c.fhi32 = (int32_t)(q.fhi > INT32_MAX ? (int64_t)INT32_MAX : q.fhi);
    }
    if constexpr (JS::filter) c.off_f = L.off[L.col_of_slot[SL_FILTER]];
    if constexpr (JS::join != J_NONE) c.off_k = L.off[L.col_of_slot[SL_FK]];
    stage_offsets<0, 0>(L, c);
    constexpr uint32_t all = (1u << ST_RPL) - 1u;
    run_pipeline(q, L, n, smem + L.table_bytes, [&](const unsigned char* stage, uint64_t, uint32_t r0) {
        consume(q, L, c, stage, r0, all);
    });
    __syncthreads();
    // rows after the last whole tile: one CTA copies them into the (now
    // idle) first stage with plain loads and evaluates them with a row mask
    const uint64_t ntiles = n / ST_TILE, whole = ntiles * ST_TILE;
    if (whole < n && blockIdx.x == ntiles % gridDim.x) {
        const uint32_t rows = (uint32_t)(n - whole);
        unsigned char* stage = smem + L.table_bytes + 2 * ST_MAX_STAGES * sizeof(uint64_t);
        for (int k = 0; k < L.n_cols; ++k) {
            const uint32_t es = (uint32_t)L.esize[k];
            const unsigned char* src = (const unsigned char*)L.src[k] + whole * es;
            for (uint32_t i = threadIdx.x; i < rows * es; i += blockDim.x) stage[L.off[k] + i] = src[i];
        }
        __syncthreads();
        if (threadIdx.x >= 32) {
            const uint32_t r0 = (threadIdx.x / 32 - 1) * (uint32_t)ST_SUB + (threadIdx.x & 31u);
            uint32_t valid = 0;
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) valid |= (uint32_t)(r0 + 32 * j < rows) << j;
            if (valid) consume(q, L, c, stage, r0, valid);
        }
        __syncthreads();
    }
    // fold this CTA's table into the global dense table (count[G], lo/hi[s][G])
    for (uint32_t gi = threadIdx.x; gi < G; gi += blockDim.x) {
        uint64_t cnt;
        if constexpr (JS::fast) cnt = ((const unsigned int*)smem)[gi];
        else cnt = ((const uint64_t*)smem)[gi];
        if (cnt == 0) continue;
        atomicAdd((unsigned long long*)&gacc[gi], (unsigned long long)cnt);
        fold_sums<0>(L, smem, gacc, G, gi, cnt);
    }
}
