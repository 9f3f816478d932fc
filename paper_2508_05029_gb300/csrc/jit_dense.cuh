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
// The host prepends a generated struct JS describing the shape (fields as in
// jit_common.cuh); every runtime value (column offsets in a stage, filter
// bounds, join table, term offsets, multiplier constants) still comes from
// the launch's QueryDev / StageLayout, so one compiled kernel serves every
// plan and batch of the same shape.
#pragma once
#include "jit_common.cuh"

namespace tpj {

// Byte offsets of the shape's columns inside a stage, by column id.
struct StageOffs {
    uint32_t off[CI_N];
};

template <class S, int F, int I>
__device__ __forceinline__ void stage_offsets(const StageLayout& L, StageOffs& o) {
    if constexpr (F < S::ng) {
        if constexpr (S::gside[F] == 0) o.off[CI_G + F] = L.off[L.col_of_slot[SL_GROUP + F]];
        stage_offsets<S, F + 1, I>(L, o);
    } else if constexpr (I < S::ns) {
        o.off[CI_A + I] = L.off[L.col_of_slot[SL_SA + I]];
        if constexpr (S::skind[I] == S_MUL_SUB) o.off[CI_B + I] = L.off[L.col_of_slot[SL_SB + I]];
        stage_offsets<S, F, I + 1>(L, o);
    }
}

// Column source of one stage: its base plus the shape's offsets.
struct StageCols {
    const unsigned char* s;
    const StageOffs* o;
    template <int T, int CI>
    __device__ __forceinline__ typename ColT<T>::type ld(uint32_t r0, int j) const {
        return lds<T>(s + o->off[CI], r0 + 32 * j);
    }
    template <int T, int CI>
    __device__ __forceinline__ uint32_t ld_lo(uint32_t r0, int j) const {
        return lds_lo<T>(s + o->off[CI], r0 + 32 * j);
    }
};

// Adds sum I (and the following ones) of group gi of this CTA's table to the
// global dense table.
template <class S, int I>
__device__ __forceinline__ void fold_sums(const StageLayout& L, const unsigned char* smem, uint64_t* gacc,
                                          uint32_t G, uint32_t gi, uint64_t cnt) {
    if constexpr (I < S::ns) {
        if constexpr (S::fast) {
            // sum = carry words * 2^32 + low words + count * offset: exact
            // modulo 2^64 and, by the bounds, inside int64
            const uint32_t* w = (const uint32_t*)smem + (uint64_t)L.sum_word[I] * G;
            uint64_t v = w[gi];
            if constexpr (S::mode[I] == 2) v += (uint64_t)w[G + gi] << 32;
            v += cnt * (uint64_t)L.sum_off[I];
            atomicAdd((unsigned long long*)&gacc[(uint64_t)G * (1 + 2 * I) + gi], (unsigned long long)v);
        } else {
            I128 v{((const uint64_t*)smem)[(uint64_t)G * (1 + 2 * I) + gi],
                   ((const uint64_t*)smem)[(uint64_t)G * (2 + 2 * I) + gi]};
            atomic_add_i128(&gacc[(uint64_t)G * (1 + 2 * I) + gi], &gacc[(uint64_t)G * (2 + 2 * I) + gi], v);
        }
        fold_sums<S, I + 1>(L, smem, gacc, G, gi, cnt);
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
    Tab t{};
    t.base = smem;
    t.G = G;
    t.sum_off = L.sum_off;
    const Flt flt = make_flt(q);
    StageOffs o{};
    if constexpr (JS::filter) o.off[CI_F] = L.off[L.col_of_slot[SL_FILTER]];
    if constexpr (JS::join != J_NONE) o.off[CI_K] = L.off[L.col_of_slot[SL_FK]];
#pragma unroll
    for (int j = 0; j < JS::nx; ++j) o.off[CI_X + j] = L.off[L.col_of_slot[SL_FKX + j]];
    stage_offsets<JS, 0, 0>(L, o);
    constexpr uint32_t all = (1u << ST_RPL) - 1u;
    run_pipeline(q, L, n, smem + L.table_bytes, [&](const unsigned char* stage, uint64_t, uint32_t r0) {
        consume<JS>(q, flt, t, StageCols{stage, &o}, r0, all);
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
            if (valid) consume<JS>(q, flt, t, StageCols{stage, &o}, r0, valid);
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
        fold_sums<JS, 0>(L, smem, gacc, G, gi, cnt);
    }
}
