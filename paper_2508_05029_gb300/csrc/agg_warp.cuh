// Warp-aggregated updates of a global aggregation table.
//
// The lanes of a warp that hold rows with the same group key find each other
// with __match_any_sync; the lowest lane of each such set adds the others'
// count and terms over shuffles and updates the table once.  A key repeated
// among a warp's rows then costs one slot lookup and one set of atomics
// instead of one per row.  Paper basis: Section 3.1 (group-by over batches of
// columns) and Section 4 (decimal sums held as 128-bit integers); the warp
// aggregation is this library's design.
#pragma once
#include "device.cuh"

namespace tpk {

// Adds the count and terms of every other lane in `rest` (the caller's set of
// lanes with its key) to this lane's values.  Every lane of the warp runs the
// same shuffles, as many rounds as the largest set has other members.
template <int NS, bool FAST>
__device__ __forceinline__ void warp_reduce_set(int n_sum, uint32_t rest, int64_t (&t)[NS > 0 ? NS : 1],
                                                I128 (&tm)[NS > 0 ? NS : 1]) {
    const int lane = threadIdx.x & 31;
    while (__any_sync(0xffffffffu, rest != 0)) {
        const int src = rest ? __ffs(rest) - 1 : lane;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (s >= n_sum) break;
            if constexpr (FAST) {
                const int64_t y = __shfl_sync(0xffffffffu, t[s], src);
                if (rest) t[s] += y;
            } else {
                const uint64_t ylo = __shfl_sync(0xffffffffu, tm[s].lo, src);
                const uint64_t yhi = __shfl_sync(0xffffffffu, tm[s].hi, src);
                if (rest) tm[s] = i128_add(tm[s], I128{ylo, yhi});
            }
        }
        rest &= rest - 1u;
    }
}

// One row per lane (valid or not) with its key and terms: the lanes sharing a
// key combine, and the lowest of them updates the table.  All 32 lanes call
// it.  claims counts the fresh hashed slots this lane took.
template <int NS, bool FAST>
__device__ __forceinline__ void agg_warp_row(const AggTable& tab, uint32_t* err, int n_sum, bool valid,
                                             uint64_t key, int64_t (&t)[NS > 0 ? NS : 1],
                                             I128 (&tm)[NS > 0 ? NS : 1], uint32_t& claims) {
    const uint32_t vm = __ballot_sync(0xffffffffu, valid);
    if (vm == 0) return;
    const int lane = threadIdx.x & 31;
    const uint32_t peers = __match_any_sync(0xffffffffu, (unsigned long long)key) & vm;
    const bool head = valid && __ffs(peers) - 1 == lane;
    warp_reduce_set<NS, FAST>(n_sum, head ? peers & (peers - 1u) : 0u, t, tm);
    if (!head) return;
    bool claimed;
    uint64_t* p = agg_slot_any(tab, key, err, claimed);
    claims += claimed ? 1u : 0u;
    if (!p) return;
    atomicAdd((unsigned long long*)(p + 1), (unsigned long long)__popc(peers));
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if (s >= n_sum) break;
        if constexpr (FAST) atomicAdd((unsigned long long*)(p + 2 + 2 * s), (unsigned long long)t[s]);
        else atomic_add_i128(p + 2 + 2 * s, p + 3 + 2 * s, tm[s]);
    }
}

}  // namespace tpk
