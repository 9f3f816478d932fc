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

// Slots of R keys at once (only where want[j]): the probe loads of all R
// keys are in flight together, then the claims of empty slots, so a lane's
// rows cost about two round trips to L2 instead of two per row.  claimed[j]
// is set for fresh hashed slots; slot[j] is nullptr for keys of another
// pass's range (or, with ERR_OVERFLOW / ERR_INTERNAL, a full table).
template <int R>
__device__ __forceinline__ void agg_slots(const AggTable& t, const uint64_t (&key)[R], const bool (&want)[R],
                                          uint32_t* err, uint64_t* (&slot)[R], bool (&claimed)[R]) {
    bool act[R];
    uint64_t s[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        slot[j] = nullptr;
        claimed[j] = false;
        act[j] = want[j] && !(t.split && (key[j] < t.key_lo || key[j] > t.key_hi));
        if (!act[j]) continue;
        if (t.direct) {
            const uint64_t d = key[j] - t.kmin;
            if (d > t.mask) atomicOr(err, ERR_INTERNAL);
            else slot[j] = t.slots + d * t.words;
            act[j] = false;
        } else if (key[j] == EMPTY64) {
            slot[j] = t.slots + (t.mask + 1) * t.words;   // side slot
            act[j] = false;
        } else {
            s[j] = fmix64(key[j]) & t.mask;
        }
    }
    for (uint64_t it = 0; it <= t.mask; ++it) {
        uint64_t k[R];
#pragma unroll
        for (int j = 0; j < R; ++j)
            if (act[j]) k[j] = __ldcg((const unsigned long long*)(t.slots + s[j] * t.words));
        unsigned long long prev[R];
        bool cas[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            cas[j] = act[j] && k[j] == EMPTY64;
            if (cas[j])
                prev[j] = atomicCAS((unsigned long long*)(t.slots + s[j] * t.words), (unsigned long long)EMPTY64,
                                    (unsigned long long)key[j]);
        }
        bool any = false;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (!act[j]) continue;
            const bool mine = cas[j] ? (prev[j] == EMPTY64 || prev[j] == key[j]) : k[j] == key[j];
            if (mine) {
                slot[j] = t.slots + s[j] * t.words;
                claimed[j] = cas[j] && prev[j] == EMPTY64;
                act[j] = false;
            } else {
                s[j] = (s[j] + 1) & t.mask;
                any = true;
            }
        }
        if (!any) return;
    }
#pragma unroll
    for (int j = 0; j < R; ++j)
        if (act[j]) atomicOr(err, ERR_OVERFLOW);
}

// R rows per lane (valid or not) with their keys and terms: for each row
// index j the lanes sharing a key combine (the lowest one keeps the set's
// count and terms), then the table slots of all the lane's set leaders are
// found together and updated.  All 32 lanes call it.  claims counts the
// fresh hashed slots this lane took.
template <int NS, bool FAST, int R>
__device__ __forceinline__ void agg_warp_rows(const AggTable& tab, uint32_t* err, int n_sum, const bool (&valid)[R],
                                              const uint64_t (&key)[R], int64_t (&t)[NS > 0 ? NS : 1][R],
                                              I128 (&tm)[NS > 0 ? NS : 1][R], uint32_t& claims) {
    constexpr int NSX = NS > 0 ? NS : 1;
    const int lane = threadIdx.x & 31;
    bool head[R];
    uint32_t cnt[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const uint32_t vm = __ballot_sync(0xffffffffu, valid[j]);
        head[j] = false;
        cnt[j] = 0;
        if (vm == 0) continue;   // warp-uniform
        const uint32_t peers = __match_any_sync(0xffffffffu, (unsigned long long)key[j]) & vm;
        head[j] = valid[j] && __ffs(peers) - 1 == lane;
        cnt[j] = __popc(peers);
        int64_t tj[NSX];
        I128 tmj[NSX];
#pragma unroll
        for (int s = 0; s < NSX; ++s) {
            tj[s] = t[s][j];
            tmj[s] = tm[s][j];
        }
        warp_reduce_set<NS, FAST>(n_sum, head[j] ? peers & (peers - 1u) : 0u, tj, tmj);
#pragma unroll
        for (int s = 0; s < NSX; ++s) {
            t[s][j] = tj[s];
            tm[s][j] = tmj[s];
        }
    }
    uint64_t* slot[R];
    bool claimed[R];
    agg_slots<R>(tab, key, head, err, slot, claimed);
#pragma unroll
    for (int j = 0; j < R; ++j) {
        claims += claimed[j] ? 1u : 0u;
        uint64_t* p = slot[j];
        if (!p) continue;
        atomicAdd((unsigned long long*)(p + 1), (unsigned long long)cnt[j]);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (s >= n_sum) break;
            if constexpr (FAST) atomicAdd((unsigned long long*)(p + 2 + 2 * s), (unsigned long long)t[s][j]);
            else atomic_add_i128(p + 2 + 2 * s, p + 3 + 2 * s, tm[s][j]);
        }
    }
}

}  // namespace tpk
