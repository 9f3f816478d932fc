// Pieces of the staged (bulk-copy) pipeline shared by its kernels: mbarrier
// and bulk-copy PTX wrappers, bounded waits, shared-memory row loads, and
// batched join probes.  sm_90+ PTX, built for sm_103a.
#pragma once
#include "device.cuh"

namespace tpk {

// ------------------------------------------------------------- PTX wrappers

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for completion of the phase with the given parity; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_test(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// global -> shared bulk copy; both addresses 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                          uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

// ------------------------------------------------------------ row passes

// Loads rows r0 + 32 j (j < 8) of a column tile held in shared memory.
__device__ __forceinline__ void load8_smem(const unsigned char* base, int type, uint32_t r0, int64_t v[ST_RPL]) {
    switch (type) {
    case T_I32:
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) v[j] = ((const int*)base)[r0 + 32 * j];
        break;
    case T_I64:
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) v[j] = ((const long long*)base)[r0 + 32 * j];
        break;
    default:
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) v[j] = base[r0 + 32 * j];
        break;
    }
}

// Reads of join tables.  Tables built by an earlier launch are read-only for
// the probing kernel and go through the non-coherent path; a kernel that
// builds its tables itself before probing them (the batched queue defines
// TP_TABLES_BUILT_IN_LAUNCH) reads them with ordinary loads, which its
// dependency waits' fences order after the build.
#ifdef TP_TABLES_BUILT_IN_LAUNCH
#define TP_LDT(p) (*(p))
#else
#define TP_LDT(p) __ldg(p)
#endif

// The four 8-byte words of the aligned 32-byte sector at p, as two 128-bit
// loads.  (One 256-bit load, available from sm_100 on, measured slower in
// the probe loop.)
__device__ __forceinline__ void ld_sector(const uint64_t* p, uint64_t (&w)[4]) {
    const ulonglong2 lo = TP_LDT((const ulonglong2*)p), hi = TP_LDT((const ulonglong2*)p + 1);
    w[0] = lo.x;
    w[1] = lo.y;
    w[2] = hi.x;
    w[3] = hi.y;
}

// Batched join probes, one aligned 32-byte sector ("bucket") per round.
//
// The table is filled by slot-wise linear probing from hash & mask.  A lookup
// reads the whole aligned sector holding its current slot (4 slots of a
// 32-bit-key table, 2 of a 64-bit-key table) and examines every slot from its
// position to the end of the sector: a match is the key (keys are unique),
// an empty slot ends the search.  Slots before the starting position in the
// first sector belong to other probe sequences and are skipped.  A lane's
// rows advance independently, so a round costs one sector load per live row
// and most lookups finish in the first round.
//
// With TP_PROBE_LOADS_FIRST (the run-time compiled kernels, which have the
// registers for it) each round first issues the sector loads of all of the
// lane's live rows and only then examines them, so the rows' L2 round trips
// overlap instead of following one another: 10% off the hashed star query's
// kernel.  The ahead-of-time staged kernels run at their register cap, where
// holding every row's sector spilled to local memory, so they examine each
// row's sector as it arrives.  (A window of two sectors per round halves the
// rounds a 64-row warp needs, but measured slower: doubling the probe's L2
// traffic cost more than the round trips it saved.)  pm loses the rows whose
// key is absent; pay receives the payload of the others.
#ifndef TP_PROBE_LOADS_FIRST
#define TP_PROBE_LOADS_FIRST 0
#endif

__device__ __forceinline__ void probe_rows_k32(const JoinTable& jt, const int64_t key[ST_RPL], uint32_t& pm,
                                               uint32_t pay[ST_RPL], uint32_t* err) {
    const uint32_t mask = (uint32_t)jt.mask;
    uint32_t k[ST_RPL], pos[ST_RPL];
    uint32_t act = 0;
#pragma unroll
    for (int j = 0; j < ST_RPL; ++j) {
        const bool in32 = key[j] >= INT32_MIN && key[j] <= INT32_MAX;
        k[j] = (uint32_t)key[j];
        pos[j] = fmix32(k[j]) & mask;
        pay[j] = 0;
        if (!in32) pm &= ~(1u << j);
        if (in32 && k[j] == EMPTY32) {  // the key equal to the empty pattern lives in the side cell
            if (TP_LDT(jt.side) != 0) pay[j] = TP_LDT(jt.side + 1);
            else pm &= ~(1u << j);
        } else if (pm & (1u << j)) {
            act |= 1u << j;
        }
    }
    for (uint32_t it = 0; act && it <= mask; it += 4) {
        if constexpr (TP_PROBE_LOADS_FIRST) {
            const uint32_t live = act;
            uint64_t w[ST_RPL][4];
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j)
                if (live & (1u << j)) ld_sector(jt.slots + (pos[j] & ~3u), w[j]);
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                if (!(live & (1u << j))) continue;
                const uint32_t first = pos[j] & 3u;
                bool done = false;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (done || (uint32_t)m < first) continue;
                    const uint32_t wk = (uint32_t)w[j][m];
                    if (wk == k[j]) {
                        pay[j] = (uint32_t)(w[j][m] >> 32);
                        done = true;
                    } else if (wk == EMPTY32) {
                        pm &= ~(1u << j);
                        done = true;
                    }
                }
                if (done) act &= ~(1u << j);
                else pos[j] = ((pos[j] & ~3u) + 4) & mask;
            }
        } else {
            const ulonglong2* sectors = (const ulonglong2*)jt.slots;
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                if (!(act & (1u << j))) continue;
                const uint32_t base = pos[j] & ~3u;
                const ulonglong2 lo = TP_LDT(sectors + (base >> 1));
                const ulonglong2 hi = TP_LDT(sectors + (base >> 1) + 1);
                const uint64_t w[4] = {lo.x, lo.y, hi.x, hi.y};
                const uint32_t first = pos[j] & 3u;
                bool done = false;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (done || (uint32_t)m < first) continue;
                    const uint32_t wk = (uint32_t)w[m];
                    if (wk == k[j]) {
                        pay[j] = (uint32_t)(w[m] >> 32);
                        done = true;
                    } else if (wk == EMPTY32) {
                        pm &= ~(1u << j);
                        done = true;
                    }
                }
                if (done) act &= ~(1u << j);
                else pos[j] = (base + 4) & mask;
            }
        }
    }
    if (act) {
        atomicOr(err, ERR_INTERNAL);
        pm &= ~act;
    }
}

__device__ __forceinline__ void probe_rows_k64(const JoinTable& jt, const int64_t key[ST_RPL], uint32_t& pm,
                                               uint32_t pay[ST_RPL], uint32_t* err) {
    const uint32_t mask = (uint32_t)jt.mask;
    uint32_t pos[ST_RPL];
    uint32_t act = 0;
#pragma unroll
    for (int j = 0; j < ST_RPL; ++j) {
        pay[j] = 0;
        pos[j] = (uint32_t)fmix64((uint64_t)key[j]) & mask;
        if (!(pm & (1u << j))) continue;
        if ((uint64_t)key[j] == EMPTY64) {
            if (TP_LDT(jt.side) != 0) pay[j] = TP_LDT(jt.side + 1);
            else pm &= ~(1u << j);
            continue;
        }
        act |= 1u << j;
    }
    for (uint32_t it = 0; act && it <= mask; it += 2) {
        if constexpr (TP_PROBE_LOADS_FIRST) {
            const uint32_t live = act;
            ulonglong2 s0[ST_RPL], s1[ST_RPL];
            const ulonglong2* slots = (const ulonglong2*)jt.slots;
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                if (!(live & (1u << j))) continue;
                const uint32_t base = pos[j] & ~1u;
                s0[j] = TP_LDT(slots + base);
                s1[j] = TP_LDT(slots + base + 1);
            }
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                if (!(live & (1u << j))) continue;
                bool done = false;
                if ((pos[j] & 1u) == 0) {
                    if (s0[j].x == (uint64_t)key[j]) {
                        pay[j] = (uint32_t)s0[j].y;
                        done = true;
                    } else if (s0[j].x == EMPTY64) {
                        pm &= ~(1u << j);
                        done = true;
                    }
                }
                if (!done) {
                    if (s1[j].x == (uint64_t)key[j]) {
                        pay[j] = (uint32_t)s1[j].y;
                        done = true;
                    } else if (s1[j].x == EMPTY64) {
                        pm &= ~(1u << j);
                        done = true;
                    }
                }
                if (done) act &= ~(1u << j);
                else pos[j] = ((pos[j] & ~1u) + 2) & mask;
            }
        } else {
            const ulonglong2* slots = (const ulonglong2*)jt.slots;
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                if (!(act & (1u << j))) continue;
                const uint32_t base = pos[j] & ~1u;
                const ulonglong2 s0 = TP_LDT(slots + base);
                const ulonglong2 s1 = TP_LDT(slots + base + 1);
                bool done = false;
                if ((pos[j] & 1u) == 0) {
                    if (s0.x == (uint64_t)key[j]) {
                        pay[j] = (uint32_t)s0.y;
                        done = true;
                    } else if (s0.x == EMPTY64) {
                        pm &= ~(1u << j);
                        done = true;
                    }
                }
                if (!done) {
                    if (s1.x == (uint64_t)key[j]) {
                        pay[j] = (uint32_t)s1.y;
                        done = true;
                    } else if (s1.x == EMPTY64) {
                        pm &= ~(1u << j);
                        done = true;
                    }
                }
                if (done) act &= ~(1u << j);
                else pos[j] = (base + 2) & mask;
            }
        }
    }
    if (act) {
        atomicOr(err, ERR_INTERNAL);
        pm &= ~act;
    }
}

// Probes for the rows in pm of either table kind; tables of the staged path
// have fewer than 2^32 slots.
__device__ __forceinline__ void probe_rows(const JoinTable& jt, const int64_t key[ST_RPL], uint32_t& pm,
                                           uint32_t pay[ST_RPL], uint32_t* err) {
    lip_mask<ST_RPL>(jt, key, pm);
    if (jt.part_shift != 0) {
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j)
            if (!part_resident(jt, key[j])) pm &= ~(1u << j);
    }
    if (jt.direct) {  // one payload word per key
        uint32_t w[ST_RPL];
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) {
            const uint64_t idx = (uint64_t)key[j] - (uint64_t)jt.kmin;
            w[j] = ((pm >> j) & 1u) && idx < jt.range ? TP_LDT((const unsigned int*)jt.slots + idx) : EMPTY32;
        }
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) {
            if (w[j] == EMPTY32) pm &= ~(1u << j);
            pay[j] = w[j];
        }
        return;
    }
    if (!jt.key64) probe_rows_k32(jt, key, pm, pay, err);
    else probe_rows_k64(jt, key, pm, pay, err);
}

// Column source for one tile: its copy in the stage, or global memory (a
// column the layout does not stage is read only for rows still alive).
struct ColSrc {
    const unsigned char* p;
    int type;
    bool smem;
};

__device__ __forceinline__ int esize_dev(int type) { return type == T_I64 ? 8 : (type == T_I32 ? 4 : 1); }

__device__ __forceinline__ ColSrc col_src(const StageLayout& L, int slot, const DevCol& c,
                                          const unsigned char* stage, uint64_t row0) {
    const int k = L.col_of_slot[slot];
    if (k >= 0) return ColSrc{stage + L.off[k], c.type, true};
    return ColSrc{(const unsigned char*)c.ptr + row0 * esize_dev(c.type), c.type, false};
}

// Rows r0 + 32 j of a tile; from global memory only the rows set in pm.
__device__ __forceinline__ void load_rows(const ColSrc& c, uint32_t r0, uint32_t pm, int64_t v[ST_RPL]) {
    if (c.smem) {
        load8_smem(c.p, c.type, r0, v);
        return;
    }
    switch (c.type) {
    case T_I32:
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) v[j] = (pm >> j & 1u) ? (int64_t)__ldcs((const int*)c.p + r0 + 32 * j) : 0;
        break;
    case T_I64:
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j)
            v[j] = (pm >> j & 1u) ? (int64_t)__ldcs((const long long*)c.p + r0 + 32 * j) : 0;
        break;
    default:
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j)
            v[j] = (pm >> j & 1u) ? (int64_t)__ldcs((const unsigned char*)c.p + r0 + 32 * j) : 0;
        break;
    }
}

// The bulk-copy pipeline over the whole tiles of [0, n) that a CTA owns
// (tiles blockIdx.x, blockIdx.x + gridDim.x, ...).  Its ring lives in
// dynamic shared memory: 2 * ST_MAX_STAGES mbarriers ("full" then "empty"
// per stage) followed by L.n_stages stages.
struct Ring {
    uint64_t* full;
    uint64_t* empty;
    unsigned char* stages;
};

// Initialises the ring's barriers; every thread of the CTA calls it.
__device__ __forceinline__ Ring pipeline_setup(const StageLayout& L, unsigned char* area) {
    Ring r{(uint64_t*)area, (uint64_t*)area + ST_MAX_STAGES, area + 2 * ST_MAX_STAGES * sizeof(uint64_t)};
    if (threadIdx.x == 0) {
        for (int s = 0; s < L.n_stages; ++s) {
            mbar_init(&r.full[s], 1);
            mbar_init(&r.empty[s], ST_CONSUMERS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    return r;
}

// The producer (one lane): for every tile of this CTA, waits until the
// consumers released its stage, then issues the tile's bulk copies.
__device__ __forceinline__ void pipeline_produce(const QueryDev& q, const StageLayout& L, uint64_t ntiles,
                                                 const Ring& R) {
    const uint64_t pol = l2_evict_first();
    uint32_t filled = 0, fill_parity = 0;   // per stage: ever filled; parity of its last fill
    bool ok = true;
    int s = 0;        // stage of this tile
    uint32_t u = 0;   // how many times the ring has wrapped: stage s's use count
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (u > 0 && !mbar_wait(&R.empty[s], (u - 1) & 1u, L.wait_ns)) {
            atomicOr(q.err, ERR_TIMEOUT);
            ok = false;
            break;
        }
        mbar_arrive_expect_tx(&R.full[s], L.tile_bytes);
        unsigned char* dst = R.stages + (uint64_t)s * L.stage_bytes;
        for (int c = 0; c < L.n_cols; ++c) {
            const uint32_t bytes = (uint32_t)ST_TILE * (uint32_t)L.esize[c];
            bulk_load(dst + L.off[c], (const unsigned char*)L.src[c] + t * bytes, bytes, &R.full[s], pol);
        }
        filled |= 1u << s;
        fill_parity = (fill_parity & ~(1u << s)) | ((u & 1u) << s);
        if (++s == L.n_stages) {
            s = 0;
            ++u;
        }
    }
    if (!ok) {  // consumers gave up: let the copies already issued land before exit
        for (int s = 0; s < L.n_stages; ++s)
            if (filled >> s & 1u) mbar_wait(&R.full[s], fill_parity >> s & 1u, L.wait_ns);
    }
}

// Runs the pipeline over the first floor(n / ST_TILE) tiles: warp 0 lane 0
// produces, warps 1..ST_CONSUMERS call consume(stage, tile's first row, r0)
// for each tile, r0 being the lane's first tile-local row.  Returns after
// this thread's part of the pipeline is done; the caller synchronises the
// CTA before reading what consumers produced.
template <class Consume>
__device__ __forceinline__ void run_pipeline(const QueryDev& q, const StageLayout& L, uint64_t n,
                                             unsigned char* area, Consume&& consume) {
    const Ring R = pipeline_setup(L, area);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t ntiles = n / ST_TILE;
    if (warp == 0) {
        if (lane == 0) pipeline_produce(q, L, ntiles, R);
        return;
    }
    const uint32_t r0 = (uint32_t)(warp - 1) * ST_SUB + (uint32_t)lane;
    int s = 0;
    uint32_t phase = 0;   // parity of stage s's current use
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (!mbar_wait(&R.full[s], phase, L.wait_ns)) {
            atomicOr(q.err, ERR_TIMEOUT);
            return;
        }
        consume(R.stages + (uint64_t)s * L.stage_bytes, t * ST_TILE, r0);
        __syncwarp();
        if (lane == 0) mbar_arrive(&R.empty[s]);
        if (++s == L.n_stages) {
            s = 0;
            phase ^= 1u;
        }
    }
}

}  // namespace tpk
