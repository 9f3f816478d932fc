// Device helpers shared by the operator kernels: hashing, column loads,
// exact 128-bit sums, join probing, the per-lane row evaluation of the fused
// filter -> probe -> key pipeline, and the global aggregation slot lookup.
#pragma once
#include "kernels.cuh"

namespace tpk {

// 32-bit finaliser of MurmurHash3 (Appleby, public domain): hash of 32-bit
// join keys, whose tables have fewer than 2^32 slots.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// Hash of a join key: fmix32 for 32-bit key tables, fmix64 for 64-bit ones.
__device__ __forceinline__ uint64_t join_hash(const JoinTable& jt, int64_t key) {
    return jt.key64 ? fmix64((uint64_t)key) : (uint64_t)fmix32((uint32_t)key);
}

// ------------------------------------------------------------------ loads

__device__ __forceinline__ int64_t ld1(const DevCol& c, uint64_t i) {
    switch (c.type) {
    case T_I32: return __ldcs((const int*)c.ptr + i);
    case T_I64: return __ldcs((const long long*)c.ptr + i);
    default: return (int64_t)__ldcs((const unsigned char*)c.ptr + i);
    }
}

// rows r, r+1, r+64, r+65 of a full tile (r even)
__device__ __forceinline__ void ld4(const DevCol& c, uint64_t r, int64_t v[4]) {
    switch (c.type) {
    case T_I32: {
        const int2* p = reinterpret_cast<const int2*>((const int32_t*)c.ptr + r);
        int2 a = __ldcs(p), b = __ldcs(p + 32);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
        break;
    }
    case T_I64: {
        const longlong2* p = reinterpret_cast<const longlong2*>((const int64_t*)c.ptr + r);
        longlong2 a = __ldcs(p), b = __ldcs(p + 32);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
        break;
    }
    default: {
        const uchar2* p = reinterpret_cast<const uchar2*>((const uint8_t*)c.ptr + r);
        uchar2 a = __ldcs(p), b = __ldcs(p + 32);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
        break;
    }
    }
}

template <bool FULL>
__device__ __forceinline__ void load_rows(const DevCol& c, uint64_t r, uint64_t n, const bool want[4],
                                          int64_t v[4]) {
    if (FULL) {
        ld4(c, r, v);
    } else {
        const uint64_t rows[4] = {r, r + 1, r + 64, r + 65};
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = (want[i] && rows[i] < n) ? ld1(c, rows[i]) : 0;
    }
}

// ------------------------------------------------------------- 128-bit sums

struct I128 {
    uint64_t lo;
    uint64_t hi;
};

__device__ __forceinline__ I128 i128_from_i64(int64_t v) {
    return I128{(uint64_t)v, (uint64_t)(v >> 63)};
}

__device__ __forceinline__ I128 i128_add(I128 a, I128 b) {
    I128 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
    return r;
}

// a * (k - b) for 64-bit a, b, k: exact, since |a| < 2^63 and |k - b| < 2^64
// keep the product below 2^127 in magnitude.
__device__ __forceinline__ I128 mul_sub(int64_t a, int64_t k, int64_t b) {
    __int128 d = (__int128)k - (__int128)b;
    __int128 p = (__int128)a * d;
    return I128{(uint64_t)p, (uint64_t)((unsigned __int128)p >> 64)};
}

// Adds t to the 128-bit value (lo, hi) with two 64-bit atomics: the carry out
// of each low-word addition follows from the value the atomic returned, so the
// high word receives exactly the sum of all carries plus all high words.
__device__ __forceinline__ void atomic_add_i128(uint64_t* lo, uint64_t* hi, I128 t) {
    unsigned long long old = atomicAdd((unsigned long long*)lo, (unsigned long long)t.lo);
    uint64_t h = t.hi + ((old + t.lo) < old ? 1ull : 0ull);
    if (h != 0) atomicAdd((unsigned long long*)hi, (unsigned long long)h);
}

// ------------------------------------------------------ lookahead filter
//
// Lookahead information passing (Section 5): the keys of the dimension rows
// that pass the dimension predicate go into a blocked Bloom filter, and fact
// rows test their key before the probe (and before a partitioned join spills
// them).  With h = fmix64(key), the top bits of h pick one 256-bit block (an
// aligned 32-byte sector) and word w of the block holds bit
// (lo32(h) * M_w) >> 27 with the odd multiplier M_w = 0x9E3779B1 * (2w + 1).
// A test reads one sector; an inserted key always passes.

__device__ __forceinline__ uint32_t lip_bit(uint32_t h, uint32_t w) {
    return 1u << ((h * (0x9E3779B1u * (2u * w + 1u))) >> 27);
}

__device__ __forceinline__ bool lip_test(const JoinTable& jt, int64_t key) {
    const uint64_t h = fmix64((uint64_t)key);
    const uint4* blk = reinterpret_cast<const uint4*>(jt.lip + ((h >> jt.lip_shift) << 3));
    const uint4 a = __ldg(blk), b = __ldg(blk + 1);
    const uint32_t l = (uint32_t)h;
    const uint32_t miss = (~a.x & lip_bit(l, 0)) | (~a.y & lip_bit(l, 1)) | (~a.z & lip_bit(l, 2)) |
                          (~a.w & lip_bit(l, 3)) | (~b.x & lip_bit(l, 4)) | (~b.y & lip_bit(l, 5)) |
                          (~b.z & lip_bit(l, 6)) | (~b.w & lip_bit(l, 7));
    return miss == 0;
}

__device__ __forceinline__ void lip_insert(const JoinTable& jt, int64_t key) {
    const uint64_t h = fmix64((uint64_t)key);
    uint32_t* blk = jt.lip + ((h >> jt.lip_shift) << 3);
#pragma unroll
    for (uint32_t w = 0; w < 8; ++w) atomicOr(blk + w, lip_bit((uint32_t)h, w));
}

// Clears bit j of pm for rows whose key the lookahead filter rules out.
template <int N>
__device__ __forceinline__ void lip_mask(const JoinTable& jt, const int64_t* key, uint32_t& pm) {
    if (jt.lip == nullptr) return;
#pragma unroll
    for (int j = 0; j < N; ++j)
        if (((pm >> j) & 1u) && !lip_test(jt, key[j])) pm &= ~(1u << j);
}

// Does dimension row i pass the dimension predicate?
__device__ __forceinline__ bool dim_row_admitted(const BuildDev& b, uint64_t i) {
    if (!b.has_filter) return true;
    const int64_t v = ld1(b.fcol, i);
    return v >= b.flo && v <= b.fhi;
}

// ------------------------------------------------------------------ probing

// Partitioned joins: does this key's partition have its rows in the table?
__device__ __forceinline__ bool part_resident(const JoinTable& jt, int64_t key) {
    return jt.part_shift == 0 || ((jt.part_mask >> (fmix64((uint64_t)key) >> jt.part_shift)) & 1ull) != 0;
}

// Table word load: through the read-only path (NC), or coherent at L2 for
// tables written earlier in the same kernel launch.
template <bool NC, typename T>
__device__ __forceinline__ T ld_table(const T* p) {
    if constexpr (NC) return __ldg(p);
    else return __ldcg(p);
}

// Looks up four keys at once so their table loads overlap.  pass[i] is
// cleared for rows whose key is absent.
template <bool NC = true>
__device__ __forceinline__ void probe4(const JoinTable& jt, const int64_t key[4], bool pass[4],
                                       uint32_t payload[4], uint32_t* err) {
    if (jt.lip != nullptr) {
#pragma unroll
        for (int i = 0; i < 4; ++i) pass[i] = pass[i] && lip_test(jt, key[i]);
    }
    if (jt.part_shift != 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) pass[i] = pass[i] && part_resident(jt, key[i]);
    }
    if (jt.direct) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint64_t idx = (uint64_t)key[i] - (uint64_t)jt.kmin;
            const bool in = pass[i] && idx < jt.range;
            w[i] = in ? ld_table<NC>((const unsigned int*)jt.slots + idx) : EMPTY32;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            pass[i] = pass[i] && w[i] != EMPTY32;
            payload[i] = w[i];
        }
        return;
    }
    uint64_t slot[4];
    bool act[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        act[i] = pass[i];
        payload[i] = 0;
        if (!act[i]) continue;
        bool special;
        if (jt.key64) {
            special = (uint64_t)key[i] == EMPTY64;
        } else {
            if (key[i] < INT32_MIN || key[i] > INT32_MAX) {  // cannot match a 32-bit key
                pass[i] = false;
                act[i] = false;
                continue;
            }
            special = (uint32_t)key[i] == EMPTY32;
        }
        if (special) {
            pass[i] = ld_table<NC>(jt.side) != 0;
            payload[i] = ld_table<NC>(jt.side + 1);
            act[i] = false;
            continue;
        }
        slot[i] = join_hash(jt, key[i]) & jt.mask;
    }
    for (uint64_t it = 0; it <= jt.mask; ++it) {
        bool any = false;
        if (!jt.key64) {
            uint64_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (act[i]) w[i] = ld_table<NC>((const unsigned long long*)jt.slots + slot[i]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (!act[i]) continue;
                uint32_t wk = (uint32_t)w[i];
                if (wk == (uint32_t)key[i]) {
                    payload[i] = (uint32_t)(w[i] >> 32);
                    act[i] = false;
                } else if (wk == EMPTY32) {
                    pass[i] = false;
                    act[i] = false;
                } else {
                    slot[i] = (slot[i] + 1) & jt.mask;
                    any = true;
                }
            }
        } else {
            ulonglong2 w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (act[i]) w[i] = ld_table<NC>((const ulonglong2*)jt.slots + slot[i]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (!act[i]) continue;
                if (w[i].x == (uint64_t)key[i]) {
                    payload[i] = (uint32_t)w[i].y;
                    act[i] = false;
                } else if (w[i].x == EMPTY64) {
                    pass[i] = false;
                    act[i] = false;
                } else {
                    slot[i] = (slot[i] + 1) & jt.mask;
                    any = true;
                }
            }
        }
        if (!any) return;
    }
    atomicOr(err, ERR_INTERNAL);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (act[i]) pass[i] = false;
}

// ------------------------------------------------------------ tile pipeline
//
// A lane evaluates its four rows in phases so that only the row state (pass
// bits and packed keys) stays live across phases: filter, then join probe,
// then the group key, then each aggregate column in turn, fed straight into
// the accumulators.

__device__ __forceinline__ bool any4(const bool p[4]) { return p[0] || p[1] || p[2] || p[3]; }

// Filter, join and key packing of the lane's four rows in warp tile t0.
// Returns false when no row of the lane survives.
template <bool FULL, bool NC = true>
__device__ __forceinline__ bool eval_keys(const QueryDev& q, uint64_t t0, uint64_t n, int lane,
                                          bool pass[4], uint64_t key[4], uint32_t m = 0) {
    const uint64_t r = t0 + 2ull * (uint64_t)lane;
    const uint64_t rows[4] = {r, r + 1, r + 64, r + 65};
#pragma unroll
    for (int i = 0; i < 4; ++i) pass[i] = FULL || rows[i] < n;
    int64_t v[4];
    if (q.has_filter) {
        load_rows<FULL>(q.fcol, r, n, pass, v);
#pragma unroll
        for (int i = 0; i < 4; ++i) pass[i] = pass[i] && v[i] >= q.flo && v[i] <= q.fhi;
        if (!any4(pass)) return false;
    }
    uint32_t payload[4] = {0, 0, 0, 0};
    if (q.has_join) {
        load_rows<FULL>(q.fk, r, n, pass, v);
        probe4<NC>(q.jt, v, pass, payload, q.err);
        if (q.jt.many) {   // fan-out: the m-th row of the key's run, if the run is that long
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (!pass[i]) continue;
                const uint64_t at = (uint64_t)payload[i] + m;
                pass[i] = at < q.jt.mn && __ldg(q.jt.mkeys + at) == (uint64_t)v[i];
                if (pass[i]) payload[i] = __ldg(q.jt.mpay + at);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (pass[i] && (payload[i] & PAYLOAD_BAD)) {
                atomicOr(q.err, ERR_RANGE);
                pass[i] = false;
            }
        }
        if (!any4(pass)) return false;
    }
    // star join: every further table must hold the row's key too
    uint32_t xpay[MAX_XJOIN][4];
#pragma unroll
    for (int j = 0; j < MAX_XJOIN; ++j) {
#pragma unroll
        for (int i = 0; i < 4; ++i) xpay[j][i] = 0;
        if (j >= q.n_xjoin) continue;
        load_rows<FULL>(q.fkx[j], r, n, pass, v);
        probe4<NC>(q.jtx[j], v, pass, xpay[j], q.err);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (pass[i] && (xpay[j][i] & PAYLOAD_BAD)) {
                atomicOr(q.err, ERR_RANGE);
                pass[i] = false;
            }
        }
        if (!any4(pass)) return false;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) key[i] = 0;
#pragma unroll
    for (int g = 0; g < MAX_GROUP; ++g) {
        if (g >= q.n_group) break;
        const int bits = q.gbits[g];
        const bool fact_side = q.gside[g] == 0;
        if (fact_side) load_rows<FULL>(q.gcol[g], r, n, pass, v);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint32_t pw = payload[i];   // the payload of the field's join
#pragma unroll
            for (int j = 0; j < MAX_XJOIN; ++j)
                if (q.gdim[g] == j + 1) pw = xpay[j][i];
            const uint64_t f = fact_side ? (uint64_t)v[i]
                                         : (uint64_t)(pw >> q.gdpos[g]) & ((1ull << bits) - 1ull);
            if (bits < 64) {
                if (pass[i] && (f >> bits) != 0) {
                    atomicOr(q.err, ERR_RANGE);
                    pass[i] = false;
                }
                key[i] = (key[i] << bits) | f;
            } else {
                key[i] = f;
            }
        }
    }
    return any4(pass);
}

// The four terms of aggregate s for the lane's rows.
template <bool FULL>
__device__ __forceinline__ void eval_terms(const QueryDev& q, int s, uint64_t t0, uint64_t n, int lane,
                                           const bool pass[4], I128 t[4]) {
    const uint64_t r = t0 + 2ull * (uint64_t)lane;
    int64_t a[4];
    load_rows<FULL>(q.sa[s], r, n, pass, a);
    if (q.skind[s] == S_MUL_SUB) {
        int64_t b[4];
        load_rows<FULL>(q.sb[s], r, n, pass, b);
#pragma unroll
        for (int i = 0; i < 4; ++i) t[i] = mul_sub(a[i], q.sk[s], b[i]);
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) t[i] = i128_from_i64(a[i]);
    }
}


// ---------------------------------------------------------------- finalise

// Correctly rounded conversion of a 128-bit integer to double.  Values that
// fit in 64 bits use the hardware conversion directly.  Wider magnitudes keep
// their top 64 bits and fold every discarded bit into the lowest kept bit
// (a "sticky" bit): with 64 kept bits and 53 significand bits the rounding
// decision (round bit plus "anything below it") is unchanged, so one
// round-to-nearest conversion of the 64-bit value, scaled by an exact power
// of two, is the correctly rounded result.
__device__ __forceinline__ double i128_to_double(uint64_t lo, uint64_t hi) {
    if (hi == (uint64_t)((int64_t)lo >> 63)) return __ll2double_rn((long long)lo);
    const bool neg = (int64_t)hi < 0;
    uint64_t mlo = lo, mhi = hi;
    if (neg) {  // two's complement negate; -2^127 maps to 2^127 as unsigned
        mlo = ~lo + 1ull;
        mhi = ~hi + (mlo == 0 ? 1ull : 0ull);
    }
    double d;
    if (mhi == 0) {
        d = __ull2double_rn(mlo);
    } else {
        const int lz = __clzll((long long)mhi);
        const int s = 64 - lz;  // 1..64
        uint64_t top, sticky;
        if (s == 64) {
            top = mhi;
            sticky = mlo != 0;
        } else {
            top = (mhi << (64 - s)) | (mlo >> s);
            sticky = (mlo & ((1ull << s) - 1ull)) != 0;
        }
        d = ldexp(__ull2double_rn(top | sticky), s);
    }
    return neg ? -d : d;
}

__device__ __forceinline__ void write_row(const OutDev& o, uint64_t pos, uint64_t key, uint64_t c,
                                          const uint64_t* lo_hi, int n_sum) {
    o.keys[pos] = key;
    o.counts[pos] = (int64_t)c;
    for (int s = 0; s < n_sum; ++s) {
        o.sums[s][2 * pos] = lo_hi[2 * s];
        o.sums[s][2 * pos + 1] = lo_hi[2 * s + 1];
        if (o.has_avg[s])
            o.avgs[s][pos] = __ddiv_rn(i128_to_double(lo_hi[2 * s], lo_hi[2 * s + 1]),
                                       __ll2double_rn((long long)c));
    }
}

// Non-empty groups among [g0, g1) of a dense table (count[G] first); every
// thread of the CTA calls it and gets the total.
__device__ __forceinline__ uint32_t dense_range_count(const uint64_t* __restrict__ gacc, uint32_t g0, uint32_t g1) {
    __shared__ uint32_t warp_cnt[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t c = 0;
    for (uint32_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) c += gacc[g] != 0 ? 1u : 0u;
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if (lane == 0) warp_cnt[warp] = c;
    __syncthreads();
    uint32_t total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) total += warp_cnt[w];
    __syncthreads();
    return total;
}

// One CTA writes the non-empty groups among [g0, g1) of a dense table
// (count[G], then lo/hi per sum) in key order at output rows first,
// first + 1, ...; returns how many it wrote.  lo_only: high words are the
// sign extension of the low words.  Every thread of the CTA must call it.
__device__ __forceinline__ uint64_t dense_range_emit(const uint64_t* __restrict__ gacc, uint32_t G, uint32_t g0,
                                                     uint32_t g1, int n_sum, const OutDev& o, bool lo_only,
                                                     uint64_t first) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint64_t base;
    if (threadIdx.x == 0) base = first;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t c0 = g0; c0 < g1; c0 += blockDim.x) {
        const uint32_t g = c0 + threadIdx.x;
        const bool has = g < g1 && gacc[g] != 0;
        const unsigned m = __ballot_sync(0xffffffffu, has);
        if (lane == 0) warp_tot[warp] = __popc(m);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < warp) before += warp_tot[w];
            total += warp_tot[w];
        }
        if (has) {
            const uint64_t pos = base + before + __popc(m & ((1u << lane) - 1u));
            uint64_t lh[2 * MAX_SUM];
            for (int s = 0; s < n_sum; ++s) {
                lh[2 * s] = gacc[(uint64_t)G * (1 + 2 * s) + g];
                lh[2 * s + 1] = lo_only ? (uint64_t)((int64_t)lh[2 * s] >> 63) : gacc[(uint64_t)G * (2 + 2 * s) + g];
            }
            write_row(o, pos, g, gacc[g], lh, n_sum);
        }
        __syncthreads();
        if (threadIdx.x == 0) base += total;
        __syncthreads();
    }
    const uint64_t n = base - first;
    __syncthreads();
    return n;
}

// One CTA writes every non-empty group of a dense table in key order, so the
// output is sorted, and the group count.
__device__ __forceinline__ void final_dense_block(const uint64_t* __restrict__ gacc, uint32_t G, int n_sum,
                                                  const OutDev& o, bool lo_only) {
    const uint64_t n = dense_range_emit(gacc, G, 0, G, n_sum, o, lo_only, 0);
    if (threadIdx.x == 0) *o.n_groups = n;
}

// ------------------------------------------------------------- join build

// Inserts dimension row i into the join table: CAS on the key (32-bit keys:
// key and payload in one word), ERR_DUP on a repeated key.
__device__ __forceinline__ void build_insert(const BuildDev& b, uint64_t i) {
    const JoinTable& jt = b.jt;
    if (!dim_row_admitted(b, i)) return;
    int64_t key = ld1(b.key, i);
    if (jt.lip != nullptr) lip_insert(jt, key);
    // Dimension group fields packed into bits 0..30 of the payload; bit 31
    // marks a row with a field outside its width.  That is an error only
    // if a surviving fact row joins to it, which the probe side reports.
    uint32_t payload = 0;
    for (int f = 0; f < b.n_dfield; ++f) {
        int64_t v = ld1(b.dcol[f], i);
        if (v < 0 || ((uint64_t)v >> b.dbits[f]) != 0) payload |= PAYLOAD_BAD;
        else payload |= (uint32_t)((uint64_t)v << b.dpos[f]);
    }
    if (jt.direct) {  // slot key - kmin: the host sized the table to the key range
        const uint32_t v = (payload & PAYLOAD_BAD) ? PAYLOAD_BAD : payload;
        const uint64_t idx = (uint64_t)key - (uint64_t)jt.kmin;
        if (idx >= jt.range) { atomicOr(b.err, ERR_INTERNAL); return; }
        if (atomicCAS((unsigned int*)jt.slots + idx, EMPTY32, v) != EMPTY32) atomicOr(b.err, ERR_DUP);
        return;
    }
    bool special = jt.key64 ? (uint64_t)key == EMPTY64 : (uint32_t)key == EMPTY32;
    if (special) {
        if (atomicCAS(jt.side, 0u, 1u) != 0u) atomicOr(b.err, ERR_DUP);
        else jt.side[1] = payload;
        return;
    }
    uint64_t s = join_hash(jt, key) & jt.mask;
    bool placed = false;
    for (uint64_t it = 0; it <= jt.mask; ++it) {
        if (!jt.key64) {
            unsigned long long want = ((unsigned long long)payload << 32) | (uint32_t)key;
            unsigned long long prev =
                atomicCAS((unsigned long long*)jt.slots + s, (unsigned long long)EMPTY64, want);
            if (prev == EMPTY64) { placed = true; break; }
            if ((uint32_t)prev == (uint32_t)key) { atomicOr(b.err, ERR_DUP); placed = true; break; }
        } else {
            unsigned long long prev = atomicCAS((unsigned long long*)jt.slots + 2 * s,
                                                (unsigned long long)EMPTY64, (unsigned long long)key);
            if (prev == EMPTY64) {
                jt.slots[2 * s + 1] = payload;
                placed = true;
                break;
            }
            if (prev == (unsigned long long)key) { atomicOr(b.err, ERR_DUP); placed = true; break; }
        }
        s = (s + 1) & jt.mask;
    }
    if (!placed) atomicOr(b.err, ERR_INTERNAL);
}

// ------------------------------------------------------- global aggregation slot

// Slot of key in a hashed global table, claiming an empty slot for a new key;
// claimed is set when this call took a fresh slot.  Callers count their
// claims and add them to t.used in bulk (agg_add_claims): one counter word
// updated once per new key by every thread would serialise at its L2 slice.
// A table that fills up ends the probe with ERR_OVERFLOW.
__device__ __forceinline__ uint64_t* agg_slot(const AggTable& t, uint64_t key, uint32_t* err, bool& claimed) {
    claimed = false;
    if (key == EMPTY64) return t.slots + (t.mask + 1) * t.words;   // side slot
    uint64_t s = fmix64(key) & t.mask;
    for (uint64_t it = 0; it <= t.mask; ++it) {
        uint64_t* p = t.slots + s * t.words;
        uint64_t k = __ldcg((const unsigned long long*)p);
        if (k == key) return p;
        if (k == EMPTY64) {
            unsigned long long prev =
                atomicCAS((unsigned long long*)p, (unsigned long long)EMPTY64, (unsigned long long)key);
            if (prev == EMPTY64) {
                claimed = true;
                return p;
            }
            if (prev == key) return p;
        }
        s = (s + 1) & t.mask;
    }
    atomicOr(err, ERR_OVERFLOW);
    return nullptr;
}

// Slot of a key in either kind of global table (direct: key - kmin, in
// range by the column bounds the host checked; nothing is claimed).
__device__ __forceinline__ uint64_t* agg_slot_any(const AggTable& t, uint64_t key, uint32_t* err, bool& claimed) {
    claimed = false;
    if (t.split && (key < t.key_lo || key > t.key_hi)) return nullptr;   // another pass's key range
    if (t.direct) {
        const uint64_t s = key - t.kmin;
        if (s > t.mask) {
            atomicOr(err, ERR_INTERNAL);
            return nullptr;
        }
        return t.slots + s * t.words;
    }
    return agg_slot(t, key, err, claimed);
}

// Adds n claimed slots to the table's occupancy count; past max_used the
// execution is retried with a larger table (ERR_OVERFLOW).
__device__ __forceinline__ void agg_add_claims(const AggTable& t, uint32_t* err, uint32_t n) {
    if (n == 0 || t.direct) return;
    const unsigned long long u = atomicAdd(t.used, (unsigned long long)n);
    if (u + n > t.max_used) atomicOr(err, ERR_OVERFLOW);
}

// Warp-wide sum of per-lane claim counts, added to the table by lane 0.  All
// 32 lanes must call it.
__device__ __forceinline__ void agg_add_claims_warp(const AggTable& t, uint32_t* err, uint32_t n) {
    const uint32_t tot = __reduce_add_sync(0xffffffffu, n);
    if ((threadIdx.x & 31) == 0) agg_add_claims(t, err, tot);
}

}  // namespace tpk
