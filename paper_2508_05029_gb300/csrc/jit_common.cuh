// Row evaluation of the run-time compiled kernels, specialised on a plan
// shape S (a struct of compile-time constants written by the host).
//
// Paper basis: Section 3.1 (operators over batches of equal-length columns),
// Section 3.2 (join), Section 4 (decimals held as 128-bit integers).  A
// consumer warp evaluates 32 * ST_RPL rows -- lane l takes rows l, l + 32, ...
// of a row block whose columns are given by pointers (a stage in shared
// memory, or the columns in device memory) -- through filter -> probe ->
// group key -> count and sums, accumulating into a dense table of G groups.
//
// A shape S provides:
//   filter, ftype            filter present; its column type (T_*)
//   join, ktype              J_NONE / J_DIRECT / J_HASH32 / J_HASH64; fk type
//   part                     partition filter on the join (hybrid join)
//   lip                      lookahead (Bloom) filter tested before the probe
//   nx, xjoin[], xktype[], xlip[]   further joins of a star query: kind, key
//                            column type, lookahead filter
//   gdim[]                   join whose payload holds dimension field F
//                            (0 = the first, 1 + j = further join j)
//   many                     the first join fans out (repeated build keys)
//   ng, gside[], gtype[], gbits[]   group fields, first field highest
//   ns, skind[], atype[], btype[]   sums: S_SUM / S_MUL_SUB and column types
//   mode[]                   1: low word, 2: low + carry word (fast), 0: exact
//   narrow[]                 mode 2 MUL_SUB operands proved to fit in int32
//   fast                     32-bit dense table (column bounds proved every
//                            sum stays inside int64); otherwise the table holds
//                            count[G], lo[s][G], hi[s][G] 64-bit words
//   lo_only                  (not fast) sums proved to stay inside int64: add
//                            64-bit terms to the low words only (the high words
//                            are their sign extension); otherwise exact 128-bit
// Runtime values (filter bounds, join table, term offsets, multipliers, the
// table's word layout) come from the launch, so one compiled kernel serves
// every plan and batch of the same shape.
#pragma once
// run-time compiled kernels have the registers to hold every row's probe
// sector at once
#define TP_PROBE_LOADS_FIRST 1
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

// Column ids of a shape's columns: filter, join key, fact group field F,
// sum I's first and second operand, further join J's key.
enum : int { CI_F = 0, CI_K = 1, CI_G = 2, CI_A = 2 + MAX_GROUP, CI_B = 2 + MAX_GROUP + MAX_SUM,
             CI_X = 2 + MAX_GROUP + 2 * MAX_SUM, CI_N = 2 + MAX_GROUP + 2 * MAX_SUM + MAX_XJOIN };

// Row evaluation reads column CI's value of row r0 + 32 j through a column
// source: ld<T, CI>(r0, j) (typed) and ld_lo<T, CI>(r0, j) (low 32 bits).
// Cols: the columns in device memory at a row block (row 0 of the block at
// each pointer); StageCols (jit_dense.cuh): a stage in shared memory;
// Eager: every column of the shape loaded into registers up front.
struct Cols {
    const unsigned char* p[CI_N];
    template <int T, int CI>
    __device__ __forceinline__ typename ColT<T>::type ld(uint32_t r0, int j) const {
        return lds<T>(p[CI], r0 + 32 * j);
    }
    template <int T, int CI>
    __device__ __forceinline__ uint32_t ld_lo(uint32_t r0, int j) const {
        return lds_lo<T>(p[CI], r0 + 32 * j);
    }
};

// Filter bounds, also clamped to int32 for narrow columns (1 > 0 when nothing
// passes).
struct Flt {
    int64_t lo, hi;
    int32_t lo32, hi32;
};

__device__ __forceinline__ Flt make_flt(const QueryDev& q) {
    Flt f;
    f.lo = q.flo;
    f.hi = q.fhi;
    if (q.flo > q.fhi || q.flo > INT32_MAX || q.fhi < INT32_MIN) {
        f.lo32 = 1;
        f.hi32 = 0;
    } else {
        f.lo32 = (int32_t)(q.flo < INT32_MIN ? (int64_t)INT32_MIN : q.flo);
        f.hi32 = (int32_t)(q.fhi > INT32_MAX ? (int64_t)INT32_MAX : q.fhi);
    }
    return f;
}

// The dense table rows accumulate into: G groups; fast: 32-bit words, block 0
// the counts, then per sum its low-word block and, in mode 2, a carry block
// (sum_word<S, I>), terms offset by sum_off[I]; exact: count[G], lo[s][G],
// hi[s][G] 64-bit words.
struct Tab {
    unsigned char* base;
    uint32_t G;
    const int64_t* sum_off;
};

// Block of sum I's low words in a fast table: 1 + the blocks of sums before it.
template <class S, int I>
__device__ __forceinline__ constexpr uint32_t sum_word() {
    uint32_t w = 1;
    for (int s = 0; s < I; ++s) w += (uint32_t)S::mode[s];
    return w;
}

// Group field F (compile-time recursion over the fields).
template <class S, int F, class C>
__device__ __forceinline__ void group_fields(const QueryDev& q, const C& c, uint32_t r0,
                                             const uint32_t (&pay)[1 + MAX_XJOIN][ST_RPL], uint32_t g[ST_RPL],
                                             uint32_t& pm) {
    if constexpr (F < S::ng) {
        constexpr int bits = S::gbits[F];
        if constexpr (S::gside[F] == 0) {
            constexpr int T = S::gtype[F];
            using U = typename ColT<T>::utype;
            uint32_t bad = 0;
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                const U v = (U)c.template ld<T, CI_G + F>(r0, j);
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
            for (int j = 0; j < ST_RPL; ++j) g[j] = (g[j] << bits) | ((pay[S::gdim[F]][j] >> pos) & mask);
        }
        group_fields<S, F + 1, C>(q, c, r0, pay, g, pm);
    }
}

// Sum I of the rows in pm (compile-time recursion over the sums).
template <class S, int I, class C>
__device__ __forceinline__ void sums(const QueryDev& q, const Tab& t, const C& c, uint32_t r0,
                                     const uint32_t g[ST_RPL], uint32_t pm) {
    if constexpr (I < S::ns) {
        constexpr int TA = S::atype[I];
        constexpr int TB = S::btype[I];
        constexpr bool MS = S::skind[I] == S_MUL_SUB;
        if constexpr (S::fast && S::mode[I] == 1) {
            // the sums of (term - offset) fit in 32 bits: only the low word of
            // every term matters, and it is exact mod 2^32
            uint32_t* lo = (uint32_t*)t.base + (uint64_t)sum_word<S, I>() * t.G;
            const uint32_t off = (uint32_t)(uint64_t)t.sum_off[I];
            const uint32_t k = (uint32_t)(uint64_t)q.sk[I];
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                uint32_t v = c.template ld_lo<TA, CI_A + I>(r0, j);
                if constexpr (MS) v *= k - c.template ld_lo<TB, CI_B + I>(r0, j);
                if (pm >> j & 1u) atomicAdd(lo + g[j], v - off);
            }
        } else if constexpr (S::fast) {
            uint32_t* lo = (uint32_t*)t.base + (uint64_t)sum_word<S, I>() * t.G;
            uint32_t* hi = lo + t.G;
            const int64_t off = t.sum_off[I];
            const int64_t k = q.sk[I];
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                int64_t v = (int64_t)c.template ld<TA, CI_A + I>(r0, j);
                if constexpr (MS) {
                    const int64_t d = k - (int64_t)c.template ld<TB, CI_B + I>(r0, j);
                    if constexpr (S::narrow[I]) v = (int64_t)(int32_t)v * (int64_t)(int32_t)d;
                    else v *= d;
                }
                const uint64_t w = (uint64_t)(v - off);
                if (pm >> j & 1u) {
                    const uint32_t old = atomicAdd(lo + g[j], (uint32_t)w);
                    const uint32_t h = (uint32_t)(w >> 32) + ((old + (uint32_t)w) < old ? 1u : 0u);
                    if (h) atomicAdd(hi + g[j], h);
                }
            }
        } else {
            uint64_t* lo = (uint64_t*)t.base + (uint64_t)t.G * (1 + 2 * I);
            uint64_t* hi = (uint64_t*)t.base + (uint64_t)t.G * (2 + 2 * I);
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                if (!(pm >> j & 1u)) continue;
                const int64_t a = (int64_t)c.template ld<TA, CI_A + I>(r0, j);
                if constexpr (S::lo_only) {
                    int64_t v = a;
                    if constexpr (MS) v *= q.sk[I] - (int64_t)c.template ld<TB, CI_B + I>(r0, j);
                    atomicAdd((unsigned long long*)(lo + g[j]), (unsigned long long)v);
                } else if constexpr (MS) {
                    atomic_add_i128(lo + g[j], hi + g[j],
                                    mul_sub(a, q.sk[I], (int64_t)c.template ld<TB, CI_B + I>(r0, j)));
                } else {
                    atomic_add_i128(lo + g[j], hi + g[j], i128_from_i64(a));
                }
            }
        }
        sums<S, I + 1, C>(q, t, c, r0, g, pm);
    }
}

// Group key, count and sums of the rows in pm, whose join payloads are pays.
template <class S, class C>
__device__ __forceinline__ void accumulate(const QueryDev& q, const Tab& t, const C& c, uint32_t r0,
                                           const uint32_t (&pays)[1 + MAX_XJOIN][ST_RPL], uint32_t pm) {
    uint32_t g[ST_RPL];
#pragma unroll
    for (int j = 0; j < ST_RPL; ++j) g[j] = 0;
    group_fields<S, 0, C>(q, c, r0, pays, g, pm);
    if (!pm) return;
#pragma unroll
    for (int j = 0; j < ST_RPL; ++j) {
        if (!(pm >> j & 1u)) continue;
        if constexpr (S::fast) atomicAdd((unsigned int*)t.base + g[j], 1u);
        else atomicAdd((unsigned long long*)t.base + g[j], 1ull);
    }
    sums<S, 0, C>(q, t, c, r0, g, pm);
}

// Star join: further join J (and the following ones) of the rows in pm --
// lookahead filter, probe of its own table, payload into pays[1 + J]; rows
// without a partner leave pm.
template <class S, int J, class C>
__device__ __forceinline__ void further_joins(const QueryDev& q, const C& c, uint32_t r0,
                                              uint32_t (&pays)[1 + MAX_XJOIN][ST_RPL], uint32_t& pm) {
    if constexpr (J < S::nx) {
        const JoinTable& jt = q.jtx[J];
        int64_t key[ST_RPL];
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) key[j] = (int64_t)c.template ld<S::xktype[J], CI_X + J>(r0, j);
        if constexpr (S::xlip[J]) lip_mask<ST_RPL>(jt, key, pm);
        uint32_t* pay = pays[1 + J];
        if constexpr (S::xjoin[J] == J_DIRECT) {
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                const uint64_t idx = (uint64_t)(key[j] - jt.kmin);
                pay[j] = ((pm >> j) & 1u) && idx < jt.range ? TP_LDT((const unsigned int*)jt.slots + idx) : EMPTY32;
            }
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j)
                if (pay[j] == EMPTY32) pm &= ~(1u << j);
        } else if constexpr (S::xjoin[J] == J_HASH32) {
            probe_rows_k32(jt, key, pm, pay, q.err);
        } else {
            probe_rows_k64(jt, key, pm, pay, q.err);
        }
        uint32_t bad = 0;
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) bad |= (uint32_t)((pay[j] & PAYLOAD_BAD) != 0) << j;
        if (bad & pm) {
            atomicOr(q.err, ERR_RANGE);
            pm &= ~bad;
        }
        if (!pm) return;
        further_joins<S, J + 1, C>(q, c, r0, pays, pm);
    }
}

// One warp's rows of a block (rows r0 + 32 j whose bit j is set in valid):
// filter -> probe -> group key -> count and sums.
template <class S, class C>
__device__ __forceinline__ void consume(const QueryDev& q, const Flt& flt, const Tab& t, const C& c, uint32_t r0,
                                        uint32_t valid) {
    uint32_t pm = valid;
    if constexpr (S::filter) {
        pm = 0;
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) {
            if constexpr (S::ftype == T_I64) {
                const int64_t v = c.template ld<T_I64, CI_F>(r0, j);
                pm |= (uint32_t)(v >= flt.lo && v <= flt.hi) << j;
            } else {
                const int32_t v = (int32_t)c.template ld<S::ftype, CI_F>(r0, j);
                pm |= (uint32_t)(v >= flt.lo32 && v <= flt.hi32) << j;
            }
        }
        pm &= valid;
        if (!pm) return;
    }
    uint32_t pays[1 + MAX_XJOIN][ST_RPL];   // payloads of the first join and the further ones
    uint32_t (&pay)[ST_RPL] = pays[0];
#pragma unroll
    for (int j = 0; j < ST_RPL; ++j) pay[j] = 0;
    if constexpr (S::join != J_NONE && S::lip) {
        int64_t key[ST_RPL];
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) key[j] = (int64_t)c.template ld<S::ktype, CI_K>(r0, j);
        lip_mask<ST_RPL>(q.jt, key, pm);
        if (!pm) return;
    }
    if constexpr (S::join == J_DIRECT) {
        const unsigned int* dt = (const unsigned int*)q.jt.slots;
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) {
            const uint64_t idx = (uint64_t)((int64_t)c.template ld<S::ktype, CI_K>(r0, j) - q.jt.kmin);
            pay[j] = ((pm >> j) & 1u) && idx < q.jt.range ? TP_LDT(dt + idx) : EMPTY32;
        }
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j)
            if (pay[j] == EMPTY32) pm &= ~(1u << j);
    } else if constexpr (S::join == J_HASH32 || S::join == J_HASH64) {
        int64_t key[ST_RPL];
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) key[j] = (int64_t)c.template ld<S::ktype, CI_K>(r0, j);
        if constexpr (S::part) {
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j)
                if (!part_resident(q.jt, key[j])) pm &= ~(1u << j);
        }
        if constexpr (S::join == J_HASH32) probe_rows_k32(q.jt, key, pm, pay, q.err);
        else probe_rows_k64(q.jt, key, pm, pay, q.err);
    }
    if constexpr (S::join != J_NONE) {
        uint32_t bad = 0;
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) bad |= (uint32_t)((pay[j] & PAYLOAD_BAD) != 0) << j;
        if (bad & pm) {
            atomicOr(q.err, ERR_RANGE);
            pm &= ~bad;
        }
        if (!pm) return;
    }
    if constexpr (S::nx > 0) {
        further_joins<S, 0, C>(q, c, r0, pays, pm);
        if (!pm) return;
    }
    if constexpr (S::many) {
        // fan-out: pay[j] is the first row of the key's run in the sorted
        // build rows; pair the row with each row of the run in turn
        uint32_t first[ST_RPL];
        int64_t key[ST_RPL];
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) {
            first[j] = pay[j];
            key[j] = (int64_t)c.template ld<S::ktype, CI_K>(r0, j);
        }
        uint32_t live = pm;
        for (uint32_t m = 0; live; ++m) {
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) {
                if (!((live >> j) & 1u)) continue;
                const uint64_t at = (uint64_t)first[j] + m;
                if (at < q.jt.mn && TP_LDT(q.jt.mkeys + at) == (uint64_t)key[j]) pay[j] = TP_LDT(q.jt.mpay + at);
                else live &= ~(1u << j);
            }
            uint32_t pmm = live, bad = 0;
#pragma unroll
            for (int j = 0; j < ST_RPL; ++j) bad |= (uint32_t)((pay[j] & PAYLOAD_BAD) != 0) << j;
            if (bad & pmm) {
                atomicOr(q.err, ERR_RANGE);
                pmm &= ~bad;
            }
            if (pmm) accumulate<S, C>(q, t, c, r0, pays, pmm);
        }
        return;
    }
    accumulate<S, C>(q, t, c, r0, pays, pm);
}

// Column pointers of a block starting at row `row` of the query's columns in
// device memory (compile-time recursion over the fields and sums).
template <class S, int F, int I>
__device__ __forceinline__ void query_cols_rest(const QueryDev& q, uint64_t row, Cols& c) {
    if constexpr (F < S::ng) {
        if constexpr (S::gside[F] == 0)
            c.p[CI_G + F] = (const unsigned char*)q.gcol[F].ptr + row * sizeof(typename ColT<S::gtype[F]>::type);
        query_cols_rest<S, F + 1, I>(q, row, c);
    } else if constexpr (I < S::ns) {
        c.p[CI_A + I] = (const unsigned char*)q.sa[I].ptr + row * sizeof(typename ColT<S::atype[I]>::type);
        if constexpr (S::skind[I] == S_MUL_SUB)
            c.p[CI_B + I] = (const unsigned char*)q.sb[I].ptr + row * sizeof(typename ColT<S::btype[I]>::type);
        query_cols_rest<S, F, I + 1>(q, row, c);
    }
}

template <class S, int J>
__device__ __forceinline__ void query_cols_x(const QueryDev& q, uint64_t row, Cols& c) {
    if constexpr (J < S::nx) {
        c.p[CI_X + J] = (const unsigned char*)q.fkx[J].ptr + row * sizeof(typename ColT<S::xktype[J]>::type);
        query_cols_x<S, J + 1>(q, row, c);
    }
}

template <class S>
__device__ __forceinline__ Cols query_cols(const QueryDev& q, uint64_t row) {
    Cols c{};
    if constexpr (S::filter) c.p[CI_F] = (const unsigned char*)q.fcol.ptr + row * sizeof(typename ColT<S::ftype>::type);
    if constexpr (S::join != J_NONE)
        c.p[CI_K] = (const unsigned char*)q.fk.ptr + row * sizeof(typename ColT<S::ktype>::type);
    query_cols_rest<S, 0, 0>(q, row, c);
    query_cols_x<S, 0>(q, row, c);
    return c;
}

// Every column of shape S for this lane's rows r0 + 32 j (bit j of valid),
// loaded from a column source into registers at once: with columns in device
// memory the loads of all columns overlap instead of following the filter,
// probe and group-key dependencies one by one.
template <class S, int CI>
struct ColType {   // element type of column CI in shape S (T_I64 for columns the shape does not read)
    static constexpr int t = CI == CI_F ? (S::filter ? S::ftype : T_I64)
                           : CI == CI_K ? (S::join != J_NONE ? S::ktype : T_I64)
                           : CI < CI_A ? (CI - CI_G < S::ng && S::gside[CI - CI_G] == 0 ? S::gtype[CI - CI_G] : T_I64)
                           : CI < CI_B ? (CI - CI_A < S::ns ? S::atype[CI - CI_A] : T_I64)
                           : CI < CI_X ? (CI - CI_B < S::ns && S::skind[CI - CI_B] == S_MUL_SUB ? S::btype[CI - CI_B]
                                                                                               : T_I64)
                           : (CI - CI_X < S::nx ? S::xktype[CI - CI_X] : T_I64);
    static constexpr bool used = CI == CI_F ? (bool)S::filter
                               : CI == CI_K ? S::join != J_NONE
                               : CI < CI_A ? (CI - CI_G < S::ng && S::gside[CI - CI_G] == 0)
                               : CI < CI_B ? (CI - CI_A < S::ns)
                               : CI < CI_X ? (CI - CI_B < S::ns && S::skind[CI - CI_B] == S_MUL_SUB)
                               : (CI - CI_X < S::nx);
};

template <class S>
struct Eager {
    uint64_t v[CI_N][ST_RPL];
    template <int CI, class C>
    __device__ __forceinline__ void fill(const C& c, uint32_t r0, uint32_t valid) {
        if constexpr (CI < CI_N) {
            if constexpr (ColType<S, CI>::used) {
#pragma unroll
                for (int j = 0; j < ST_RPL; ++j)
                    v[CI][j] = (valid >> j & 1u) ? (uint64_t)(int64_t)c.template ld<ColType<S, CI>::t, CI>(r0, j) : 0;
            }
            fill<CI + 1>(c, r0, valid);
        }
    }
    template <int T, int CI>
    __device__ __forceinline__ typename ColT<T>::type ld(uint32_t, int j) const {
        return (typename ColT<T>::type)v[CI][j];
    }
    template <int T, int CI>
    __device__ __forceinline__ uint32_t ld_lo(uint32_t, int j) const {
        return (uint32_t)v[CI][j];
    }
};

}  // namespace tpj

