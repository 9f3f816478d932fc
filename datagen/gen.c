/*
 * Seeded, counter-based column generator for the synthetic star schema.
 *
 * This module only produces INPUT data.  It holds none of the query
 * arithmetic (no filter, join, grouping or aggregation): the oracle and the
 * CUDA path both consume its output and share nothing else.
 *
 * Every value is a pure function of (seed, stream, row index), so any row
 * range can be regenerated independently and in parallel:
 *
 *   key(seed, stream) = splitmix64_output(seed, stream)
 *   raw(key, i)       = splitmix64_output(key, i)
 *
 * where splitmix64_output(s, i) is the i-th output of the SplitMix64
 * generator started from state s (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): mix(s + (i+1) * gamma).
 *
 * Distributions built on raw():
 *   uniform [lo, hi]  : lo + floor(raw * (hi - lo + 1) / 2^64)   (multiply-high)
 *   permutation of [0,n): balanced 4-round Feistel network on the smallest
 *                       even-width power-of-two domain >= n, with
 *                       cycle-walking back into [0, n) (Black & Rogaway,
 *                       "Ciphers with arbitrary finite domains", 2002)
 *   Zipf(s) over n ranks: inverse CDF by binary search on a table of
 *                       normalised prefix sums of k^-s, k = 1..n
 *   lognormal         : exp(mu + sigma * z), z from the Box-Muller transform
 *                       of two uniforms (Box & Muller, 1958)
 *
 * Host C only; builds identically on x86-64 and AArch64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DG_GAMMA 0x9E3779B97F4A7C15ull

static inline uint64_t dg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t dg_stream_key(uint64_t seed, uint64_t stream) {
    return dg_mix(seed + (stream + 1ull) * DG_GAMMA);
}

static inline uint64_t dg_raw(uint64_t key, uint64_t i) {
    return dg_mix(key + (i + 1ull) * DG_GAMMA);
}

static inline uint64_t dg_mulhi(uint64_t a, uint64_t b) {
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

/* uniform integer in [lo, hi] (inclusive); hi >= lo */
static inline int64_t dg_uniform(uint64_t x, int64_t lo, int64_t hi) {
    uint64_t span = (uint64_t)hi - (uint64_t)lo + 1ull; /* 0 means 2^64 */
    if (span == 0) return (int64_t)x;
    return (int64_t)((uint64_t)lo + dg_mulhi(x, span));
}

/* uniform double in [0, 1) with 53 random bits */
static inline double dg_unit(uint64_t x) {
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

/* ---------------------------------------------------------------- permutation */

typedef struct {
    uint64_t key;
    uint64_t n;
    unsigned half;     /* bits per Feistel half */
    uint64_t hmask;
} dg_perm;

static dg_perm dg_perm_make(uint64_t key, uint64_t n) {
    dg_perm p;
    unsigned bits = 2;
    while (bits < 64 && (1ull << bits) < n) bits += 2;
    p.key = key;
    p.n = n;
    p.half = bits / 2;
    p.hmask = (p.half >= 64) ? ~0ull : ((1ull << p.half) - 1ull);
    return p;
}

static inline uint64_t dg_feistel(const dg_perm* p, uint64_t x) {
    uint64_t l = (x >> p->half) & p->hmask;
    uint64_t r = x & p->hmask;
    for (uint64_t round = 0; round < 4; ++round) {
        uint64_t f = dg_mix(p->key ^ (round * 0xD6E8FEB86659FD93ull) ^ r) & p->hmask;
        uint64_t nl = r;
        r = l ^ f;
        l = nl;
    }
    return (l << p->half) | r;
}

static inline uint64_t dg_perm_at(const dg_perm* p, uint64_t i) {
    uint64_t x = dg_feistel(p, i);
    while (x >= p->n) x = dg_feistel(p, x);
    return x;
}

/* ---------------------------------------------------------------- column fills */

/* kinds of columns */
enum {
    DG_UNIFORM = 0,   /* a..b uniform, times mult                        */
    DG_IOTA = 1,      /* row index + a                                   */
    DG_PERM = 2,      /* permutation of [0, n) at row index (n = b)      */
    DG_PERM_DIV = 3,  /* permutation of [0, n) at (row index >> a), n = b */
    DG_RAW64 = 4,     /* raw 64-bit output (unique per row)              */
    DG_MODULAR = 5,   /* ((row + a) mod b) * mult + c                    */
};

/* element types */
enum { DG_I32 = 0, DG_I64 = 1, DG_U8 = 2 };

static inline void dg_store(void* out, int type, uint64_t j, int64_t v) {
    switch (type) {
    case DG_I32: ((int32_t*)out)[j] = (int32_t)v; break;
    case DG_I64: ((int64_t*)out)[j] = v; break;
    default: ((uint8_t*)out)[j] = (uint8_t)v; break;
    }
}

/*
 * Fill out[0..n) with rows row0..row0+n-1 of one column.
 * kind/a/b/c/mult as in the enum above.  Returns 0, or -1 on bad arguments.
 */
int dg_fill(uint64_t seed, uint64_t stream, int kind, int type, int64_t a, int64_t b,
            int64_t c, int64_t mult, uint64_t row0, uint64_t n, void* out) {
    uint64_t key = dg_stream_key(seed, stream);
    if (type < DG_I32 || type > DG_U8) return -1;
    if (kind == DG_UNIFORM && b < a) return -1;
    if ((kind == DG_PERM || kind == DG_PERM_DIV || kind == DG_MODULAR) && b <= 0) return -1;
    if (kind == DG_PERM || kind == DG_PERM_DIV) {
        dg_perm p = dg_perm_make(key, (uint64_t)b);
        int shift = (kind == DG_PERM_DIV) ? (int)a : 0;
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < (int64_t)n; ++j)
            dg_store(out, type, (uint64_t)j, (int64_t)dg_perm_at(&p, (row0 + (uint64_t)j) >> shift));
        return 0;
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (int64_t)n; ++j) {
        uint64_t i = row0 + (uint64_t)j;
        int64_t v;
        switch (kind) {
        case DG_UNIFORM: v = dg_uniform(dg_raw(key, i), a, b) * mult; break;
        case DG_IOTA: v = (int64_t)i + a; break;
        case DG_RAW64: v = (int64_t)dg_raw(key, i); break;
        default: v = (int64_t)(((i + (uint64_t)a) % (uint64_t)b)) * mult + c; break;
        }
        dg_store(out, type, (uint64_t)j, v);
    }
    return (kind >= DG_UNIFORM && kind <= DG_MODULAR) ? 0 : -1;
}

/*
 * Row indices into a table of n_target rows, one per output row:
 *   dist 0: uniform over [0, n_target)
 *   dist 1: Zipf(s) rank r in [0, n_target) mapped through a seeded
 *           permutation, so the hottest rows are scattered
 * cdf must hold n_target doubles from dg_zipf_cdf (dist 1 only).
 */
int dg_fill_index(uint64_t seed, uint64_t stream, int dist, uint64_t n_target,
                  const double* cdf, uint64_t row0, uint64_t n, int64_t* out) {
    uint64_t key = dg_stream_key(seed, stream);
    if (n_target == 0) return -1;
    if (dist == 0) {
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < (int64_t)n; ++j)
            out[j] = dg_uniform(dg_raw(key, row0 + (uint64_t)j), 0, (int64_t)n_target - 1);
        return 0;
    }
    if (dist != 1 || cdf == NULL) return -1;
    dg_perm p = dg_perm_make(dg_mix(key ^ 0x5A5A5A5A5A5A5A5Aull), n_target);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (int64_t)n; ++j) {
        double u = dg_unit(dg_raw(key, row0 + (uint64_t)j));
        uint64_t lo = 0, hi = n_target - 1; /* first k with cdf[k] > u */
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (cdf[mid] > u) hi = mid; else lo = mid + 1;
        }
        out[j] = (int64_t)dg_perm_at(&p, lo);
    }
    return 0;
}

/* normalised prefix sums of k^-s for k = 1..n; cdf[n-1] == 1 */
int dg_zipf_cdf(double s, uint64_t n, double* cdf) {
    double acc = 0.0;
    if (n == 0) return -1;
    for (uint64_t k = 0; k < n; ++k) {
        acc += pow((double)(k + 1), -s);
        cdf[k] = acc;
    }
    for (uint64_t k = 0; k < n; ++k) cdf[k] /= acc;
    cdf[n - 1] = 1.0;
    return 0;
}

/* out[j] = table[idx[j]] for an int64 index column (gather a key column) */
int dg_gather(const void* table, int type, const int64_t* idx, uint64_t n, void* out) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (int64_t)n; ++j) {
        int64_t v;
        switch (type) {
        case DG_I32: v = ((const int32_t*)table)[idx[j]]; break;
        case DG_I64: v = ((const int64_t*)table)[idx[j]]; break;
        default: v = ((const uint8_t*)table)[idx[j]]; break;
        }
        dg_store(out, type, (uint64_t)j, v);
    }
    return 0;
}

/* n samples of round(exp(mu + sigma*z)) clamped to [lo, hi] */
int dg_lognormal(uint64_t seed, uint64_t stream, double mu, double sigma, int64_t lo, int64_t hi,
                 uint64_t n, int64_t* out) {
    uint64_t key = dg_stream_key(seed, stream);
    for (uint64_t j = 0; j < n; ++j) {
        double u1 = dg_unit(dg_raw(key, 2 * j));
        double u2 = dg_unit(dg_raw(key, 2 * j + 1));
        if (u1 <= 0.0) u1 = 1.0 / 9007199254740992.0;
        double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
        double v = exp(mu + sigma * z);
        int64_t r = (int64_t)llround(v);
        out[j] = r < lo ? lo : (r > hi ? hi : r);
    }
    return 0;
}

/* n samples of round(exp(uniform(ln lo, ln hi))), clamped to [lo, hi] */
int dg_loguniform(uint64_t seed, uint64_t stream, int64_t lo, int64_t hi, uint64_t n, int64_t* out) {
    uint64_t key = dg_stream_key(seed, stream);
    double a = log((double)lo), b = log((double)hi);
    for (uint64_t j = 0; j < n; ++j) {
        double v = exp(a + (b - a) * dg_unit(dg_raw(key, j)));
        int64_t r = (int64_t)llround(v);
        out[j] = r < lo ? lo : (r > hi ? hi : r);
    }
    return 0;
}

/* out[j] = raw 64-bit output of stream at row idx[j] (row-indexable RAW64 column) */
int dg_raw_at(uint64_t seed, uint64_t stream, const int64_t* idx, uint64_t n, int64_t* out) {
    uint64_t key = dg_stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (int64_t)n; ++j) out[j] = (int64_t)dg_raw(key, (uint64_t)idx[j]);
    return 0;
}
