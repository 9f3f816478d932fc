/*
 * TEST INFRASTRUCTURE ONLY -- the oracle.  Plain, slow, single-threaded C.
 * Only tests, the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * It writes out the relational definition of the query directly:
 *   1. Filter (Section 3.1, the Filter operator): keep fact row f when
 *      lo <= f.filter_col <= hi.
 *   2. Join (Section 3.2, the Adaptive Join; here a PK-FK inner equi-join):
 *      pair f with the unique dimension row d whose key equals f's foreign
 *      key; rows without a partner drop out.  A dimension predicate, when
 *      given, first keeps only dimension rows with lo <= d.col <= hi (the
 *      predicate whose surviving keys lookahead information passing,
 *      Section 5, hands to the fact side).  The surviving dimension keys are
 *      sorted and searched by bisection; duplicates among them are an error.
 *      A star join repeats this for every further dimension, each on its own
 *      fact foreign key: a fact row survives only with a partner in all.
 *      With join_many the first dimension's keys may repeat: the fact row
 *      pairs with each of its partners there, and every pair is a row of the
 *      join (the relational inner join without the key constraint).
 *   3. Group and aggregate: the group key concatenates the group fields, the
 *      first field in the highest bits.  Surviving (key, row) pairs are sorted
 *      and each run of equal keys is reduced with exact 128-bit integer sums
 *      (Section 4: decimals held as 128-bit integers).  AVG is one IEEE
 *      double division of the exact sum, converted to double, by the count.
 * No step is blocked, fused or reordered beyond that definition.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

static int64_t col_at(const orc_column* c, uint64_t i) {
    switch (c->type) {
    case ORC_I32: return ((const int32_t*)c->data)[i];
    case ORC_I64: return ((const int64_t*)c->data)[i];
    default: return ((const uint8_t*)c->data)[i];
    }
}

typedef struct { int64_t key; uint64_t row; } key_row;

static int cmp_key_row_signed(const void* a, const void* b) {
    const key_row* x = (const key_row*)a;
    const key_row* y = (const key_row*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->row < y->row ? -1 : (x->row > y->row);
}

static int cmp_key_row_unsigned(const void* a, const void* b) {
    const key_row* x = (const key_row*)a;
    const key_row* y = (const key_row*)b;
    uint64_t kx = (uint64_t)x->key, ky = (uint64_t)y->key;
    if (kx != ky) return kx < ky ? -1 : 1;
    return x->row < y->row ? -1 : (x->row > y->row);
}

/* dimension row holding key k, or -1 */
static int64_t find_dim_row(const key_row* sorted, uint64_t n, int64_t k) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (sorted[mid].key < k) lo = mid + 1; else hi = mid;
    }
    return (lo < n && sorted[lo].key == k) ? (int64_t)sorted[lo].row : -1;
}

static int valid_col(int32_t c, int32_t n) { return c >= 0 && c < n; }

/* One joined dimension: its table, join columns and predicate. */
typedef struct {
    uint64_t n;
    int32_t n_cols;
    const orc_column* cols;
    int32_t fact_col, key_col;
    int32_t filter_col;
    int64_t filter_lo, filter_hi;
} dim_side;

/* Dimension k of the query: 0 = the first join, 1 + j = further dimension j. */
static dim_side side_of(const orc_query* q, int k) {
    dim_side d;
    if (k == 0) {
        d.n = q->n_dim; d.n_cols = q->n_dim_cols; d.cols = q->dim;
        d.fact_col = q->join_fact_col; d.key_col = q->join_dim_col;
        d.filter_col = q->dim_filter_col; d.filter_lo = q->dim_filter_lo; d.filter_hi = q->dim_filter_hi;
    } else {
        int j = k - 1;
        d.n = q->n_xdim[j]; d.n_cols = q->n_xdim_cols[j]; d.cols = q->xdim[j];
        d.fact_col = q->xjoin_fact_col[j]; d.key_col = q->xjoin_dim_col[j];
        d.filter_col = q->xdim_filter_col[j]; d.filter_lo = q->xdim_filter_lo[j]; d.filter_hi = q->xdim_filter_hi[j];
    }
    return d;
}

static int n_dims(const orc_query* q) { return q->join_fact_col < 0 ? 0 : 1 + q->n_extra_dims; }

static int32_t validate(const orc_query* q) {
    int total = 0;
    if (q->n_group < 0 || q->n_group > 4 || q->n_agg < 0 || q->n_agg > 8) return ORC_INVALID;
    if (q->filter_col >= 0 && !valid_col(q->filter_col, q->n_fact_cols)) return ORC_INVALID;
    if (q->n_extra_dims < 0 || q->n_extra_dims > 3 || (q->n_extra_dims > 0 && q->join_fact_col < 0))
        return ORC_INVALID;
    for (int k = 0; k < n_dims(q); ++k) {
        dim_side d = side_of(q, k);
        if (!valid_col(d.fact_col, q->n_fact_cols) || !valid_col(d.key_col, d.n_cols)) return ORC_INVALID;
        if (d.filter_col >= 0 && !valid_col(d.filter_col, d.n_cols)) return ORC_INVALID;
    }
    if (q->join_fact_col < 0 && q->dim_filter_col >= 0) return ORC_INVALID;
    for (int g = 0; g < q->n_group; ++g) {
        int bits = q->group_bits[g];
        if (bits < 1 || bits > 64) return ORC_INVALID;
        total += bits;
        int side = q->group_side[g];
        if (side == 0) {
            if (!valid_col(q->group_col[g], q->n_fact_cols)) return ORC_INVALID;
        } else {
            if (side < 1 || side > n_dims(q) || !valid_col(q->group_col[g], side_of(q, side - 1).n_cols))
                return ORC_INVALID;
        }
    }
    if (total > 64) return ORC_INVALID;
    for (int a = 0; a < q->n_agg; ++a) {
        const orc_agg* ag = &q->aggs[a];
        if (ag->kind == ORC_SUM || ag->kind == ORC_AVG) {
            if (!valid_col(ag->col_a, q->n_fact_cols)) return ORC_INVALID;
        } else if (ag->kind == ORC_SUM_MUL_SUB) {
            if (!valid_col(ag->col_a, q->n_fact_cols) || !valid_col(ag->col_b, q->n_fact_cols))
                return ORC_INVALID;
        } else if (ag->kind != ORC_COUNT) {
            return ORC_INVALID;
        }
    }
    return ORC_OK;
}

double orc_i128_to_double(uint64_t lo, int64_t hi) {
    i128 v = (i128)(((u128)(uint64_t)hi << 64) | (u128)lo);
    return (double)v;
}

int32_t orc_run(const orc_query* q, orc_result* out) {
    int32_t rc = validate(q);
    memset(out, 0, sizeof(*out));
    if (rc != ORC_OK) return rc;
    key_row* kept = NULL;
    uint64_t n_kept = 0;

    /* Join sides: keep each dimension's rows its predicate admits, sort
     * their (pk, row) and reject duplicate keys. */
    const int nd = n_dims(q);
    key_row* dim[4] = {NULL, NULL, NULL, NULL};
    uint64_t n_adm[4] = {0, 0, 0, 0};
    for (int k = 0; k < nd; ++k) {
        dim_side ds = side_of(q, k);
        if (ds.n == 0) continue;
        dim[k] = (key_row*)malloc(ds.n * sizeof(key_row));
        if (!dim[k]) { rc = ORC_NOMEM; goto out; }
        for (uint64_t i = 0; i < ds.n; ++i) {
            if (ds.filter_col >= 0) {
                int64_t v = col_at(&ds.cols[ds.filter_col], i);
                if (v < ds.filter_lo || v > ds.filter_hi) continue;
            }
            dim[k][n_adm[k]].key = col_at(&ds.cols[ds.key_col], i);
            dim[k][n_adm[k]].row = i;
            ++n_adm[k];
        }
        qsort(dim[k], n_adm[k], sizeof(key_row), cmp_key_row_signed);
        if (k == 0 && q->join_many) continue;   /* repeated keys are partners, not an error */
        for (uint64_t i = 1; i < n_adm[k]; ++i)
            if (dim[k][i].key == dim[k][i - 1].key) { rc = ORC_DUP_KEY; goto out; }
    }

    /* Filter, join and key every fact row; keep (group key, fact row) per
     * joined row. */
    uint64_t cap_kept = q->n_fact ? q->n_fact : 1;
    kept = (key_row*)malloc(cap_kept * sizeof(key_row));
    if (!kept) { rc = ORC_NOMEM; goto out; }
    for (uint64_t i = 0; i < q->n_fact; ++i) {
        if (q->filter_col >= 0) {
            int64_t v = col_at(&q->fact[q->filter_col], i);
            if (v < q->filter_lo || v > q->filter_hi) continue;
        }
        int64_t d[4] = {-1, -1, -1, -1};
        int joined = 1;
        for (int k = 0; k < nd && joined; ++k) {
            dim_side ds = side_of(q, k);
            d[k] = dim[k] ? find_dim_row(dim[k], n_adm[k], col_at(&q->fact[ds.fact_col], i)) : -1;
            joined = d[k] >= 0;
        }
        if (!joined) continue;
        /* partners in the first dimension: one, or with join_many every
         * admitted row with the key (the sorted run starting at the first) */
        uint64_t first = 0, n_partner = 1;
        if (nd > 0 && q->join_many) {
            const int64_t fk = col_at(&q->fact[q->join_fact_col], i);
            uint64_t lo = 0, hi = n_adm[0];
            while (lo < hi) {
                uint64_t mid = lo + (hi - lo) / 2;
                if (dim[0][mid].key < fk) lo = mid + 1; else hi = mid;
            }
            first = lo;
            n_partner = 0;
            while (first + n_partner < n_adm[0] && dim[0][first + n_partner].key == fk) ++n_partner;
        }
        for (uint64_t m = 0; m < n_partner; ++m) {
        if (nd > 0 && q->join_many) d[0] = (int64_t)dim[0][first + m].row;
        uint64_t key = 0;
        for (int g = 0; g < q->n_group; ++g) {
            int bits = q->group_bits[g];
            int side = q->group_side[g];
            int64_t v = side == 0 ? col_at(&q->fact[q->group_col[g]], i)
                                  : col_at(&side_of(q, side - 1).cols[q->group_col[g]], (uint64_t)d[side - 1]);
            if (bits < 64) {
                if (v < 0 || (uint64_t)v >= (1ull << bits)) { rc = ORC_RANGE; goto out; }
                key = (key << bits) | (uint64_t)v;
            } else {
                key = (uint64_t)v;
            }
        }
        if (n_kept == cap_kept) {
            key_row* grown = (key_row*)realloc(kept, 2 * cap_kept * sizeof(key_row));
            if (!grown) { rc = ORC_NOMEM; goto out; }
            kept = grown;
            cap_kept *= 2;
        }
        kept[n_kept].key = (int64_t)key;
        kept[n_kept].row = i;
        ++n_kept;
        }
    }
    for (int k = 0; k < 4; ++k) { free(dim[k]); dim[k] = NULL; }
    qsort(kept, n_kept, sizeof(key_row), cmp_key_row_unsigned);

    /* Count groups, then reduce each run of equal keys. */
    uint64_t n_groups = 0;
    for (uint64_t i = 0; i < n_kept; ++i)
        if (i == 0 || kept[i].key != kept[i - 1].key) ++n_groups;
    int na = q->n_agg;
    out->n_groups = n_groups;
    out->keys = (uint64_t*)malloc((n_groups ? n_groups : 1) * sizeof(uint64_t));
    out->counts = (int64_t*)malloc((n_groups ? n_groups : 1) * sizeof(int64_t));
    out->sums = (uint64_t*)calloc((n_groups ? n_groups : 1) * (na ? na : 1) * 2, sizeof(uint64_t));
    out->avgs = (double*)calloc((n_groups ? n_groups : 1) * (na ? na : 1), sizeof(double));
    if (!out->keys || !out->counts || !out->sums || !out->avgs) {
        free(kept); orc_free(out);
        return ORC_NOMEM;
    }
    uint64_t g = 0, start = 0;
    while (start < n_kept) {
        uint64_t end = start;
        while (end < n_kept && kept[end].key == kept[start].key) ++end;
        int64_t count = (int64_t)(end - start);
        out->keys[g] = (uint64_t)kept[start].key;
        out->counts[g] = count;
        for (int a = 0; a < na; ++a) {
            const orc_agg* ag = &q->aggs[a];
            u128 s = 0; /* wraps modulo 2^128, like any fixed-width sum */
            for (uint64_t r = start; r < end; ++r) {
                uint64_t i = kept[r].row;
                if (ag->kind == ORC_SUM || ag->kind == ORC_AVG) {
                    s += (u128)(i128)col_at(&q->fact[ag->col_a], i);
                } else if (ag->kind == ORC_SUM_MUL_SUB) {
                    i128 av = col_at(&q->fact[ag->col_a], i);
                    i128 bv = col_at(&q->fact[ag->col_b], i);
                    s += (u128)(av * ((i128)ag->k - bv)); /* |product| < 2^127 */
                } else {
                    s += 1;
                }
            }
            out->sums[(g * na + a) * 2] = (uint64_t)s;
            out->sums[(g * na + a) * 2 + 1] = (uint64_t)(s >> 64);
            if (ag->kind == ORC_AVG)
                out->avgs[g * na + a] = (double)(i128)s / (double)count;
        }
        ++g;
        start = end;
    }
    free(kept);
    return ORC_OK;
out:
    for (int k = 0; k < 4; ++k) free(dim[k]);
    free(kept);
    return rc;
}

void orc_free(orc_result* r) {
    free(r->keys);
    free(r->counts);
    free(r->sums);
    free(r->avgs);
    memset(r, 0, sizeof(*r));
}
