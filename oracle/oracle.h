/*
 * TEST INFRASTRUCTURE ONLY.  The oracle: a plain, slow, single-threaded CPU
 * evaluation of the relational query the GPU path computes.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may call it; the
 * product library never links or loads it.  It shares no code, header, table
 * or constant with the CUDA path.
 *
 * What it computes (the plain relational definition; Section 3.1 of the paper
 * describes batches as row slices of equal-length columns and operators such as
 * Filter and Join over them; Section 4 states decimal(11,2) values held in
 * 128-bit integers):
 *
 *   R = { (g, aggregates) : f in Fact, d in Dim, e_j in Dim_j (j < n_extra_dims),
 *         filter_lo <= f.filter_col <= filter_hi,
 *         dim_filter_lo <= d.dim_filter_col <= dim_filter_hi, f.fk == d.pk,
 *         the same for every further dimension e_j on its own foreign key,
 *         g = packed(group fields of f, d and the e_j) }
 *
 * sorted ascending by the packed 64-bit key g.
 */
#ifndef THESEUS_ORACLE_H
#define THESEUS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_I32 = 0, ORC_I64 = 1, ORC_U8 = 2 };
enum { ORC_SUM = 0, ORC_SUM_MUL_SUB = 1, ORC_COUNT = 2, ORC_AVG = 3 };
enum { ORC_OK = 0, ORC_INVALID = 1, ORC_DUP_KEY = 4, ORC_RANGE = 8, ORC_NOMEM = 9 };

typedef struct {
    int32_t type;        /* ORC_I32 / ORC_I64 / ORC_U8 */
    const void* data;    /* n values */
} orc_column;

typedef struct {
    int32_t kind;        /* ORC_SUM, ORC_SUM_MUL_SUB, ORC_COUNT, ORC_AVG */
    int32_t col_a;       /* fact column of SUM / AVG, or the factor a */
    int32_t col_b;       /* fact column b of SUM_MUL_SUB */
    int64_t k;           /* constant K of SUM_MUL_SUB: sum of a*(K-b) */
} orc_agg;

typedef struct {
    uint64_t n_fact;
    int32_t n_fact_cols;
    const orc_column* fact;
    uint64_t n_dim;
    int32_t n_dim_cols;
    const orc_column* dim;
    int32_t filter_col;              /* fact column, or -1 for no filter */
    int64_t filter_lo, filter_hi;    /* inclusive */
    int32_t join_fact_col;           /* -1: no join */
    int32_t join_dim_col;
    int32_t n_group;                 /* 0..4 fields */
    int32_t group_side[4];           /* 0 = fact, 1 = dim, 2 + j = further dimension j */
    int32_t group_col[4];
    int32_t group_bits[4];           /* 1..64, total <= 64 */
    int32_t n_agg;                   /* 0..8 */
    orc_agg aggs[8];
    /* dimension predicate: only dimension rows with lo <= value <= hi join
     * (and only their keys must be unique); column -1 = every row */
    int32_t dim_filter_col;
    int64_t dim_filter_lo, dim_filter_hi;
    /* further dimensions of a star join, each joined like the first on its
     * own fact foreign key; group_side 2 + j reads further dimension j */
    int32_t n_extra_dims;                /* 0..3; needs the first join */
    uint64_t n_xdim[3];
    int32_t n_xdim_cols[3];
    const orc_column* xdim[3];
    int32_t xjoin_fact_col[3], xjoin_dim_col[3];
    int32_t xdim_filter_col[3];          /* -1: every row */
    int64_t xdim_filter_lo[3], xdim_filter_hi[3];
    /* first join with repeated build keys allowed: a fact row pairs with
     * every admitted dimension row holding its key (fan-out), and every pair
     * counts once in its group */
    int32_t join_many;
} orc_query;

typedef struct {
    uint64_t n_groups;
    uint64_t* keys;      /* [n_groups] ascending */
    int64_t* counts;     /* [n_groups] rows per group */
    uint64_t* sums;      /* [n_groups][n_agg][2] int128 as (lo, hi) words */
    double* avgs;        /* [n_groups][n_agg]; AVG entries only, else 0 */
} orc_result;

/* Evaluates q; on ORC_OK fills *out (free with orc_free). */
int32_t orc_run(const orc_query* q, orc_result* out);
void orc_free(orc_result* r);

/* (double) of a 128-bit integer given as (lo, hi) words, as C converts it. */
double orc_i128_to_double(uint64_t lo, int64_t hi);

#ifdef __cplusplus
}
#endif
#endif
