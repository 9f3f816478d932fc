/*
 * theseus_gb.h -- C ABI of the GB300 relational hot path.
 *
 * One GPU, one process.  The library evaluates
 *
 *     SELECT g, SUM(..), SUM(a*(K-b)), COUNT(*), AVG(..)
 *     FROM fact [JOIN dim ON fact.fk = dim.pk]
 *     WHERE lo <= fact.c <= hi
 *     GROUP BY g
 *
 * over columnar tables (paper, Section 3.1: a batch is a slice of all columns
 * of a table with the same number of rows).  Decimals are scaled 64-bit
 * integers; every SUM is an exact 128-bit integer (Section 4 holds
 * decimal(11,2) values in 128 bits).  AVG is the exact sum, rounded to double,
 * divided by the count in one IEEE double division.
 *
 * Conventions for every call:
 *   - Returns tp_status: TP_OK (0) or a TP_E_* code.  No C++ exception ever
 *     crosses this boundary.  After an error, tp_last_error() returns a
 *     human-readable message for the calling thread.
 *   - Objects (engine, tables, plans, results) are opaque and owned by the
 *     library until the matching *_destroy / *_free / tp_shutdown.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     device memory of the engine's GPU.  Caller buffers passed in are only
 *     read during the call unless stated otherwise.
 *   - One engine may be used from several host threads; calls on one engine
 *     serialise internally where they touch shared state.
 */
#ifndef THESEUS_GB_H
#define THESEUS_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */

typedef int32_t tp_status;
enum {
    TP_OK = 0,
    TP_E_INVALID = 1,     /* bad argument, plan or call order                 */
    TP_E_POOL_EMPTY = 2,  /* the pinned page pool has no free page            */
    TP_E_BUDGET = 3,      /* the device-memory reservation does not fit       */
    TP_E_DUP_KEY = 4,     /* the join's build side holds a key twice          */
    TP_E_TIMEOUT = 5,     /* a bounded wait expired (host or device side)     */
    TP_E_CUDA = 6,        /* a CUDA runtime call failed                       */
    TP_E_INTERNAL = 7,    /* a device-side consistency check failed           */
    TP_E_RANGE = 8,       /* a group field value does not fit its bit width   */
    TP_E_NOMEM = 9        /* host allocation failed                           */
};

/* ----------------------------------------------------------------- engine */

typedef struct tp_engine tp_engine;
typedef struct tp_table tp_table;
typedef struct tp_plan tp_plan;
typedef struct tp_result tp_result;

enum { TP_AGG_AUTO = 0, TP_AGG_SHARED = 1, TP_AGG_GLOBAL = 2 };

/*
 * Engine configuration.  Start from tp_config_default() and change fields.
 *
 *   page_bytes, n_pages   the pinned host page pool, allocated once in
 *                         tp_init (Section 3.4: a pool of pre-allocated
 *                         fixed-size page-locked buffers, allocated during
 *                         engine initialisation).  page_bytes is rounded up
 *                         to a multiple of 4096.  n_pages may be 0.
 *   device_budget_bytes   cap on device bytes the engine may reserve
 *                         (Section 3.3.2: tasks reserve memory before they
 *                         run).  0 = 90% of the GPU's free memory at init.
 *   prefetch_depth        batches copied ahead of compute on the copy stream
 *                         (Section 3.3.3, compute-task pre-loading).  0 =
 *                         no prefetch: the compute stream copies each batch
 *                         itself before using it.
 *   batch_rows            default rows per batch for host-page tables.
 *   cuda_device           CUDA device ordinal.
 *   load_factor           target fill of the hash tables, in (0.05, 0.9].
 *   agg_strategy          TP_AGG_AUTO, TP_AGG_SHARED (per-CTA shared-memory
 *                         tables, few groups) or TP_AGG_GLOBAL (one device
 *                         hash table).
 *   compute_stream        optional cudaStream_t (as void*) on which all
 *                         compute work is issued; NULL = engine-owned stream.
 *   flags                 TP_FLAG_TIME_KERNELS: bracket every fused
 *                         filter/probe/aggregate launch with CUDA events on
 *                         the compute stream and accumulate its device time
 *                         in tp_stats (agg_kernel_ms, agg_kernel_launches).
 *                         TP_FLAG_NO_STAGED: never use the bulk-copy staged
 *                         kernels (plain-load kernels only).
 *                         TP_FLAG_EXACT_ONLY: never use 64-bit accumulation,
 *                         even where column bounds prove it cannot overflow.
 *                         TP_FLAG_NO_DIRECT_JOIN: always hash the join keys,
 *                         even when they are dense enough for a
 *                         direct-mapped table (key range <= 2 x rows).
 *                         TP_FLAG_NO_DIRECT_AGG: always hash the group keys of
 *                         the device-memory aggregation, even when column
 *                         bounds show a dense key range (a direct-addressed
 *                         table needs no probing and yields sorted groups).
 *                         TP_FLAG_RAW_PAGES: store appended columns in pages
 *                         at their full width.  Without it every batch stores
 *                         each integer column as (value - the batch's minimum)
 *                         bit-packed in the fewest bits that hold the batch's
 *                         range (up to 31; 8, 16 and 32 bits as plain bytes,
 *                         words), and the device widens it after the copy:
 *                         fewer bytes cross the host link.
 *                         TP_FLAG_NO_JIT: never compile plan-specialised
 *                         kernels at run time (NVRTC); the ahead-of-time
 *                         staged kernels run every shape.  Without the flag a
 *                         plan shape is compiled once per process on first
 *                         use (tens to hundreds of milliseconds) and cached;
 *                         when the run-time compiler cannot be loaded or
 *                         fails, the ahead-of-time kernels run instead and
 *                         tp_stats counts the failure.
 */
enum {
    TP_FLAG_TIME_KERNELS = 1,
    TP_FLAG_NO_STAGED = 2,
    TP_FLAG_EXACT_ONLY = 4,
    TP_FLAG_NO_DIRECT_JOIN = 8,
    TP_FLAG_NO_JIT = 16,
    TP_FLAG_NO_DIRECT_AGG = 32,
    TP_FLAG_RAW_PAGES = 64
};
typedef struct {
    uint64_t page_bytes;
    uint32_t n_pages;
    uint32_t flags;
    uint64_t device_budget_bytes;
    int32_t prefetch_depth;
    int32_t cuda_device;
    uint64_t batch_rows;
    float load_factor;
    int32_t agg_strategy;
    void* compute_stream;
} tp_config;

/* Fills *cfg with defaults: 64 MiB pages, 0 pages, budget 0 (auto),
 * prefetch_depth 2, batch_rows 4M, device 0, load_factor 0.5, AUTO. */
void tp_config_default(tp_config* cfg);

/* Creates an engine on cfg->cuda_device: pins the page pool, creates the
 * copy and compute streams.  *out receives the engine.
 * Errors: TP_E_INVALID (bad config), TP_E_CUDA, TP_E_NOMEM. */
tp_status tp_init(const tp_config* cfg, tp_engine** out);

/* Waits for outstanding work, frees every table, plan, result, page and
 * stream of the engine.  NULL is ignored. */
void tp_shutdown(tp_engine* eng);

/* ---------------------------------------------------------------- page pool */

/* A page is an index into the engine's pool (Section 3.4). */
typedef uint32_t tp_page;

/* Takes one free page.  O(1); never allocates.  TP_E_POOL_EMPTY if none. */
tp_status tp_page_alloc(tp_engine* eng, tp_page* out);
/* Returns a page to the pool.  TP_E_INVALID if it is not currently lent out. */
tp_status tp_page_free(tp_engine* eng, tp_page page);
/* Host address of a page (page-locked, page_bytes long), or NULL. */
void* tp_page_ptr(tp_engine* eng, tp_page page);
/* Size of every page in bytes. */
uint64_t tp_page_bytes(const tp_engine* eng);
/* Pages currently free in the pool. */
uint32_t tp_pages_free(const tp_engine* eng);

/* ------------------------------------------------------------------ budget */

/* Changes the device-memory cap; a lower cap applies to later reservations. */
tp_status tp_set_device_budget(tp_engine* eng, uint64_t bytes);
/* Bytes currently reserved and the cap. Either pointer may be NULL. */
tp_status tp_budget_query(tp_engine* eng, uint64_t* reserved, uint64_t* cap);

/* ------------------------------------------------------- transfer options */

/*
 * How batches in host pages reach the device, for the executions that start
 * after the call (call it while none runs).  prefetch_depth: batches copied
 * ahead of the kernels on the copy stream (Section 3.3.3, pre-loading); 0
 * copies each batch and then runs it, on one stream.  flags:
 * TP_COPY_PINNED_PER_BATCH copies every batch first into a page-locked buffer
 * allocated for it (cudaHostAlloc) and freed once its copies are done, as an
 * engine without a pinned page pool would (Section 3.4: pinning memory is
 * slow, which is why the pool is allocated once); results are unchanged.
 * TP_E_INVALID for a negative depth or unknown flags.
 */
enum { TP_COPY_PINNED_PER_BATCH = 1 };
tp_status tp_set_copy_options(tp_engine* eng, int32_t prefetch_depth, uint32_t flags);

/* ------------------------------------------------------------------ tables */

enum { TP_I32 = 0, TP_I64 = 1, TP_U8 = 2 };
enum { TP_HOST_PAGES = 1, TP_DEVICE = 2 };

typedef struct {
    const char* name;     /* copied; may be NULL */
    int32_t type;         /* TP_I32, TP_I64 or TP_U8 */
    int32_t scale;        /* decimal scale (digits after the point); metadata only */
} tp_column_desc;

typedef struct {
    int32_t n_cols;                 /* 1..32 */
    const tp_column_desc* cols;     /* n_cols entries */
    uint64_t batch_rows;            /* rows per batch; 0 = engine default */
} tp_table_desc;

/* Creates an empty table whose rows will live in pool pages. */
tp_status tp_table_create(tp_engine* eng, const tp_table_desc* desc, tp_table** out);

/* Copies nrows rows from host arrays cols[0..n_cols) (one contiguous array
 * per column, element type as declared) into pool pages.  Rows are cut into
 * batches of batch_rows; within a batch the columns lie back to back across
 * as many pages as they need, so one column may span pages, and the tail of
 * the batch's last page stays unused (Section 3.4).  Unless the engine has
 * TP_FLAG_RAW_PAGES, each integer column of a batch is stored as (value -
 * the batch's minimum) in the fewest bits that hold the batch's range:
 * bit-packed, value i at bit i * bits of a little-endian 32-bit word stream,
 * or as plain 1-, 2- or 4-byte integers when that is 8, 16 or 32 bits.  The
 * caller keeps its arrays.  Errors: TP_E_POOL_EMPTY (pool exhausted: the
 * append is undone), TP_E_INVALID (table already on the device). */
tp_status tp_table_append(tp_table* t, const void* const* cols, uint64_t nrows);

/* Moves the table: TP_DEVICE copies every column into one contiguous device
 * array (reserving its bytes in the budget) and returns the pages;
 * TP_HOST_PAGES is a no-op for a paged table.  Errors: TP_E_BUDGET,
 * TP_E_CUDA, TP_E_INVALID. */
tp_status tp_table_place(tp_table* t, int32_t placement);

/* Registers caller-owned device columns without copying (for example tensors
 * held by PyTorch).  dev_cols[i] must hold nrows elements, be 16-byte aligned
 * and outlive the table.  Not counted against the budget. */
tp_status tp_table_wrap_device(tp_engine* eng, const tp_table_desc* desc,
                               const void* const* dev_cols, uint64_t nrows, tp_table** out);

uint64_t tp_table_rows(const tp_table* t);
/* Number of batches (paged tables) or 1 (device tables). */
uint64_t tp_table_batches(const tp_table* t);
/* Frees the table's pages or device memory (not wrapped caller memory). */
void tp_table_destroy(tp_table* t);

/* ------------------------------------------------------------------- plans */

/* Group field sides: the fact table, the first dimension (TP_SIDE_DIM), or
 * further dimension j of a star join (TP_SIDE_DIM + 1 + j). */
enum { TP_SIDE_FACT = 0, TP_SIDE_DIM = 1 };
#define TP_MAX_EXTRA_DIMS 3
enum { TP_AGG_SUM = 0, TP_AGG_SUM_MUL_SUB = 1, TP_AGG_COUNT = 2, TP_AGG_AVG = 3 };

typedef struct {
    int32_t col;          /* column (fact, or dimension for dim_filter), -1 = no filter */
    int64_t lo, hi;       /* keep rows with lo <= value <= hi (inclusive) */
} tp_filter;

enum { TP_LIP_AUTO = 0, TP_LIP_OFF = 1, TP_LIP_ON = 2 };

typedef struct {
    int32_t fact_col;     /* fact foreign-key column, -1 = no join */
    int32_t dim_col;      /* dimension key column; keys must be unique */
} tp_join;

typedef struct {
    int32_t side;         /* TP_SIDE_FACT or TP_SIDE_DIM */
    int32_t col;
    int32_t bits;         /* 1..64; the value must lie in [0, 2^bits) unless bits == 64 */
} tp_group_field;

typedef struct {
    int32_t kind;         /* TP_AGG_* */
    int32_t col_a;        /* fact column summed (SUM, AVG) or factor a (SUM_MUL_SUB) */
    int32_t col_b;        /* fact column b of SUM_MUL_SUB */
    int64_t k;            /* constant K of SUM_MUL_SUB: SUM(a * (K - b)) */
} tp_agg;

/*
 * A query over one fact table and an optional dimension table.  The group key
 * packs the fields first-field-highest into at most 64 bits; dimension-side
 * fields may use at most 32 bits in total.  Aggregates read fact columns.
 */
typedef struct {
    tp_table* fact;
    tp_table* dim;                  /* NULL when join.fact_col < 0 */
    tp_filter filter;
    tp_join join;
    int32_t n_group;                /* 0..4 (0: one group, key 0) */
    tp_group_field group[4];
    int32_t n_agg;                  /* 1..8 */
    tp_agg aggs[8];
    int32_t agg_strategy;           /* TP_AGG_*; AUTO = engine choice */
    float load_factor;              /* 0 = engine default */
    uint64_t expected_groups;       /* sizing hint for TP_AGG_GLOBAL; 0 = estimate */
    /* Join partitions P (Section 3.3.2: spill what does not fit).  0 = auto:
     * a hashed join whose table would take more than half of the free budget
     * runs as a hybrid hash join with 64 partitions; 1 = never partition;
     * 2..64 (a power of two) = always partition into P.  A partitioned join
     * reserves the free budget that streaming buffers, the aggregation table
     * and the result leave.  Every partition stays resident when one table
     * of all build rows fits it; otherwise room for the largest partition's
     * table is kept and partitions are made resident in order while the
     * rest fits.  The other partitions' build and fact rows are spilled to
     * pool pages and joined one partition at a time (TP_E_POOL_EMPTY when
     * the pool cannot hold them). */
    int32_t join_partitions;
    /* Dimension predicate, applied when dim_filter_on != 0 (a zeroed
     * descriptor has none): only dimension rows with lo <= value <= hi of
     * dimension column dim_filter.col take part in the join, and only their
     * keys must be unique. */
    tp_filter dim_filter;
    int32_t dim_filter_on;
    /* Lookahead information passing (Section 5): a blocked Bloom filter of
     * the keys the dimension predicate admits, built with the join table and
     * tested on each fact row's key before its probe, and before a
     * partitioned join spills the row.  TP_LIP_AUTO: with a dimension
     * predicate, when the join table would not stay in L2 (64 MB or more) or the
     * join is partitioned; TP_LIP_ON: whenever there is a dimension predicate;
     * TP_LIP_OFF: never.  Join tables shared through the server's cache and
     * batched executions run without it.  Results never depend on it. */
    int32_t lip;
    /* Star join: further dimension tables, each joined like the first
     * (Section 3.2: a PK-FK inner equi-join) on its own fact foreign key,
     * extra_join[j].fact_col = key column extra_join[j].dim_col of
     * extra_dim[j]; a fact row survives only with a partner in every
     * dimension.  Group fields of extra_dim[j] use side TP_SIDE_DIM + 1 + j;
     * the fields of each dimension take at most 31 bits.  extra_dim_filter[j]
     * applies when extra_dim_filter_on[j] != 0, with a lookahead filter of its
     * own under the rule above.  Needs the first join.  Only the first join
     * is ever partitioned: the further tables stay resident (TP_E_BUDGET when
     * they do not fit).  Batched executions and the allocation-free entry
     * point take one dimension (TP_E_INVALID otherwise).  The tables belong
     * to the caller's engine and must outlive the plan, like fact and dim. */
    int32_t n_extra_dims;                         /* 0..TP_MAX_EXTRA_DIMS */
    tp_table* extra_dim[TP_MAX_EXTRA_DIMS];
    tp_join extra_join[TP_MAX_EXTRA_DIMS];
    tp_filter extra_dim_filter[TP_MAX_EXTRA_DIMS];
    int32_t extra_dim_filter_on[TP_MAX_EXTRA_DIMS];
    /* Fan-out: the first join's build keys may repeat.  A fact row then pairs
     * with every admitted dimension row holding its key (an inner join
     * without the key constraint) and every pair counts once in its group.
     * The build sorts the admitted rows by key and indexes the first row of
     * each key.  Never partitioned (join_partitions must be 0 or 1;
     * TP_E_BUDGET when the table does not fit), not cached by the server;
     * batched executions and the allocation-free entry point refuse it.  At
     * most 2^31 admitted build rows (TP_E_INVALID at execution). */
    int32_t join_many;
} tp_plan_desc;

/* Validates and stores a plan.  TP_E_INVALID on any inconsistency. */
tp_status tp_plan_create(tp_engine* eng, const tp_plan_desc* desc, tp_plan** out);
void tp_plan_destroy(tp_plan* p);

/* ----------------------------------------------------------------- execute */

/*
 * Runs the plan and waits for it:
 *   1. reserve device memory for hash tables, accumulators and staging
 *      (TP_E_BUDGET if the estimate exceeds the cap);
 *   2. build the dimension hash table (TP_E_DUP_KEY on a repeated key);
 *   3. for each fact batch: filter, probe and aggregate in one kernel; a
 *      paged fact table streams through device staging slots, copied ahead on
 *      the copy stream while the previous batch computes;
 *   4. merge, compute AVG, compact and sort the groups by key.
 * *out receives a result that stays on the device until read.
 */
tp_status tp_execute(tp_plan* p, tp_result** out);

/* --------------------------------------------------------- batched execution */

/*
 * Many uneven queries in one persistent kernel launch, captured once in a CUDA
 * graph and replayed by every tp_batch_execute.  Section 3.1 has operators
 * spawn tasks over batches and Section 3.3.1 has the Compute Executor run
 * them asynchronously; here the tasks of all queries -- hash-build chunks,
 * probe tiles, finalisation -- form one work queue that resident CTAs drain in
 * order.  A probe tile of query q waits (bounded, TP_E_TIMEOUT on expiry)
 * until every build chunk of q is done, and q's finalisation until every
 * probe tile of q is done; tasks are taken in queue order, so every task
 * waited on is already held by a running CTA.
 *
 * Every fact and dimension table must be on the device (TP_DEVICE or
 * wrapped) and every group key at most 20 bits wide (the groups of a query
 * live in a dense device table of 2^bits entries); otherwise TP_E_INVALID.
 * The batch reserves and owns all device memory it needs (join tables,
 * accumulators, results); TP_E_BUDGET if that does not fit.
 *
 *   tuning_path  optional table written by tp_autotune: per query class
 *                (fact-size, group-width and dimension-size buckets) the
 *                join load factor, rows per warp of a probe tile, and
 *                shared-memory versus device-memory aggregation.  NULL or a
 *                missing file: built-in defaults.
 */
typedef struct tp_batch tp_batch;
tp_status tp_batch_create(tp_engine* eng, tp_plan* const* plans, int32_t n, const char* tuning_path,
                          tp_batch** out);
/* Replays the batch and fills results[0..n) (ownership as tp_execute's, but
 * the arrays live in the batch: a result stays valid until the next
 * tp_batch_execute or tp_batch_destroy of its batch). */
tp_status tp_batch_execute(tp_batch* b, tp_result** results);
/* Device time of the last tp_batch_execute in milliseconds (CUDA events). */
double tp_batch_last_ms(const tp_batch* b);
void tp_batch_destroy(tp_batch* b);
/* Fault injection for tests of the bounded device waits: from the next
 * tp_batch_execute on, every dependency wait of the batch's persistent kernel
 * gives up after wait_ns (instead of 2 s) and the finalisation of query
 * `query` waits for one probe tile more than exists, so that wait runs out:
 * tp_batch_execute returns TP_E_TIMEOUT with the device context intact.
 * query = -1 restores the batch (2 s limit, true tile counts).  The paper
 * has no counterpart (its tasks wait on the host). */
tp_status tp_debug_batch_stall(tp_batch* b, int32_t query, uint64_t wait_ns);

/*
 * Autotuner: for every query class present in plans[0..n) (buckets of fact
 * rows, group-key bits and dimension rows), tries the rows per warp of a
 * probe tile (128, 256, 512, 1024), shared-memory versus device-memory
 * aggregation and the join load factor (0.5, 0.7), one knob at a time.  Each
 * candidate value is applied to every class in one batched launch of all n
 * plans; the launch records, per query, the CTA time its tasks took, and a
 * class keeps the value when its queries' time fell by 2% or more (best of
 * three runs).  Writes the choice per class to tuning_path (text), which
 * tp_batch_create reads.  The plans' own results are unaffected.
 */
tp_status tp_autotune(tp_engine* eng, tp_plan* const* plans, int32_t n, const char* tuning_path);

/* ------------------------------------------------------------------ serving */

/*
 * A request server over one engine: queries are submitted as they arrive
 * (Section 3.3.1: executors take tasks from a queue; Section 3.3.2: a task is
 * admitted by its device-memory reservation).
 *
 * With TP_SERVE_BATCH (continuous batching), a dispatcher thread takes every
 * queued request a batched launch can run (the conditions of tp_batch_create:
 * device-resident tables, at most one join, no fan-out, at most 20 key bits),
 * up to max_inflight of them (0 = 256) and as many as the budget admits, and
 * starts them as one persistent queue launch; requests arriving meanwhile
 * form the next launch, which starts at once on a second stream and overlaps
 * the running one on the device.  Each request has its own join table,
 * accumulators, error word and result: its result and its status are the
 * ones it gets alone.  A lone request on an idle GPU runs at once as a single
 * query instead of waiting for company.  The probe tasks are compiled at run
 * time for every plan shape the server has seen; the first batched launch
 * after a new shape arrives waits for that compilation.
 *
 * Other requests (and every request without TP_SERVE_BATCH) run on `workers`
 * lanes, each a host thread with its own compute and copy streams, so their
 * kernels overlap on the device (each Compute Executor thread drives its own
 * CUDA stream).  At most max_inflight run on lanes at once (0 = workers);
 * requests of the same plan object run one at a time there.
 *
 * Admission: a request whose reservation does not fit waits in the queue
 * while others run and is admitted as soon as completions release memory; it
 * fails with TP_E_BUDGET only when it cannot fit even with nothing else
 * running.  Plans must outlive their requests.
 *
 * With TP_SERVE_CACHE_DIM the join table of a dimension stays on the device
 * across lane requests, keyed by dimension table, key column, dimension group
 * fields and load factor; cached tables hold their reservation until evicted
 * (least recently used, when a reservation does not fit) or the server stops.
 * Hashed joins that would be partitioned bypass the cache.  Batched requests
 * build their join tables inside their launch.
 */
enum { TP_SERVE_CACHE_DIM = 1, TP_SERVE_BATCH = 2 };
typedef struct tp_server tp_server;
typedef uint64_t tp_ticket;

tp_status tp_server_start(tp_engine* eng, int32_t workers, int32_t max_inflight, uint32_t flags,
                          tp_server** out);
/* Queues one execution of p; returns at once with a ticket. */
tp_status tp_submit(tp_server* srv, tp_plan* p, tp_ticket* out);
/*
 * Waits up to timeout_ns (< 0: forever) for a ticket.  TP_E_TIMEOUT if it is
 * still queued or running (the ticket stays valid); otherwise the request's
 * own status, with *out its result on TP_OK.  times (may be NULL) receives
 * three steady-clock nanosecond stamps: submitted, started, finished.  A
 * finished ticket is consumed by the call.  One thread at a time may wait on
 * a ticket: a second concurrent tp_wait on it returns TP_E_INVALID.
 */
tp_status tp_wait(tp_server* srv, tp_ticket t, int64_t timeout_ns, tp_result** out, int64_t* times);
typedef struct {
    uint64_t submitted, completed, failed;
    uint64_t budget_waits;        /* admissions deferred because the reservation did not fit */
    uint64_t cache_hits, cache_misses, cache_evictions;
    uint32_t inflight_peak;       /* most requests running at once (lanes and batched launches) */
    uint32_t batches;             /* batched launches started (TP_SERVE_BATCH) */
} tp_server_stats;
tp_status tp_server_stats_get(tp_server* srv, tp_server_stats* out);
/* Finishes queued and running requests, frees cached tables and lanes. */
void tp_server_stop(tp_server* srv);

/* ----------------------------------------------------------------- results */

typedef struct {
    uint64_t lo;          /* low 64 bits */
    int64_t hi;           /* high 64 bits (two's complement) */
} tp_i128;

uint64_t tp_result_groups(const tp_result* r);
/* Host arrays of tp_result_groups() entries, ascending by key; copied from
 * the device on first use and owned by the result.  NULL on error or when
 * the aggregate has no such output. */
const uint64_t* tp_result_keys(tp_result* r);
const int64_t* tp_result_count(tp_result* r);
/* Exact sum of aggregate `agg` (SUM, SUM_MUL_SUB or AVG). */
const tp_i128* tp_result_sum(tp_result* r, int32_t agg);
/* AVG of aggregate `agg` (AVG only). */
const double* tp_result_avg(tp_result* r, int32_t agg);
/* Device addresses of the same arrays (no copy); NULL where absent. */
const void* tp_result_device_keys(const tp_result* r);
const void* tp_result_device_count(const tp_result* r);
const void* tp_result_device_sum(const tp_result* r, int32_t agg);
const void* tp_result_device_avg(const tp_result* r, int32_t agg);
void tp_result_free(tp_result* r);

/* ------------------------------------------------------------- diagnostics */

typedef struct {
    uint64_t h2d_bytes;          /* bytes copied host -> device */
    uint64_t d2h_bytes;          /* bytes copied device -> host */
    uint64_t batches;            /* fact batches processed */
    uint64_t kernel_launches;    /* kernels launched by the library */
    uint64_t peak_reserved;      /* highest reservation seen */
    uint64_t retries;            /* executions repeated with a larger table */
    uint32_t pages_in_use;
    uint32_t pages_total;
    double agg_kernel_ms;        /* device time of fused aggregate kernels (TP_FLAG_TIME_KERNELS) */
    uint64_t agg_kernel_launches;
    uint64_t agg_kernel_rows;    /* fact rows those launches processed */
    uint64_t jit_compiles;       /* plan shapes compiled at run time by this engine */
    uint64_t jit_failures;       /* shapes whose compilation failed (ahead-of-time kernel used) */
    uint64_t jit_launches;       /* launches of run-time compiled kernels */
    double jit_compile_ms;       /* host time spent compiling */
    uint64_t agg_split_passes;   /* extra passes of aggregations split by key range to fit the budget */
    uint64_t lip_filters;        /* lookahead filters built */
    /* host wall time of the partitioned joins' phases: build side (histogram,
     * resident inserts, build spill), fact stream (probe and spill), joins of
     * the spilled partitions */
    double part_build_ms, part_stream_ms, part_spilled_ms;
} tp_stats;

/* Message for the last error on this thread ("" if none). */
const char* tp_last_error(void);
tp_status tp_stats_get(tp_engine* eng, tp_stats* out);
/* Fault injection for tests: the next n host page allocations and device
 * reservations fail as if exhausted. */
tp_status tp_debug_fail_next_alloc(tp_engine* eng, int32_t n);
/* The page encoding of a bit-packed column, for tests (host only, no GPU):
 * packs values[0..n) (each below 2^bits, 1 <= bits <= 31) into
 * words[0..ceil(n * bits / 32)), value i at bits [i * bits, (i + 1) * bits)
 * of the stream, least significant bit first, stream bit j being bit (j % 32)
 * of words[j / 32].  The same function writes tp_table_append's pages.
 * Errors: TP_E_INVALID (NULL pointers with n > 0, bits out of range, or a
 * value that does not fit). */
tp_status tp_debug_pack_bits(const uint64_t* values, uint64_t n, int32_t bits, uint32_t* words);

/* ------------------------------------------------------ allocation-free call */

/*
 * tp_execute_noalloc -- the paper has no counterpart to this call; it exists
 * for callers that cannot allocate device memory while they run a query:
 * applications that have given all GPU memory to their own allocator (a
 * database buffer pool, PyTorch's caching allocator) and forbid side
 * allocations, or latency-bound code that cannot afford a cudaMalloc or
 * cudaFree, which may synchronise the device or fail under fragmentation.
 *
 * It runs the same filter -> join -> low-cardinality group-by as tp_execute,
 * on caller-owned device columns and into caller-owned device outputs, and
 * allocates nothing: no engine, no cudaMalloc/cudaFree, no host heap (the
 * driver places the array and the kernels at the first call; see below).  Its
 * scratch (join hash table, per-group accumulators, status words) is one
 * fixed device array of 8,945,920 bytes inside this library, which every GPU
 * that loads the library holds until the process exits.
 *
 *   d            query; d->fact and d->dim are ignored, column indices refer
 *                to fact_cols / dim_cols.  join.fact_col < 0 means no join.
 *   fact_cols    n_fact_cols device pointers (16-byte aligned), n_fact rows,
 *                types TP_I32 / TP_I64 / TP_U8 in fact_types (host array).
 *   dim_cols     n_dim_cols device pointers, n_dim rows (join only).
 *   keys, counts device arrays of 2^(total group bits) entries (the most
 *                groups there can be); groups are written ascending by key.
 *   sums[a]      device tp_i128 array of the same length for every SUM,
 *                SUM_MUL_SUB and AVG aggregate a (other entries ignored).
 *   avgs[a]      device double array for every AVG aggregate a.
 *   n_groups     host; receives the number of groups written.
 *   stream       cudaStream_t (as void*) of the current device; the call
 *                synchronises it before returning.
 *
 * Limits (TP_E_INVALID with a message beyond them): a group key of at most
 * 12 bits; a join table of at most 2^20 slots for 32-bit keys (2^19 for
 * 64-bit keys), i.e. at most ceil(0.5 * 2^20) = 524,288 dimension rows at the
 * default load factor 0.5.  Other errors as tp_execute (TP_E_DUP_KEY,
 * TP_E_RANGE, TP_E_CUDA).
 *
 * The first call on a device sets it up, with that device current: it looks
 * up the scratch array's device address and loads the kernels the call uses,
 * which is when the CUDA driver places the array and the kernel code in
 * device memory.  Make that first call at start-up -- before handing the rest
 * of device memory to another allocator, and before any stream capture;
 * later calls allocate no device memory.  Every call reuses the array and
 * clears what must start at zero; calls whose GPU work overlaps (other
 * streams or host threads) race on it, so the caller must serialise them.
 */
tp_status tp_execute_noalloc(const tp_plan_desc* d, const void* const* fact_cols, const int32_t* fact_types,
                             int32_t n_fact_cols, uint64_t n_fact, const void* const* dim_cols,
                             const int32_t* dim_types, int32_t n_dim_cols, uint64_t n_dim, uint64_t* keys,
                             int64_t* counts, tp_i128* const* sums, double* const* avgs, uint64_t* n_groups,
                             void* stream);

#ifdef __cplusplus
}
#endif
#endif
