// Device-side parameter blocks and launchers of the relational hot path.
//
// Hash tables use open addressing with linear probing.  The slot of a key is
// hash(key) & mask, where hash is the 64-bit finaliser of MurmurHash3
// (Appleby, public domain) for 64-bit keys and its 32-bit finaliser for join
// tables with 32-bit keys.
#pragma once
#ifdef __CUDACC_RTC__
// run-time compilation (NVRTC) of the device code: no host headers
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef long long int64_t;
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
typedef unsigned long long uintptr_t;
#define INT32_MIN (-2147483647 - 1)
#define INT32_MAX 2147483647
#define INT64_MIN (-9223372036854775807LL - 1)
#define INT64_MAX 9223372036854775807LL
#else
#include <cuda_runtime.h>
#include <stdint.h>
#endif

namespace tpk {

enum : int32_t { T_I32 = 0, T_I64 = 1, T_U8 = 2 };
enum : int32_t { S_SUM = 0, S_MUL_SUB = 1 };

// error bits written by kernels into the per-execution error word
enum : uint32_t {
    ERR_RANGE = 1u,      // group field outside [0, 2^bits)
    ERR_DUP = 2u,        // duplicate build key
    ERR_OVERFLOW = 4u,   // aggregation table full: execution must be retried larger
    ERR_INTERNAL = 8u,   // probe ran past the table size (cannot happen below full load)
    ERR_TIMEOUT = 16u,   // a bounded device wait expired
};

constexpr uint64_t EMPTY64 = ~0ull;
constexpr uint32_t PAYLOAD_BAD = 0x80000000u;   // join payload: a dim field is out of range
constexpr int MAX_DIM_BITS = 31;                // dimension group fields share 31 payload bits
constexpr uint32_t EMPTY32 = ~0u;
constexpr int MAX_GROUP = 4;
constexpr int MAX_SUM = 8;
constexpr int MAX_XJOIN = 3;                    // further joins of a star query

struct DevCol {
    const void* ptr;
    int32_t type;
    int32_t pad;
};

// Join table.
//   Hash: 32-bit keys: one 64-bit word per slot, payload << 32 | key, EMPTY =
//   all ones.  64-bit keys: two words per slot {key, payload}, EMPTY key = all
//   ones.  A key equal to the EMPTY pattern lives in side[]: side[0] = 1 when
//   present, side[1] = its payload.
//   Direct (dense keys: the key range is at most twice the row count): one
//   32-bit payload word per key in [kmin, kmin + range), at slot key - kmin;
//   EMPTY32 = absent (an out-of-range payload is stored as exactly
//   PAYLOAD_BAD, so no present payload equals EMPTY32).
struct JoinTable {
    uint64_t* slots;
    uint64_t mask;          // hash: capacity - 1 (capacity a power of two)
    uint32_t* side;         // hash: 2 words
    int32_t key64;
    int32_t direct;         // 1: direct-mapped table
    int64_t kmin;           // direct: smallest key
    uint64_t range;         // direct: number of slots
    // partitioned join (part_shift != 0): a row joins only when bit
    // (fmix64(key) >> part_shift) of part_mask is set; part_shift == 0 (the
    // zero-initialised default) means no partition filter
    uint64_t part_mask;
    int32_t part_shift;
    int32_t pad2;
    // lookahead filter (lip != nullptr): a blocked Bloom filter of the
    // admitted build keys, 8 words per block; a key's block is
    // fmix64(key) >> lip_shift
    uint32_t* lip;
    int32_t lip_shift;
    int32_t pad3;
    // fan-out (many != 0, repeated build keys): the table maps a key to the
    // index of its first row in mkeys/mpay, the admitted build rows sorted by
    // key; a fact row pairs with rows first, first + 1, ... while mkeys
    // holds its key
    const uint64_t* mkeys;
    const uint32_t* mpay;
    uint64_t mn;
    int32_t many;
    int32_t pad4;
};

// The query as the per-batch kernels see it.  Column pointers address the
// current batch (row 0 = first row of the batch).
struct QueryDev {
    DevCol fcol;            // filter column
    int64_t flo, fhi;
    int32_t has_filter;
    int32_t has_join;
    DevCol fk;              // fact foreign key
    JoinTable jt;
    int32_t n_group;
    int32_t n_sum;
    int32_t eager;          // 1: load every column of a tile up front; 0: load past the
                            // filter only for rows that pass (selective filters)
    int32_t pad;
    DevCol gcol[MAX_GROUP]; // fact-side group columns (unused for dim fields)
    int32_t gside[MAX_GROUP];
    int32_t gbits[MAX_GROUP];
    int32_t gdpos[MAX_GROUP];   // bit offset of a dim field inside the join payload
    int32_t skind[MAX_SUM];
    DevCol sa[MAX_SUM];
    DevCol sb[MAX_SUM];
    int64_t sk[MAX_SUM];
    uint32_t* err;
    // star join: further joins, each on its own fact key column; a row must
    // find a partner in every table.  gdim[g]: the join whose payload holds
    // dimension field g (0 = jt, 1 + j = jtx[j])
    int32_t n_xjoin;
    int32_t gdim[MAX_GROUP];
    int32_t pad_x;
    DevCol fkx[MAX_XJOIN];
    JoinTable jtx[MAX_XJOIN];
};

// Build-side parameters: key column, dim group fields packed into the payload.
struct BuildDev {
    DevCol key;
    int32_t n_dfield;
    int32_t pad;
    DevCol dcol[MAX_GROUP];
    int32_t dbits[MAX_GROUP];
    int32_t dpos[MAX_GROUP];
    JoinTable jt;
    uint32_t* err;
    DevCol fcol;            // dimension predicate: rows outside [flo, fhi] do not join
    int64_t flo, fhi;
    int32_t has_filter;
    int32_t pad2;
};

// Global aggregation table: slot = {key, count, (lo, hi) per sum}, EMPTY key =
// all ones; the all-ones key itself is kept in a dedicated side slot placed
// after the last regular slot.
//   Direct (dense key range, direct != 0): the slot of key k is k - kmin,
//   mask + 1 slots cover every key the column bounds allow; the key word is
//   unused (zero) and a slot is occupied when its count is non-zero.
struct AggTable {
    uint64_t* slots;
    uint64_t mask;
    uint32_t words;          // 64-bit words per slot = 2 + 2 * n_sum
    int32_t direct;
    unsigned long long* used;   // occupied slots counter (hashed)
    uint64_t max_used;          // beyond this, new keys set ERR_OVERFLOW (hashed)
    uint64_t kmin;              // direct: smallest key
    // key-range pass of a split aggregation (split != 0): keys outside
    // [key_lo, key_hi] are skipped, another pass takes them
    uint64_t key_lo, key_hi;
    int32_t split;
    int32_t pad2;
};

// Output arrays of one result (device memory).
struct OutDev {
    uint64_t* keys;
    int64_t* counts;
    uint64_t* sums[MAX_SUM];    // (lo, hi) pairs
    double* avgs[MAX_SUM];      // per sum slot, only where avg_of_sum set
    int32_t has_avg[MAX_SUM];
    unsigned long long* n_groups;
};

// --------------------------------------------------------- staged pipeline
//
// A staged launch runs one producer warp that copies whole tiles of every
// column the query reads into a ring of shared-memory stages with 1-D bulk
// copies (cp.async.bulk, completion on an mbarrier), and ST_CONSUMERS warps
// that evaluate the rows from shared memory, 8 rows per lane.

#ifndef TP_ST_CONSUMERS
#define TP_ST_CONSUMERS 16     // consumer warps per CTA
#endif
#ifndef TP_ST_RPL
#define TP_ST_RPL 2            // rows per lane per stage
#endif
#ifndef TP_ST_CTAS
#define TP_ST_CTAS 2           // resident CTAs per SM (shared memory is split between them)
#endif
constexpr int ST_CONSUMERS = TP_ST_CONSUMERS;
constexpr int ST_RPL = TP_ST_RPL;
constexpr int ST_CTAS = TP_ST_CTAS;
constexpr int ST_SUB = 32 * ST_RPL;                // rows per consumer warp per stage
constexpr int ST_TILE = ST_CONSUMERS * ST_SUB;     // rows per stage
constexpr int ST_THREADS = 32 * (1 + ST_CONSUMERS);
constexpr int ST_MAX_COLS = 22;
constexpr int ST_MAX_STAGES = 8;

// Geometry of a staged kernel: consumer warps per CTA, rows per lane per
// stage, resident CTAs per SM its shared memory is split for.
struct StageGeom {
    int32_t consumers;
    int32_t rpl;
    int32_t ctas;
};
// The ahead-of-time staged kernels.
constexpr StageGeom AOT_GEOM{ST_CONSUMERS, ST_RPL, ST_CTAS};
// The run-time compiled dense kernel: one CTA of 24 consumer warps per SM
// and a ring of exactly JIT_DENSE_STAGES stages.  Measured on the star
// query: the shared memory the ring leaves becomes L1 cache, which holds the
// hot part of the join table (more stages were slower, fewer starved the
// copies).
constexpr StageGeom JIT_DENSE_GEOM{24, 2, 1};
constexpr int JIT_DENSE_STAGES = 3;
// column slots of a QueryDev: filter, fk, 4 group columns, 8 + 8 sum columns
enum : int { SL_FILTER = 0, SL_FK = 1, SL_GROUP = 2, SL_SA = 6, SL_SB = 14, SL_FKX = 22, SL_COUNT = 25 };

struct StageLayout {
    const void* src[ST_MAX_COLS];      // global base of each staged column
    uint32_t off[ST_MAX_COLS];         // byte offset of its tile inside a stage
    int32_t esize[ST_MAX_COLS];
    int8_t col_of_slot[SL_COUNT];      // staged column feeding each slot, -1 if none
    int16_t pad;
    int32_t n_cols;
    uint32_t stage_bytes;              // bytes between consecutive stages
    uint32_t tile_bytes;               // bytes one full tile brings in (expect_tx)
    int32_t n_stages;
    int32_t tile;                      // rows per stage (consumer warps * 32 * rows per lane)
    int32_t threads;                   // threads per CTA (a producer warp + the consumer warps)
    int32_t ctas;                      // resident CTAs per SM the shared memory was split for
    uint32_t table_bytes;              // shared-memory aggregation table in front of the stages
    uint32_t smem_bytes;               // total dynamic shared memory
    uint64_t wait_ns;                  // limit of every mbarrier wait
    // narrow (32-bit) shared-memory table, used with 64-bit accumulation:
    // count[G] in word 0, then per sum its low words and, for mode 2, a carry
    // word block.  Terms are offset by sum_off so they are non-negative.
    int8_t sum_mode[MAX_SUM];          // 1: low word only, 2: low word + carry word
    uint32_t sum_word[MAX_SUM];        // index (in blocks of G words) of sum s's low words
    int64_t sum_off[MAX_SUM];
};

// Proven range of one aggregate's per-row term, from column statistics.
struct TermBounds {
    int64_t lo;      // minimum term
    uint64_t span;   // maximum term - minimum term
};

// --------------------------------------------------------- batched execution

enum : uint32_t { BI_BUILD = 0, BI_PROBE = 1, BI_FINAL = 2 };

// One task of the batch queue.
struct BatchItem {
    uint32_t q;        // query index
    uint32_t kind;     // BI_*
    uint64_t r0, r1;   // row range (build: dimension rows, probe: fact rows, final: groups)
    uint64_t pad;
};

// Groups one finalisation task of a batched query writes: a query's non-empty
// groups are emitted by ceil(2^key_bits / FINAL_CHUNK) tasks, range k after
// range k - 1 has published where its rows end.
constexpr uint32_t FINAL_CHUNK = 8192;

// One query of a batch, as the persistent kernel sees it.
struct BatchQuery {
    QueryDev q;                 // columns, filter, join table, groups, sums; err = batch error word
    BuildDev b;                 // build side, same join table
    uint64_t* acc;              // dense table of 2^key_bits groups: count, then lo/hi per sum
    OutDev out;
    uint32_t key_bits;
    int32_t smem;               // aggregate a probe tile in shared memory first (needs fast)
    int32_t fast;               // 64-bit accumulation proved safe: low words only
    uint32_t build_items;
    uint32_t probe_items;
    int32_t shape;              // shape id of the run-time compiled probe task
    int8_t sum_mode[MAX_SUM];   // shared-memory table: 1 low word, 2 low + carry word
    int64_t sum_off[MAX_SUM];   // term offsets making terms non-negative
    unsigned long long* task_ns;   // when set: nanoseconds of CTA time this query's tasks took
    unsigned* final_done;          // finalisation ranges that published their end (zeroed per run)
    unsigned long long* final_end; // output rows written by the published ranges
};

constexpr int BATCH_THREADS = 512;

#ifndef __CUDACC_RTC__
// Runs the whole queue: n_items tasks, ctr[0] the next task index,
// done[q] build chunks finished, done[n_q + q] probe tiles finished.
cudaError_t launch_batch(const BatchQuery* qs, const BatchItem* items, uint32_t n_items, uint32_t n_q,
                         unsigned* ctr, uint32_t* err, const uint64_t* wait_ns, uint32_t smem_bytes, int grid,
                         cudaStream_t st);
int batch_grid(uint32_t smem_bytes, int num_sms);
#endif

#ifndef __CUDACC_RTC__
// The same query over the rows from `row` on: every fact column pointer
// advanced by `row` elements.
inline QueryDev offset_rows(const QueryDev& q, uint64_t row) {
    QueryDev r = q;
    auto adv = [row](DevCol& c) {
        if (!c.ptr) return;
        const uint64_t sz = c.type == T_I64 ? 8 : (c.type == T_I32 ? 4 : 1);
        c.ptr = (const unsigned char*)c.ptr + row * sz;
    };
    adv(r.fcol);
    adv(r.fk);
    for (int j = 0; j < MAX_XJOIN; ++j) adv(r.fkx[j]);
    for (int g = 0; g < MAX_GROUP; ++g) adv(r.gcol[g]);
    for (int s = 0; s < MAX_SUM; ++s) {
        adv(r.sa[s]);
        adv(r.sb[s]);
    }
    return r;
}

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return cudaGetLastError().

// Raises (never lowers) a kernel's dynamic shared-memory limit to `bytes`.
// The attribute is process-wide, so lowering it could fail a concurrent
// launch of the same kernel on another stream that needs more.
cudaError_t ensure_smem_limit(const void* fn, int bytes);

cudaError_t launch_fill_u64(uint64_t* p, uint64_t n, uint64_t v, cudaStream_t st);
// aggregation table slots: key word = EMPTY64, every other word 0
cudaError_t launch_init_agg(uint64_t* slots, uint64_t n_slots, uint32_t words, cudaStream_t st);
cudaError_t launch_build(const BuildDev& b, uint64_t n, int num_sms, cudaStream_t st);
cudaError_t launch_agg_shared(const QueryDev& q, uint64_t n, uint64_t* gacc, uint32_t key_bits,
                              int grid, cudaStream_t st);
size_t agg_shared_smem_bytes(uint32_t key_bits, int n_sum);
int agg_shared_grid(uint32_t key_bits, int n_sum, int num_sms);
cudaError_t launch_agg_global(const QueryDev& q, uint64_t n, const AggTable& t, int num_sms,
                              cudaStream_t st);
// lo_only: the table's sums were accumulated as 64-bit values (overflow ruled
// out by column bounds); their high words are the sign extension of the low.
cudaError_t launch_final_dense(const uint64_t* gacc, uint32_t key_bits, int n_sum, const OutDev& o,
                               cudaStream_t st, bool lo_only = false);
// Loads the build, plain shared-memory aggregation and dense finalisation
// kernels on the current device now (with lazy module loading the first
// launch would load them, placing their code in device memory then).
cudaError_t load_plain_kernels();

// Staged shared-memory aggregation.  staged_layout_shared() fills *L for the
// query (false when the staged kernel cannot run it: misaligned columns,
// too little shared memory); fast selects 64-bit accumulation.  The launch
// covers the first floor(n / ST_TILE) * ST_TILE rows; the caller runs the
// remaining rows through launch_agg_shared (64-bit accumulation stays exact
// there: both keep the same low words, and the high words are ignored).
// With fast, bounds[s] must give every sum's term range; the layout fails
// when a 32-bit table cannot hold `rows` rows' worth of sums.
// geom: the kernel's geometry (the ahead-of-time kernel's is AOT_GEOM);
// max_stages caps the ring, leaving the shared memory it does not take to
// the L1 cache.
bool staged_layout_shared(const QueryDev& q, uint32_t key_bits, bool fast, const TermBounds* bounds,
                          uint64_t rows, int num_sms, const StageGeom& geom, int max_stages, StageLayout* L);
cudaError_t launch_agg_shared_staged(const QueryDev& q, const StageLayout& L, uint64_t n, uint64_t* gacc,
                                     uint32_t key_bits, bool fast, int num_sms, cudaStream_t st);
// The same launch of a run-time compiled, plan-specialised kernel with the
// signature of tpj_dense (grid and block from the layout); it covers all n
// rows, the ragged tail included (n must hold at least one whole tile).
cudaError_t launch_agg_shared_staged_jit(const void* kernel, const QueryDev& q, const StageLayout& L, uint64_t n,
                                         uint64_t* gacc, uint32_t key_bits, int num_sms, cudaStream_t st);

// Staged global-table aggregation.  stage_all = false stages only the filter
// column (selective filters: the other columns are read for surviving rows
// only).  fast: 64-bit reductions on low words (bounds proved).  Equal keys
// among a warp's rows update the table once.  Whole tiles only, as above; the
// caller runs the remaining rows through launch_agg_global.
bool staged_layout_global(const QueryDev& q, bool stage_all, StageLayout* L);
cudaError_t launch_agg_global_staged(const QueryDev& q, const StageLayout& L, uint64_t n, const AggTable& t,
                                     bool fast, int num_sms, cudaStream_t st);

// Global-table aggregation under a selective filter, in two launches:
// launch_select appends the indices of the rows of [0, n) that pass q's
// filter to sel (room for n entries) at *cursor (zeroed by the caller), and
// launch_agg_selected joins, keys and aggregates those *cursor rows (at most
// max_rows; the filter is not evaluated again).  select_usable: the query and
// row count suit it (a filter on a 16-byte aligned column, no further joins,
// no fan-out, fewer than 2^32 rows).
bool select_usable(const QueryDev& q, uint64_t n);
cudaError_t launch_select(const QueryDev& q, uint64_t n, uint32_t* sel, unsigned long long* cursor, int num_sms,
                          cudaStream_t st);
cudaError_t launch_agg_selected(const QueryDev& q, const uint32_t* sel, const unsigned long long* count,
                                uint64_t max_rows, const AggTable& t, bool fast, int num_sms, cudaStream_t st);

// ------------------------------------------------------- partitioned join
//
// Partition of a join key: the top log2(P) bits of fmix64(key), for every key
// width.  counts[p] += rows of partition p (build rows the dimension
// predicate admits; fact rows passing the query's filter and the lookahead
// filter).
cudaError_t launch_part_hist(const BuildDev& b, uint64_t n, int shift, unsigned long long* counts, int num_sms,
                             cudaStream_t st);
// Fan-out build: the admitted rows' (key, payload) pairs appended at *ctr
// (and their keys into the lookahead filter); after sorting by key, the first
// row of every run of equal keys as (key, its index) pairs at *ctr.
cudaError_t launch_many_collect(const BuildDev& b, uint64_t n, uint64_t* keys, uint32_t* pays,
                                unsigned long long* ctr, int num_sms, cudaStream_t st);
cudaError_t launch_many_heads(const uint64_t* keys, uint64_t n, int64_t* hkeys, uint32_t* hidx,
                              unsigned long long* ctr, int num_sms, cudaStream_t st);
cudaError_t launch_part_hist_fact(const QueryDev& q, uint64_t n, int shift, uint64_t spill_mask,
                                  unsigned long long* counts, int num_sms, cudaStream_t st);
// Build side: rows of resident partitions (bit set in b.jt.part_mask) are
// inserted; the others go to (keys, pays) at base[p] + cursor[p]++.
cudaError_t launch_build_part(const BuildDev& b, uint64_t n, const unsigned long long* base,
                              unsigned long long* cursor, int64_t* keys, uint32_t* pays, int num_sms,
                              cudaStream_t st);
// Inserts (key, payload) pairs spilled by launch_build_part.
cudaError_t launch_build_pairs(const JoinTable& jt, const int64_t* keys, const uint32_t* pays, uint64_t n,
                               uint32_t* err, int num_sms, cudaStream_t st);
// Fact side: rows that pass the filter and whose key falls in a partition of
// spill_mask are copied, column by column (cols[c] != nullptr), to
// out[c] + (base[p] + cursor[p]++) * size.
// A column's rows are stored narrow when w[c] < esize[c]: (value - base[c])
// in w[c] bytes (frame of reference, as host pages store them).
struct SpillCols {
    const void* src[32];
    void* dst[32];
    int64_t base[32];
    int32_t esize[32];
    int32_t w[32];
    int32_t n;
};
cudaError_t launch_fact_spill(const QueryDev& q, uint64_t n, uint64_t spill_mask, const SpillCols& cols,
                              const unsigned long long* base, unsigned long long* cursor, int num_sms,
                              cudaStream_t st);

// Minimum and maximum of a column (out[0] = min, out[1] = max, initialised by
// the caller to INT64_MAX / INT64_MIN).
cudaError_t launch_minmax(const DevCol& c, uint64_t n, long long* out, int num_sms, cudaStream_t st);
// Direct tables: the output rows in key order without a sort.  Occupied
// slots per chunk of DIRECT_CHUNK slots, an exclusive scan of those counts
// (offsets[n_chunks] = total), then each chunk writes its rows.
constexpr uint32_t DIRECT_CHUNK = 4096;
cudaError_t launch_direct_count(const AggTable& t, uint64_t n_slots, uint32_t* counts, int num_sms,
                                cudaStream_t st);
cudaError_t launch_direct_scan(const uint32_t* counts, uint64_t n_chunks, unsigned long long* offsets,
                               cudaStream_t st);
cudaError_t launch_direct_emit(const AggTable& t, uint64_t n_slots, const unsigned long long* offsets, int n_sum,
                               const OutDev& o, bool lo_only, int num_sms, cudaStream_t st);
// compaction of the global table into (key, slot) pairs + max key
cudaError_t launch_compact_global(const AggTable& t, uint64_t cap_with_side, uint64_t* keys,
                                  uint32_t* idx, unsigned long long* count,
                                  unsigned long long* maxkey, int num_sms, cudaStream_t st);
// lo_only: sums were accumulated as 64-bit low words (high words by sign extension)
cudaError_t launch_gather_global(const AggTable& t, const uint64_t* sorted_keys,
                                 const uint32_t* sorted_idx, uint64_t n, int n_sum, const OutDev& o,
                                 int num_sms, cudaStream_t st, bool lo_only = false);

// Narrow columns of host-page batches widened after their copy: entry k holds
// rows[k] values of (value - base[k]) as unsigned integers, either bits[k]
// bits per row packed LSB first into little-endian 32-bit words (src need not
// be word-aligned: the words are read from the aligned address below it) or
// w[k] bytes per row (1, 2 or 4); dst gets the out[k]-byte (1, 4 or 8) values.
// One launch widens every (batch, column) entry of a staging slot.
constexpr int MAX_DECODE = 64;
struct DecodeCols {
    const void* src[MAX_DECODE];
    void* dst[MAX_DECODE];
    int64_t base[MAX_DECODE];
    uint64_t rows[MAX_DECODE];
    uint8_t w[MAX_DECODE];
    uint8_t bits[MAX_DECODE];
    uint8_t out[MAX_DECODE];
    int32_t n;
};
cudaError_t launch_decode(const DecodeCols& d, int num_sms, cudaStream_t st);

// Rows of the filter column that pass, among `samples` evenly spaced rows.
cudaError_t launch_sample_filter(const QueryDev& q, uint64_t n, uint32_t samples,
                                 unsigned long long* out, cudaStream_t st);

// LSD radix sort of (key, value) pairs by the low `bits` key bits, 8 bits per
// pass.  *keys/*vals and *tmp_keys/*tmp_vals are swapped as passes ping-pong,
// so on return *keys/*vals point at the sorted data.  hist is scratch of
// radix_sort_hist_words(n) 32-bit words.
uint64_t radix_sort_hist_words(uint64_t n);
cudaError_t radix_sort_pairs(uint64_t** keys, uint32_t** vals, uint64_t** tmp_keys,
                             uint32_t** tmp_vals, uint32_t* hist, uint64_t n, int bits,
                             cudaStream_t st);
#endif  // __CUDACC_RTC__

}  // namespace tpk
