// Device-side parameter blocks and launchers of the relational hot path.
//
// Hash tables use open addressing with linear probing.  The slot of a key is
// fmix64(key) & mask, where fmix64 is the 64-bit finaliser of MurmurHash3
// (Appleby, public domain).  The top 6 bits of the same hash pick the radix
// partition, so partition bits and slot bits never overlap for tables below
// 2^58 slots.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

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

struct DevCol {
    const void* ptr;
    int32_t type;
    int32_t pad;
};

// Join hash table.  32-bit keys: one 64-bit word per slot, payload << 32 | key,
// EMPTY = all ones.  64-bit keys: two words per slot {key, payload}, EMPTY key
// = all ones.  A key equal to the EMPTY pattern lives in side[]:
// side[0] = 1 when present, side[1] = its payload.
struct JoinTable {
    uint64_t* slots;
    uint64_t mask;          // capacity - 1 (capacity a power of two)
    uint32_t* side;         // 2 words
    int32_t key64;
    int32_t pad;
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
};

// Global aggregation table: slot = {key, count, (lo, hi) per sum}, EMPTY key =
// all ones; the all-ones key itself is kept in a dedicated side slot placed
// after the last regular slot.
struct AggTable {
    uint64_t* slots;
    uint64_t mask;
    uint32_t words;          // 64-bit words per slot = 2 + 2 * n_sum
    uint32_t pad;
    unsigned long long* used;   // occupied slots counter
    uint64_t max_used;          // beyond this, new keys set ERR_OVERFLOW
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

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return cudaGetLastError().

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
cudaError_t launch_final_dense(const uint64_t* gacc, uint32_t key_bits, int n_sum, const OutDev& o,
                               cudaStream_t st);
// compaction of the global table into (key, slot) pairs + max key
cudaError_t launch_compact_global(const AggTable& t, uint64_t cap_with_side, uint64_t* keys,
                                  uint32_t* idx, unsigned long long* count,
                                  unsigned long long* maxkey, int num_sms, cudaStream_t st);
cudaError_t launch_gather_global(const AggTable& t, const uint64_t* sorted_keys,
                                 const uint32_t* sorted_idx, uint64_t n, int n_sum, const OutDev& o,
                                 int num_sms, cudaStream_t st);

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

}  // namespace tpk
