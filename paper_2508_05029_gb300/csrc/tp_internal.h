// Host-side state behind the C ABI: engine, page pool, budget, tables, plans
// and results.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/theseus_gb.h"
#include "kernels.cuh"

namespace tp {

// thread-local error message; returns code for tail calls
tp_status fail(tp_status code, const char* fmt, ...);
void clear_error();

#define TP_TRY_CUDA(call)                                                             \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return ::tp::fail(TP_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int type_size(int32_t type);

// ------------------------------------------------------------- page pool
// One page-locked allocation of n_pages * page_bytes made at engine init and
// cut into equal pages; a free stack gives O(1) alloc/free (Section 3.4).
struct PagePool {
    uint8_t* base = nullptr;
    uint64_t page_bytes = 0;
    uint32_t n_pages = 0;
    std::vector<uint32_t> free_stack;
    std::vector<uint8_t> lent;
    std::mutex mu;
    int fail_next = 0;
};

// ----------------------------------------------------------------- budget
// Reservations before execution (Section 3.3.2): a task states its device
// bytes up front; a reservation that does not fit under the cap fails instead
// of running into out-of-memory mid-way.
struct Budget {
    std::mutex mu;
    std::condition_variable cv;
    uint64_t cap = 0;
    uint64_t reserved = 0;
    uint64_t peak = 0;
    int fail_next = 0;
};

// A contiguous piece of one column inside one page.
struct Extent {
    uint32_t page;
    uint32_t pad;
    uint64_t offset;   // bytes into the page
    uint64_t bytes;
};

// One batch of a paged table: a row range whose columns lie back to back
// across a run of pages.
// One batch of a host-page table.  A column may be stored narrow (frame of
// reference): enc_w[c] bytes per row of (value - enc_base[c]) as an unsigned
// integer, enc_w[c] = 0 meaning the full width of the column's type.
struct Batch {
    uint64_t row0 = 0;
    uint64_t rows = 0;
    std::vector<std::vector<Extent>> cols;   // per column
    std::vector<uint32_t> pages;
    std::vector<uint8_t> enc_w;              // per column (empty: every column full width)
    std::vector<int64_t> enc_base;
    // per column (empty: none): bits per value of a bit-packed column (value -
    // enc_base, LSB first in little-endian 32-bit words), 0 for byte widths;
    // a packed column's enc_w is ceil(bits / 8), the bytes per row it takes in
    // a device staging slot
    std::vector<uint8_t> enc_bits;
    int width(int c, int32_t type) const;    // bytes per row of column c in a staging slot
    uint64_t stored_bytes(int c, int32_t type) const;   // bytes of column c in the pages
    bool narrow(int c) const { return !enc_w.empty() && enc_w[c] != 0; }
    bool packed(int c) const { return !enc_bits.empty() && enc_bits[c] != 0; }
};

enum Placement : int32_t { PL_PAGES = TP_HOST_PAGES, PL_DEVICE = TP_DEVICE, PL_WRAPPED = 3 };

// The streams and pinned status words one execution uses.  The engine owns
// one lane (its compute and copy streams); every serving worker owns its own,
// so executions on different lanes overlap on the device.
struct Lane {
    cudaStream_t compute = nullptr;
    cudaStream_t copy = nullptr;      // host -> device prefetch
    cudaStream_t spill = nullptr;     // device -> host spill copies (the other link direction)
    uint64_t* host_words = nullptr;   // 4 KB pinned
};

}  // namespace tp

struct tp_engine {
    tp_config cfg{};
    int device = 0;
    int num_sms = 0;
    tp::PagePool pool;
    tp::Budget budget;
    cudaStream_t compute = nullptr;
    cudaStream_t copy = nullptr;
    cudaStream_t spill = nullptr;
    bool own_compute = false;
    uint32_t copy_flags = 0;     // TP_COPY_* (tp_set_copy_options)
    std::mutex exec_mu;          // one execution at a time on the engine streams
    std::mutex obj_mu;
    // statistics
    std::atomic<uint64_t> h2d_bytes{0}, d2h_bytes{0}, batches{0}, launches{0}, retries{0};
    std::atomic<uint64_t> jit_compiles{0}, jit_failures{0}, jit_launches{0}, jit_us{0};
    std::atomic<uint64_t> split_passes{0}, lip_filters{0};
    // small pinned scratch for status words read back after an execution
    uint64_t* host_words = nullptr;
    tp::Lane lane0;                  // compute, copy, host_words of the engine itself
    // fused-kernel timing (TP_FLAG_TIME_KERNELS)
    std::mutex time_mu;
    double agg_ms = 0;
    double part_ms[3] = {0, 0, 0};   // partitioned join phases: build side, fact stream, spilled partitions
    uint64_t agg_launches = 0, agg_rows = 0;
};

struct tp_table {
    tp_engine* eng = nullptr;
    uint64_t serial = 0;    // unique per table created in this process
    std::vector<int32_t> types;
    std::vector<int32_t> scales;
    std::vector<std::string> names;
    uint64_t batch_rows = 0;
    uint64_t rows = 0;
    int32_t placement = tp::PL_PAGES;
    std::vector<tp::Batch> batches;
    std::vector<void*> dev_cols;       // device / wrapped placement
    uint64_t dev_reserved = 0;
    // per-column minimum and maximum over all rows (valid when rows > 0): the
    // bounds that prove when 64-bit accumulation cannot overflow
    std::vector<int64_t> cmin, cmax;
    // spill tables: appends continue one page chain owned by the table
    std::vector<uint32_t> chain;       // pages in order
    uint64_t chain_used = 0;           // bytes of the chain in use
};

struct tp_plan {
    tp_engine* eng = nullptr;
    uint64_t serial = 0;    // unique per plan created in this process
    tp_plan_desc d{};
    int n_sum = 0;
    int sum_of_agg[8];      // sum slot of each aggregate, -1 for COUNT
    int key_bits = 0;       // total packed key width
    int dim_bits = 0;
    int gdpos[4];
    int strategy = TP_AGG_SHARED;
    float load_factor = 0.5f;
    // execution history (Section 3.3.2: observed consumption refines later
    // reservations)
    uint64_t history_groups = 0;
    double selectivity = -1.0;   // sampled filter pass rate, < 0 until measured
    // joined dimensions: none, or the first (d.dim) and the star join's
    // further ones, each with its join columns and predicate (col < 0: none)
    int n_dims = 0;
    tp_table* dims[4] = {};
    tp_join joins[4] = {};
    tp_filter dflt[4] = {};
    double dim_sel[4] = {-1.0, -1.0, -1.0, -1.0};   // sampled predicate pass rates
    int gdim[4] = {-1, -1, -1, -1};                 // dimension of group field g, -1: fact
};

struct tp_result {
    tp_engine* eng = nullptr;
    cudaStream_t stream = nullptr;  // stream its device memory is ordered on (lane compute stream)
    uint64_t n_groups = 0;
    int n_agg = 0;
    int n_sum = 0;
    int sum_of_agg[8];
    bool is_avg[8];
    void* dev = nullptr;            // one device allocation holding every array
    uint64_t reserved = 0;
    uint64_t* d_keys = nullptr;
    int64_t* d_counts = nullptr;
    uint64_t* d_sums[8] = {};
    double* d_avgs[8] = {};
    // host copies, filled on first access
    std::mutex mu;
    std::vector<uint64_t> h_keys;
    std::vector<int64_t> h_counts;
    std::vector<std::vector<tp_i128>> h_sums;
    std::vector<std::vector<double>> h_avgs;
    bool have_keys = false, have_counts = false;
    std::vector<bool> have_sum, have_avg;
};

namespace tp {

// Join tables kept on the device across executions (serving): keyed by the
// dimension table, key column, dimension group fields, load factor and table
// kind.  An entry is built once by the execution that misses (its lane
// synchronises and checks the build before publishing it), then shared.
struct DimCache {
    struct Entry {
        tpk::JoinTable jt{};
        void* mem = nullptr;
        uint64_t bytes = 0;       // reserved in the engine budget
        bool ready = false;
        int users = 0;
        uint64_t last_use = 0;
    };
    std::mutex mu;
    std::condition_variable cv;
    std::map<std::string, Entry> entries;
    uint64_t tick = 0, hits = 0, misses = 0, evictions = 0;
};
// Frees idle cached tables (least recently used first) until `need` bytes
// are released (0: all idle ones); returns the number evicted.
int cache_evict_idle(tp_engine* e, DimCache* c, uint64_t need);
// One execution of p on lane (cache may be NULL); the caller serialises
// executions of the same plan and of the same lane.
tp_status execute_on_lane(tp_plan* p, Lane* lane, DimCache* cache, tp_result** out);

// Kernel `entry` compiled at run time for the shape struct in `prelude`
// (cached per process); nullptr when run-time compilation is unavailable or
// failed for this shape, with the reason in *why.
const void* jit_kernel(tp_engine* e, const std::string& prelude, const char* entry, std::string* why);

// budget helpers
tp_status reserve(tp_engine* e, uint64_t bytes);
void release(tp_engine* e, uint64_t bytes);
// QueryDev of a plan for one batch of fact columns (colptr[c] = device
// address of fact column c's first row; nullptr for unread columns); jtx:
// the further tables of a star join.
tpk::QueryDev plan_query_dev(const tp_plan* p, const std::vector<const void*>& colptr, const tpk::JoinTable& jt,
                             uint32_t* err, bool eager, const tpk::JoinTable* jtx = nullptr);
// Dense dimension keys: the key range of column col is at most twice the
// row count (and below 2^31), so a direct-mapped join table of *range slots
// serves it.
bool direct_join_range(const tp_table* dim, int col, uint64_t* range);
// Dense group keys: from the group fields' column bounds, every packed key of
// a surviving row lies in [*kmin, *kmin + *span) (false when a bound is
// negative or wider than its field).
bool direct_group_range(const tp_plan* p, const tp_table* fact, const tp_table* dim, uint64_t* kmin,
                        uint64_t* span);
// Column bounds prove every sum of the plan stays inside int64 over the fact table.
bool sums_fit_int64(const tp_plan* p, const tp_table* fact);
// Per-row term range of every sum slot (valid when sums_fit_int64 holds).
void term_bounds(const tp_plan* p, const tp_table* fact, tpk::TermBounds* out);
// out[s] = 1 for MUL_SUB sum slots whose two factors fit in int32 by the
// column statistics.
void narrow_products(const tp_plan* p, const tp_table* fact, int* out);
// A plan shape as a struct named `name` of compile-time constants for the
// run-time compiled kernels; mode[s] is sum s's 32-bit accumulation mode
// (fast only); lo_only (not fast): 64-bit low-word sums.
std::string shape_struct(const std::string& name, const tpk::QueryDev& q, const int8_t* mode, bool fast,
                         bool lo_only, const int* narrow);
// The source (shape struct JS and the kernel include) of a dense staged
// launch's run-time compiled kernel.
std::string dense_shape(const tpk::QueryDev& q, const tpk::StageLayout& L, bool fast, const int* narrow);
// Host-to-device copy of column c of batch b (t's page layout) on `st`: a
// full-width column lands at full + row_off * size, a narrow one at
// enc + row_off * size (enc is then widened by widen_batch).  Adds the bytes
// to the engine's counter.  With stage, the bytes are first copied on the
// host to *stage (page-locked, advanced past them) and sent from there.
tp_status copy_batch_column(tp_engine* e, const tp_table* t, const Batch& b, int c, void* full, void* enc,
                            uint64_t row_off, cudaStream_t st, uint8_t** stage = nullptr);
// Widens batch b's narrow columns among cols (enc -> full, the offsets of
// copy_batch_column at row_off) with one launch on st.
tp_status widen_batch(tp_engine* e, const tp_table* t, const Batch& b, const std::vector<int>& cols,
                      const std::vector<void*>& full, const std::vector<void*>& enc, uint64_t row_off,
                      cudaStream_t st);
// The same for batches [first, last) of t copied one after another into the
// same slots (each at the rows of the ones before it), in as few launches as
// the decode descriptor allows.
tp_status widen_batches(tp_engine* e, const tp_table* t, size_t first, size_t last, const std::vector<int>& cols,
                        const std::vector<void*>& full, const std::vector<void*>& enc, cudaStream_t st);
// Narrowest frame-of-reference width (1, 2 or 4 bytes) for values in [lo,
// hi] of a column of full width `full`, or 0 when it saves nothing.
int frame_width(int64_t lo, int64_t hi, int full);
// Bits that hold hi - lo (at least 1).
int frame_bits(int64_t lo, int64_t hi);
// ORs v[0..n) (each below 2^bits) into the zeroed words: value i at stream
// bits [i * bits, (i + 1) * bits), LSB first, stream bit j = bit j % 32 of
// words[j / 32] (the bit-packed page layout).
void pack_bits(const uint64_t* v, uint64_t n, int bits, uint32_t* words);
// Whether any batch of t stores a narrow column.
bool has_narrow(const tp_table* t);
// The widest narrow encoding of column c over t's batches (0: never narrow).
int narrow_width_max(const tp_table* t, int c);
// ----------------------------------------------------- batched execution
// Sizes and choices of one query inside a persistent batched launch (the
// queue kernel of batch.cu): its join table, dense accumulators and output
// arrays, probe tile, and whether a tile accumulates in a 32-bit
// shared-memory table first (mode[s]: 1 low word, 2 low + carry word).
constexpr uint64_t BATCH_BUILD_CHUNK = 65536;   // dimension rows per build task
struct BatchPrep {
    uint64_t join_cap = 0, join_bytes = 0, acc_bytes = 0, out_bytes = 0, tile = 0, range = 0;
    uint64_t build_items = 0, probe_items = 0, final_items = 0;
    bool join = false, key64 = false, smem = false, fast = false, direct = false;
    tpk::TermBounds bounds[tpk::MAX_SUM] = {};
    int8_t mode[tpk::MAX_SUM] = {};
    uint32_t smem_bytes = 0;
};
// Whether plan p (index i, for the message) can run in a batched launch:
// device-resident tables, at most one join, no fan-out, at most 20 key bits.
tp_status batch_check_plan(const tp_engine* e, const tp_plan* p, int i);
// Sizes and choices of p: join load factor lf_tuned (0: the plan's), probe
// tiles of rows_per_warp rows per warp, agg TP_AGG_GLOBAL to keep tiles out
// of shared memory.
void batch_prep(const tp_engine* e, const tp_plan* p, float lf_tuned, uint32_t rows_per_warp, int agg, BatchPrep* x);
// The device descriptor of p in a batch: its join table at join_slots (side
// cell at side), accumulators at acc, outputs in out, its finalisation
// ranges' words at final_done / final_end (both zeroed before every run);
// shape id 0.
void batch_query_desc(const tp_plan* p, const BatchPrep& x, void* join_slots, uint32_t* side, uint64_t* acc,
                      uint32_t* err, const tpk::OutDev& out, tpk::BatchQuery* B, unsigned* final_done = nullptr,
                      unsigned long long* final_end = nullptr);
// Appends query qi's tasks of one kind (BI_BUILD chunks, BI_PROBE tiles or
// its BI_FINAL group ranges) to items.
void batch_items(const tp_plan* p, const BatchPrep& x, uint32_t qi, int kind, std::vector<tpk::BatchItem>* items);
// The shape struct `name` of a batched query for the run-time compiled queue
// kernel, and that kernel's source for shapes JS_0 .. JS_{n-1}.
std::string batch_shape(const tp_plan* p, const tpk::BatchQuery& B, const BatchPrep& x, const std::string& name);
std::string batch_kernel_source(const std::vector<std::string>& shapes);
// Resident CTAs of the queue kernel (run-time compiled, or the ahead-of-time
// one for nullptr) with smem_bytes of dynamic shared memory.
int batch_kernel_grid(const void* jit_kernel_or_null, uint32_t smem_bytes, int num_sms);
// Result arrays for `cap` groups of p (reserved and allocated on st); od gets
// their device addresses, its group count pointing at n_groups_dev.
tp_status alloc_result(tp_engine* e, tp_plan* p, uint64_t cap, tp_result** out, tpk::OutDev* od,
                       unsigned long long* n_groups_dev, cudaStream_t st);

// device memory (stream-ordered allocator on the compute stream)
tp_status dev_alloc(tp_engine* e, void** p, uint64_t bytes, cudaStream_t st);
void dev_free(tp_engine* e, void* p, cudaStream_t st);

}  // namespace tp
