// Engine lifetime, pinned page pool, device-memory budget and table
// registration behind the C ABI.
//
// Paper basis: Section 3.4 (a pool of fixed-size page-locked buffers
// allocated at engine initialisation; columns laid across buffers so one
// column may span several; a small unused tail per batch), Section 3.3.2
// (tasks reserve memory before executing), Section 3.1 (batches are row
// slices of all columns).
#include <algorithm>
#include <cstdarg>
#include <climits>
#include <cstdio>
#include <cstdlib>

#include "tp_internal.h"

namespace tp {

static thread_local char g_err[512] = "";

tp_status fail(tp_status code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = 0; }

int type_size(int32_t type) {
    switch (type) {
    case TP_I32: return 4;
    case TP_I64: return 8;
    case TP_U8: return 1;
    default: return 0;
    }
}

tp_status reserve(tp_engine* e, uint64_t bytes) {
    std::lock_guard<std::mutex> lk(e->budget.mu);
    if (e->budget.fail_next > 0) {
        --e->budget.fail_next;
        return fail(TP_E_BUDGET, "device reservation of %llu bytes refused (injected)",
                    (unsigned long long)bytes);
    }
    if (e->budget.reserved + bytes > e->budget.cap)
        return fail(TP_E_BUDGET, "device reservation of %llu bytes exceeds budget (%llu of %llu reserved)",
                    (unsigned long long)bytes, (unsigned long long)e->budget.reserved,
                    (unsigned long long)e->budget.cap);
    e->budget.reserved += bytes;
    if (e->budget.reserved > e->budget.peak) e->budget.peak = e->budget.reserved;
    return TP_OK;
}

void release(tp_engine* e, uint64_t bytes) {
    {
        std::lock_guard<std::mutex> lk(e->budget.mu);
        e->budget.reserved = bytes > e->budget.reserved ? 0 : e->budget.reserved - bytes;
    }
    e->budget.cv.notify_all();
}

tp_status dev_alloc(tp_engine* e, void** p, uint64_t bytes, cudaStream_t st) {
    (void)e;
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    cudaError_t err = cudaMallocAsync(p, bytes, st);
    if (err != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(TP_E_CUDA, "device allocation of %llu bytes failed: %s", (unsigned long long)bytes,
                    cudaGetErrorString(err));
    }
    return TP_OK;
}

tp_status copy_batch_column(tp_engine* e, const tp_table* t, const Batch& b, int c, void* full, void* enc,
                            uint64_t row_off, cudaStream_t st, uint8_t** stage) {
    // a narrow column's rows land at its widest encoding's offsets (enc holds
    // narrow_width_max bytes per row)
    const uint64_t sz = b.narrow(c) ? (uint64_t)narrow_width_max(t, c) : type_size(t->types[c]);
    uint8_t* dst = (uint8_t*)(b.narrow(c) ? enc : full) + row_off * sz;
    // a bit-packed column copies the bytes its values occupy, not the rest of
    // its last word, so it stays inside its rows' share of the staging slot
    uint64_t left = b.packed(c) ? (b.rows * b.enc_bits[c] + 7) / 8 : UINT64_MAX;
    for (const Extent& x : b.cols[c]) {
        const uint64_t bytes = std::min<uint64_t>(x.bytes, left);
        if (bytes == 0) break;
        left -= bytes;
        const uint8_t* src = (const uint8_t*)tp_page_ptr(e, x.page) + x.offset;
        if (stage) {
            memcpy(*stage, src, bytes);
            src = *stage;
            *stage += bytes;
        }
        const cudaError_t err = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
        if (err != cudaSuccess) return fail(TP_E_CUDA, "batch copy: %s", cudaGetErrorString(err));
        dst += bytes;
        e->h2d_bytes += bytes;
    }
    return TP_OK;
}

namespace {

// Decode entries of one or more batches, launched whenever the descriptor is
// full and once at the end.
struct Widener {
    tp_engine* e;
    cudaStream_t st;
    tpk::DecodeCols d{};
    tp_status flush() {
        if (d.n == 0) return TP_OK;
        const cudaError_t err = tpk::launch_decode(d, e->num_sms, st);
        if (err != cudaSuccess) return fail(TP_E_CUDA, "widening a batch: %s", cudaGetErrorString(err));
        e->launches++;
        d.n = 0;
        std::fill(last.begin(), last.end(), -1);
        return TP_OK;
    }
    std::vector<int> last;   // per column of cols: its entry in d, -1 if none
    // batch b's narrow columns among cols, copied at row offset row_off of
    // the staging slots enc (narrow) / full (widened); a byte-encoded column
    // that continues the previous batch's entry (same encoding, rows at the
    // slot's width) extends it
    tp_status add(const tp_table* t, const Batch& b, const std::vector<int>& cols, const std::vector<void*>& full,
                  const std::vector<void*>& enc, uint64_t row_off) {
        if (last.size() != cols.size()) last.assign(cols.size(), -1);
        for (size_t i = 0; i < cols.size(); ++i) {
            const int c = cols[i];
            if (!b.narrow(c)) {
                last[i] = -1;
                continue;
            }
            const uint64_t sz = type_size(t->types[c]);
            const uint64_t wmax = (uint64_t)narrow_width_max(t, c);
            const uint8_t* src = (const uint8_t*)enc[i] + row_off * wmax;
            const int k = last[i];
            if (k >= 0 && !b.packed(c) && d.bits[k] == 0 && d.w[k] == b.enc_w[c] && b.enc_w[c] == wmax &&
                d.base[k] == b.enc_base[c] && (const uint8_t*)d.src[k] + d.rows[k] * wmax == src) {
                d.rows[k] += b.rows;
                continue;
            }
            last[i] = d.n;
            d.src[d.n] = src;
            d.dst[d.n] = (uint8_t*)full[i] + row_off * sz;
            d.base[d.n] = b.enc_base[c];
            d.rows[d.n] = b.rows;
            d.w[d.n] = b.enc_w[c];
            d.bits[d.n] = b.packed(c) ? b.enc_bits[c] : 0;
            d.out[d.n] = (uint8_t)sz;
            if (++d.n == tpk::MAX_DECODE) {
                tp_status s = flush();
                if (s) return s;
            }
        }
        return TP_OK;
    }
};

}  // namespace

tp_status widen_batch(tp_engine* e, const tp_table* t, const Batch& b, const std::vector<int>& cols,
                      const std::vector<void*>& full, const std::vector<void*>& enc, uint64_t row_off,
                      cudaStream_t st) {
    Widener w{e, st};
    tp_status s = w.add(t, b, cols, full, enc, row_off);
    return s ? s : w.flush();
}

tp_status widen_batches(tp_engine* e, const tp_table* t, size_t first, size_t last, const std::vector<int>& cols,
                        const std::vector<void*>& full, const std::vector<void*>& enc, cudaStream_t st) {
    Widener w{e, st};
    uint64_t row_off = 0;
    for (size_t bi = first; bi < last; ++bi) {
        tp_status s = w.add(t, t->batches[bi], cols, full, enc, row_off);
        if (s) return s;
        row_off += t->batches[bi].rows;
    }
    return w.flush();
}

void pack_bits(const uint64_t* v, uint64_t n, int bits, uint32_t* words) {
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t at = i * (uint64_t)bits;
        const uint64_t k = at >> 5;
        const int sh = (int)(at & 31);
        words[k] |= (uint32_t)(v[i] << sh);
        if (sh + bits > 32) words[k + 1] |= (uint32_t)(v[i] >> (32 - sh));
    }
}

int frame_bits(int64_t lo, int64_t hi) {
    const uint64_t span = (uint64_t)hi - (uint64_t)lo;
    int bits = 1;
    while (bits < 64 && (span >> bits) != 0) ++bits;
    return bits;
}

int frame_width(int64_t lo, int64_t hi, int full) {
    const uint64_t span = (uint64_t)hi - (uint64_t)lo;
    const int w = span <= 0xFFull ? 1 : span <= 0xFFFFull ? 2 : span <= 0xFFFFFFFFull ? 4 : 8;
    return w < full ? w : 0;
}

int narrow_width_max(const tp_table* t, int c) {
    int w = 0;
    for (const Batch& b : t->batches)
        if (b.narrow(c)) w = std::max<int>(w, b.enc_w[c]);
    return w;
}

bool has_narrow(const tp_table* t) {
    for (const Batch& b : t->batches)
        for (size_t c = 0; c < b.enc_w.size(); ++c)
            if (b.enc_w[c]) return true;
    return false;
}

void dev_free(tp_engine* e, void* p, cudaStream_t st) {
    (void)e;
    if (p) cudaFreeAsync(p, st);
}

}  // namespace tp

using namespace tp;

extern "C" {

const char* tp_last_error(void) { return tp::g_err; }

void tp_config_default(tp_config* c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->page_bytes = 64ull << 20;
    c->n_pages = 0;
    c->device_budget_bytes = 0;
    c->prefetch_depth = 2;
    c->cuda_device = 0;
    c->batch_rows = 4ull << 20;
    c->load_factor = 0.5f;
    c->agg_strategy = TP_AGG_AUTO;
    c->compute_stream = nullptr;
}

tp_status tp_init(const tp_config* cfg, tp_engine** out) {
    clear_error();
    if (!cfg || !out) return fail(TP_E_INVALID, "tp_init: NULL argument");
    *out = nullptr;
    if (cfg->page_bytes == 0 || cfg->batch_rows == 0 || cfg->prefetch_depth < 0 ||
        cfg->prefetch_depth > 64 || !(cfg->load_factor > 0.05f && cfg->load_factor <= 0.9f) ||
        cfg->agg_strategy < TP_AGG_AUTO || cfg->agg_strategy > TP_AGG_GLOBAL)
        return fail(TP_E_INVALID, "tp_init: invalid configuration");
    std::unique_ptr<tp_engine> e(new (std::nothrow) tp_engine());
    if (!e) return fail(TP_E_NOMEM, "tp_init: out of host memory");
    e->cfg = *cfg;
    e->cfg.page_bytes = (cfg->page_bytes + 4095) & ~4095ull;
    e->device = cfg->cuda_device;
    TP_TRY_CUDA(cudaSetDevice(e->device));
    TP_TRY_CUDA(cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, e->device));
    size_t free_b = 0, total_b = 0;
    TP_TRY_CUDA(cudaMemGetInfo(&free_b, &total_b));
    e->budget.cap = cfg->device_budget_bytes ? cfg->device_budget_bytes : (uint64_t)(free_b * 0.9);
    // keep freed stream-ordered allocations cached in the device pool
    cudaMemPool_t pool;
    TP_TRY_CUDA(cudaDeviceGetDefaultMemPool(&pool, e->device));
    uint64_t threshold = ~0ull;
    TP_TRY_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold));
    TP_TRY_CUDA(cudaStreamCreateWithFlags(&e->copy, cudaStreamNonBlocking));
    TP_TRY_CUDA(cudaStreamCreateWithFlags(&e->spill, cudaStreamNonBlocking));
    if (cfg->compute_stream) {
        e->compute = (cudaStream_t)cfg->compute_stream;
    } else {
        TP_TRY_CUDA(cudaStreamCreateWithFlags(&e->compute, cudaStreamNonBlocking));
        e->own_compute = true;
    }
    TP_TRY_CUDA(cudaHostAlloc((void**)&e->host_words, 4096, cudaHostAllocDefault));
    // the page pool: one page-locked allocation cut into equal pages
    PagePool& pp = e->pool;
    pp.page_bytes = e->cfg.page_bytes;
    pp.n_pages = cfg->n_pages;
    if (pp.n_pages) {
        cudaError_t err = cudaHostAlloc((void**)&pp.base, pp.page_bytes * pp.n_pages, cudaHostAllocDefault);
        if (err != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(e->host_words);
            cudaStreamDestroy(e->copy);
            cudaStreamDestroy(e->spill);
            if (e->own_compute) cudaStreamDestroy(e->compute);
            return fail(TP_E_NOMEM, "page pool of %u x %llu bytes could not be pinned: %s", pp.n_pages,
                        (unsigned long long)pp.page_bytes, cudaGetErrorString(err));
        }
        pp.free_stack.resize(pp.n_pages);
        for (uint32_t i = 0; i < pp.n_pages; ++i) pp.free_stack[i] = pp.n_pages - 1 - i;
        pp.lent.assign(pp.n_pages, 0);
    }
    e->lane0.compute = e->compute;
    e->lane0.copy = e->copy;
    e->lane0.spill = e->spill;
    e->lane0.host_words = e->host_words;
    *out = e.release();
    return TP_OK;
}

void tp_shutdown(tp_engine* e) {
    if (!e) return;
    cudaSetDevice(e->device);
    cudaStreamSynchronize(e->compute);
    cudaStreamSynchronize(e->copy);
    cudaStreamSynchronize(e->spill);
    if (e->pool.base) cudaFreeHost(e->pool.base);
    if (e->host_words) cudaFreeHost(e->host_words);
    cudaStreamDestroy(e->copy);
    cudaStreamDestroy(e->spill);
    if (e->own_compute) cudaStreamDestroy(e->compute);
    delete e;
}

// ---------------------------------------------------------------- page pool

tp_status tp_page_alloc(tp_engine* e, tp_page* out) {
    if (!e || !out) return fail(TP_E_INVALID, "tp_page_alloc: NULL argument");
    std::lock_guard<std::mutex> lk(e->pool.mu);
    if (e->pool.fail_next > 0) {
        --e->pool.fail_next;
        return fail(TP_E_POOL_EMPTY, "page pool exhausted (injected)");
    }
    if (e->pool.free_stack.empty()) return fail(TP_E_POOL_EMPTY, "page pool exhausted (%u pages)", e->pool.n_pages);
    *out = e->pool.free_stack.back();
    e->pool.free_stack.pop_back();
    e->pool.lent[*out] = 1;
    return TP_OK;
}

tp_status tp_page_free(tp_engine* e, tp_page p) {
    if (!e) return fail(TP_E_INVALID, "tp_page_free: NULL engine");
    std::lock_guard<std::mutex> lk(e->pool.mu);
    if (p >= e->pool.n_pages || !e->pool.lent[p]) return fail(TP_E_INVALID, "tp_page_free: page %u not lent", p);
    e->pool.lent[p] = 0;
    e->pool.free_stack.push_back(p);
    return TP_OK;
}

void* tp_page_ptr(tp_engine* e, tp_page p) {
    if (!e || p >= e->pool.n_pages) return nullptr;
    return e->pool.base + (uint64_t)p * e->pool.page_bytes;
}

uint64_t tp_page_bytes(const tp_engine* e) { return e ? e->pool.page_bytes : 0; }

uint32_t tp_pages_free(const tp_engine* e) {
    if (!e) return 0;
    std::lock_guard<std::mutex> lk(const_cast<tp_engine*>(e)->pool.mu);
    return (uint32_t)e->pool.free_stack.size();
}

// ------------------------------------------------------------------- budget

tp_status tp_set_device_budget(tp_engine* e, uint64_t bytes) {
    if (!e) return fail(TP_E_INVALID, "tp_set_device_budget: NULL engine");
    {
        std::lock_guard<std::mutex> lk(e->budget.mu);
        e->budget.cap = bytes;
    }
    e->budget.cv.notify_all();
    return TP_OK;
}

tp_status tp_set_copy_options(tp_engine* e, int32_t prefetch_depth, uint32_t flags) {
    clear_error();
    if (!e || prefetch_depth < 0 || prefetch_depth > 64 || (flags & ~(uint32_t)TP_COPY_PINNED_PER_BATCH))
        return fail(TP_E_INVALID, "tp_set_copy_options: bad arguments");
    std::lock_guard<std::mutex> lk(e->exec_mu);
    e->cfg.prefetch_depth = prefetch_depth;
    e->copy_flags = flags;
    return TP_OK;
}

tp_status tp_budget_query(tp_engine* e, uint64_t* reserved, uint64_t* cap) {
    if (!e) return fail(TP_E_INVALID, "tp_budget_query: NULL engine");
    std::lock_guard<std::mutex> lk(e->budget.mu);
    if (reserved) *reserved = e->budget.reserved;
    if (cap) *cap = e->budget.cap;
    return TP_OK;
}

// ------------------------------------------------------------------- tables

static tp_status check_desc(const tp_table_desc* d) {
    if (!d || d->n_cols < 1 || d->n_cols > 32 || !d->cols) return fail(TP_E_INVALID, "table: bad descriptor");
    for (int i = 0; i < d->n_cols; ++i)
        if (type_size(d->cols[i].type) == 0) return fail(TP_E_INVALID, "table: column %d has a bad type", i);
    return TP_OK;
}

static tp_table* new_table(tp_engine* e, const tp_table_desc* d) {
    static std::atomic<uint64_t> next_serial{1};
    tp_table* t = new (std::nothrow) tp_table();
    if (!t) return nullptr;
    t->eng = e;
    t->serial = next_serial++;
    t->batch_rows = d->batch_rows ? d->batch_rows : e->cfg.batch_rows;
    for (int i = 0; i < d->n_cols; ++i) {
        t->types.push_back(d->cols[i].type);
        t->scales.push_back(d->cols[i].scale);
        t->names.push_back(d->cols[i].name ? d->cols[i].name : "");
    }
    t->cmin.assign(d->n_cols, INT64_MAX);
    t->cmax.assign(d->n_cols, INT64_MIN);
    return t;
}

tp_status tp_table_create(tp_engine* e, const tp_table_desc* d, tp_table** out) {
    clear_error();
    if (!e || !out) return fail(TP_E_INVALID, "tp_table_create: NULL argument");
    tp_status s = check_desc(d);
    if (s) return s;
    *out = new_table(e, d);
    return *out ? TP_OK : fail(TP_E_NOMEM, "tp_table_create: out of host memory");
}

static void free_batch_pages(tp_engine* e, Batch& b) {
    for (uint32_t p : b.pages) tp_page_free(e, p);
    b.pages.clear();
}

int tp::Batch::width(int c, int32_t type) const { return narrow(c) ? enc_w[c] : type_size(type); }

uint64_t tp::Batch::stored_bytes(int c, int32_t type) const {
    if (packed(c)) return 4 * ((rows * enc_bits[c] + 31) / 32);   // whole 32-bit words
    return rows * (uint64_t)width(c, type);
}

namespace {

int64_t value_at(const void* col, int32_t type, uint64_t i) {
    switch (type) {
    case TP_I32: return ((const int32_t*)col)[i];
    case TP_I64: return ((const int64_t*)col)[i];
    default: return ((const uint8_t*)col)[i];
    }
}

}  // namespace

tp_status tp_table_append(tp_table* t, const void* const* cols, uint64_t nrows) {
    clear_error();
    if (!t || (!cols && nrows)) return fail(TP_E_INVALID, "tp_table_append: NULL argument");
    if (t->placement != PL_PAGES) return fail(TP_E_INVALID, "tp_table_append: table is not in host pages");
    tp_engine* e = t->eng;
    const uint64_t pb = e->pool.page_bytes;
    const size_t first_new = t->batches.size();
    const int nc = (int)t->types.size();
    const bool narrow = !(e->cfg.flags & TP_FLAG_RAW_PAGES);
    for (uint64_t r0 = 0; r0 < nrows; r0 += t->batch_rows) {
        const uint64_t rows = std::min<uint64_t>(t->batch_rows, nrows - r0);
        Batch b;
        b.row0 = t->rows + r0;
        b.rows = rows;
        if (narrow) {  // frame of reference per batch and column: the batch's minimum, the fewest bits
            b.enc_w.assign(nc, 0);
            b.enc_base.assign(nc, 0);
            b.enc_bits.assign(nc, 0);
            for (int c = 0; c < nc; ++c) {
                int64_t lo = INT64_MAX, hi = INT64_MIN;
                for (uint64_t i = r0; i < r0 + rows; ++i) {
                    const int64_t v = value_at(cols[c], t->types[c], i);
                    lo = std::min(lo, v);
                    hi = std::max(hi, v);
                }
                const int bits = frame_bits(lo, hi);
                const int full = type_size(t->types[c]);
                if (bits < 32 && bits != 8 && bits != 16 && bits < 8 * full) {   // bit-packed
                    b.enc_bits[c] = (uint8_t)bits;
                    b.enc_w[c] = (uint8_t)((bits + 7) / 8);
                } else {   // whole bytes (or full width)
                    b.enc_w[c] = (uint8_t)frame_width(lo, hi, full);
                }
                b.enc_base[c] = lo;
            }
        }
        // columns back to back, each starting on a 256-byte boundary
        std::vector<uint64_t> off(nc);
        uint64_t total = 0;
        for (int c = 0; c < nc; ++c) {
            total = (total + 255) & ~255ull;
            off[c] = total;
            total += b.stored_bytes(c, t->types[c]);
        }
        const uint64_t n_pages = (total + pb - 1) / pb;
        for (uint64_t i = 0; i < n_pages; ++i) {
            tp_page p;
            tp_status s = tp_page_alloc(e, &p);
            if (s) {
                free_batch_pages(e, b);
                for (size_t k = first_new; k < t->batches.size(); ++k) free_batch_pages(e, t->batches[k]);
                t->batches.resize(first_new);
                return s;
            }
            b.pages.push_back(p);
        }
        b.cols.resize(nc);
        std::vector<uint8_t> enc;
        std::vector<uint32_t> words;
        std::vector<uint64_t> deltas;
        for (int c = 0; c < nc; ++c) {
            const int sz = type_size(t->types[c]);
            const uint8_t* src = (const uint8_t*)cols[c] + r0 * sz;
            const int w = b.width(c, t->types[c]);
            if (b.packed(c)) {  // (value - base), LSB first, value i at bit i * bits of the word stream
                deltas.resize(rows);
                for (uint64_t i = 0; i < rows; ++i)
                    deltas[i] = (uint64_t)value_at(cols[c], t->types[c], r0 + i) - (uint64_t)b.enc_base[c];
                words.assign(b.stored_bytes(c, t->types[c]) / 4, 0u);
                pack_bits(deltas.data(), rows, b.enc_bits[c], words.data());
                src = (const uint8_t*)words.data();
            } else if (b.narrow(c)) {  // little-endian low bytes of (value - base)
                enc.resize(rows * w);
                for (uint64_t i = 0; i < rows; ++i) {
                    const uint64_t d = (uint64_t)value_at(cols[c], t->types[c], r0 + i) - (uint64_t)b.enc_base[c];
                    for (int k = 0; k < w; ++k) enc[i * w + k] = (uint8_t)(d >> (8 * k));
                }
                src = enc.data();
            }
            uint64_t pos = off[c], left = b.stored_bytes(c, t->types[c]);
            while (left) {
                const uint64_t pi = pos / pb, po = pos % pb;
                const uint64_t take = std::min<uint64_t>(left, pb - po);
                memcpy((uint8_t*)tp_page_ptr(e, b.pages[pi]) + po, src, take);
                b.cols[c].push_back(Extent{b.pages[pi], 0, po, take});
                src += take;
                pos += take;
                left -= take;
            }
        }
        t->batches.push_back(std::move(b));
    }
    // column bounds of the appended rows
    for (int c = 0; c < nc && nrows; ++c) {
        int64_t lo = t->cmin[c], hi = t->cmax[c];
        switch (t->types[c]) {
        case TP_I32: {
            const int32_t* v = (const int32_t*)cols[c];
            for (uint64_t i = 0; i < nrows; ++i) { lo = std::min<int64_t>(lo, v[i]); hi = std::max<int64_t>(hi, v[i]); }
            break;
        }
        case TP_I64: {
            const int64_t* v = (const int64_t*)cols[c];
            for (uint64_t i = 0; i < nrows; ++i) { lo = std::min(lo, v[i]); hi = std::max(hi, v[i]); }
            break;
        }
        default: {
            const uint8_t* v = (const uint8_t*)cols[c];
            for (uint64_t i = 0; i < nrows; ++i) { lo = std::min<int64_t>(lo, v[i]); hi = std::max<int64_t>(hi, v[i]); }
            break;
        }
        }
        t->cmin[c] = lo;
        t->cmax[c] = hi;
    }
    t->rows += nrows;
    return TP_OK;
}

tp_status tp_table_place(tp_table* t, int32_t placement) {
    clear_error();
    if (!t) return fail(TP_E_INVALID, "tp_table_place: NULL table");
    if (placement == TP_HOST_PAGES) {
        return t->placement == PL_PAGES ? TP_OK
                                        : fail(TP_E_INVALID, "tp_table_place: device tables stay on the device");
    }
    if (placement != TP_DEVICE) return fail(TP_E_INVALID, "tp_table_place: bad placement");
    if (t->placement != PL_PAGES) return TP_OK;
    tp_engine* e = t->eng;
    std::lock_guard<std::mutex> lk(e->exec_mu);
    const int nc = (int)t->types.size();
    uint64_t bytes = 0;
    for (int c = 0; c < nc; ++c) bytes += ((t->rows * type_size(t->types[c]) + 255) & ~255ull);
    tp_status s = reserve(e, bytes);
    if (s) return s;
    std::vector<void*> cols(nc, nullptr);
    for (int c = 0; c < nc; ++c) {
        s = dev_alloc(e, &cols[c], t->rows * type_size(t->types[c]), e->compute);
        if (s) {
            for (void* p : cols) dev_free(e, p, e->compute);
            release(e, bytes);
            return s;
        }
    }
    // narrow batches are copied into a scratch buffer of one batch, then widened in place
    uint64_t max_rows = 0;
    for (auto& b : t->batches) max_rows = std::max(max_rows, b.rows);
    void* scratch = nullptr;
    if (has_narrow(t) && (s = dev_alloc(e, &scratch, max_rows * 8 * (uint64_t)nc, e->compute))) {
        for (void* p : cols) dev_free(e, p, e->compute);
        release(e, bytes);
        return s;
    }
    cudaStreamSynchronize(e->compute);
    std::vector<int> all(nc);
    for (int c = 0; c < nc; ++c) all[c] = c;
    for (auto& b : t->batches) {
        std::vector<void*> full(nc), enc(nc);
        for (int c = 0; c < nc; ++c) {
            full[c] = (uint8_t*)cols[c] + b.row0 * type_size(t->types[c]);
            enc[c] = scratch ? (uint8_t*)scratch + (uint64_t)c * max_rows * 8 : nullptr;
            if (!s) s = copy_batch_column(e, t, b, c, full[c], enc[c], 0, e->compute);
        }
        if (!s) s = widen_batch(e, t, b, all, full, enc, 0, e->compute);   // same stream: the scratch is reused in order
        if (s) break;
    }
    if (scratch) dev_free(e, scratch, e->compute);
    const cudaError_t done = cudaStreamSynchronize(e->compute);
    if (!s && done != cudaSuccess) s = fail(TP_E_CUDA, "tp_table_place: %s", cudaGetErrorString(done));
    if (s) {
        cudaStreamSynchronize(e->compute);
        for (void* p : cols) dev_free(e, p, e->compute);
        release(e, bytes);
        return s;
    }
    for (auto& b : t->batches) free_batch_pages(e, b);
    t->batches.clear();
    t->dev_cols = cols;
    t->dev_reserved = bytes;
    t->placement = PL_DEVICE;
    return TP_OK;
}

tp_status tp_table_wrap_device(tp_engine* e, const tp_table_desc* d, const void* const* dev_cols,
                               uint64_t nrows, tp_table** out) {
    clear_error();
    if (!e || !out || !dev_cols) return fail(TP_E_INVALID, "tp_table_wrap_device: NULL argument");
    tp_status s = check_desc(d);
    if (s) return s;
    for (int c = 0; c < d->n_cols; ++c)
        if (nrows && (!dev_cols[c] || ((uintptr_t)dev_cols[c] & 15u)))
            return fail(TP_E_INVALID, "tp_table_wrap_device: column %d is NULL or not 16-byte aligned", c);
    std::unique_ptr<tp_table> t(new_table(e, d));
    if (!t) return fail(TP_E_NOMEM, "tp_table_wrap_device: out of host memory");
    t->rows = nrows;
    t->placement = PL_WRAPPED;
    for (int c = 0; c < d->n_cols; ++c) t->dev_cols.push_back(const_cast<void*>(dev_cols[c]));
    if (nrows) {  // column bounds, one reduction per column
        std::lock_guard<std::mutex> lk(e->exec_mu);
        TP_TRY_CUDA(cudaSetDevice(e->device));
        long long* h = (long long*)e->host_words;
        for (int c = 0; c < d->n_cols; ++c) {
            h[2 * c] = LLONG_MAX;
            h[2 * c + 1] = LLONG_MIN;
        }
        void* dmm = nullptr;
        tp_status s2 = dev_alloc(e, &dmm, 16 * d->n_cols, e->compute);
        if (s2) return s2;
        TP_TRY_CUDA(cudaMemcpyAsync(dmm, h, 16 * d->n_cols, cudaMemcpyHostToDevice, e->compute));
        for (int c = 0; c < d->n_cols; ++c) {
            tpk::DevCol col{};
            col.ptr = dev_cols[c];
            col.type = d->cols[c].type;
            TP_TRY_CUDA(tpk::launch_minmax(col, nrows, (long long*)dmm + 2 * c, e->num_sms, e->compute));
            e->launches++;
        }
        TP_TRY_CUDA(cudaMemcpyAsync(h, dmm, 16 * d->n_cols, cudaMemcpyDeviceToHost, e->compute));
        dev_free(e, dmm, e->compute);
        TP_TRY_CUDA(cudaStreamSynchronize(e->compute));
        for (int c = 0; c < d->n_cols; ++c) {
            t->cmin[c] = h[2 * c];
            t->cmax[c] = h[2 * c + 1];
        }
    }
    *out = t.release();
    return TP_OK;
}

uint64_t tp_table_rows(const tp_table* t) { return t ? t->rows : 0; }

uint64_t tp_table_batches(const tp_table* t) {
    if (!t) return 0;
    return t->placement == PL_PAGES ? t->batches.size() : 1;
}

void tp_table_destroy(tp_table* t) {
    if (!t) return;
    tp_engine* e = t->eng;
    if (t->placement == PL_PAGES) {
        for (auto& b : t->batches) free_batch_pages(e, b);
        for (uint32_t p : t->chain) tp_page_free(e, p);
    } else if (t->placement == PL_DEVICE) {
        cudaSetDevice(e->device);
        cudaStreamSynchronize(e->compute);
        for (void* p : t->dev_cols) dev_free(e, p, e->compute);
        release(e, t->dev_reserved);
    }
    delete t;
}

// -------------------------------------------------------------- diagnostics

tp_status tp_stats_get(tp_engine* e, tp_stats* s) {
    if (!e || !s) return fail(TP_E_INVALID, "tp_stats_get: NULL argument");
    memset(s, 0, sizeof(*s));
    s->h2d_bytes = e->h2d_bytes;
    s->d2h_bytes = e->d2h_bytes;
    s->batches = e->batches;
    s->kernel_launches = e->launches;
    s->retries = e->retries;
    s->jit_compiles = e->jit_compiles;
    s->jit_failures = e->jit_failures;
    s->jit_launches = e->jit_launches;
    s->jit_compile_ms = (double)e->jit_us.load() / 1000.0;
    s->agg_split_passes = e->split_passes;
    s->lip_filters = e->lip_filters;
    {
        std::lock_guard<std::mutex> lk(e->time_mu);
        s->agg_kernel_ms = e->agg_ms;
        s->part_build_ms = e->part_ms[0];
        s->part_stream_ms = e->part_ms[1];
        s->part_spilled_ms = e->part_ms[2];
        s->agg_kernel_launches = e->agg_launches;
        s->agg_kernel_rows = e->agg_rows;
    }
    {
        std::lock_guard<std::mutex> lk(e->budget.mu);
        s->peak_reserved = e->budget.peak;
    }
    std::lock_guard<std::mutex> lk(e->pool.mu);
    s->pages_total = e->pool.n_pages;
    s->pages_in_use = e->pool.n_pages - (uint32_t)e->pool.free_stack.size();
    return TP_OK;
}

tp_status tp_debug_pack_bits(const uint64_t* values, uint64_t n, int32_t bits, uint32_t* words) {
    clear_error();
    if (bits < 1 || bits > 31 || (n && (!values || !words)))
        return fail(TP_E_INVALID, "tp_debug_pack_bits: bad arguments");
    for (uint64_t i = 0; i < n; ++i)
        if (values[i] >> bits) return fail(TP_E_INVALID, "tp_debug_pack_bits: value %llu needs more than %d bits",
                                           (unsigned long long)values[i], bits);
    std::fill(words, words + (n * (uint64_t)bits + 31) / 32, 0u);
    pack_bits(values, n, bits, words);
    return TP_OK;
}

tp_status tp_debug_fail_next_alloc(tp_engine* e, int32_t n) {
    if (!e || n < 0) return fail(TP_E_INVALID, "tp_debug_fail_next_alloc: bad argument");
    {
        std::lock_guard<std::mutex> lk(e->pool.mu);
        e->pool.fail_next = n;
    }
    std::lock_guard<std::mutex> lk(e->budget.mu);
    e->budget.fail_next = n;
    return TP_OK;
}

}  // extern "C"
