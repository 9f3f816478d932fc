// Batched execution with plan-specialised probe tasks, compiled at run time.
//
// Paper basis: Section 3.1 (operators spawn tasks over batches; tasks run on
// the GPU asynchronously), Section 3.3.1 (the compute executor drains a task
// queue).  The queue, its task order (build chunks, probe tiles, one
// finalisation per query) and its bounded dependency waits are those of the
// ahead-of-time batch kernel; what differs is the probe task: each query
// carries a shape id, and the task runs the row evaluation compiled for that
// shape (jit_common.cuh), reading the query's columns in device memory
// directly (lane l of a warp takes rows l and l + 32 of each 64-row block, so
// every load is coalesced), every column of a block loaded up front.
//
// The host prepends the shape structs JS_0, JS_1, ... and appends the
// definition of dispatch_probe: a switch on the shape id calling
// probe_tile<JS_id>.
#pragma once
// build tasks write the join tables earlier in the same launch
#define TP_TABLES_BUILT_IN_LAUNCH 1
#include "jit_common.cuh"

namespace tpj {

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0 waits until *ctr reaches want (bounded by wait_ns); the CTA learns
// the outcome.
__device__ __forceinline__ bool wait_count(unsigned* ctr, unsigned want, uint64_t wait_ns, uint32_t* err, int* flag) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint64_t t0 = now_ns();
        while (*(volatile unsigned*)ctr < want) {
            if (now_ns() - t0 > wait_ns) {
                atomicOr(err, ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(256);
        }
        __threadfence();
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

// Adds sum I (and the following ones) of group gi of a fast shared-memory
// table to the query's accumulators: carry words * 2^32 + low words + count *
// offset.
template <class S, int I>
__device__ __forceinline__ void flush_sums(const BatchQuery& B, const uint32_t* cnt, uint32_t G, uint32_t gi,
                                           uint64_t c) {
    if constexpr (I < S::ns) {
        const uint32_t* w = cnt + (uint64_t)sum_word<S, I>() * G;
        uint64_t v = w[gi];
        if constexpr (S::mode[I] == 2) v += (uint64_t)w[G + gi] << 32;
        v += c * (uint64_t)B.sum_off[I];
        atomicAdd((unsigned long long*)&B.acc[(uint64_t)G * (1 + 2 * I) + gi], (unsigned long long)v);
        flush_sums<S, I + 1>(B, cnt, G, gi, c);
    }
}

// Probe tile [r0, r1) of query B with shape S.  fast shapes accumulate into a
// 32-bit table in shared memory (the layout of the ahead-of-time kernel:
// counts, then per sum its mode's blocks) folded into B.acc at the end; the
// others add straight into B.acc (64-bit low words when S::lo_only, else
// exact 128-bit).
template <class S>
__device__ __forceinline__ void probe_tile(const BatchQuery& B, uint64_t r0, uint64_t r1, unsigned char* smem) {
    const QueryDev& q = B.q;
    const uint32_t G = 1u << B.key_bits;
    Tab t{};
    t.G = G;
    t.sum_off = B.sum_off;
    if constexpr (S::fast) {
        t.base = smem;
        constexpr uint32_t words = sum_word<S, S::ns>();
        for (uint32_t i = threadIdx.x; i < words * G; i += blockDim.x) ((uint32_t*)smem)[i] = 0;
        __syncthreads();
    } else {
        t.base = (unsigned char*)B.acc;
    }
    const Flt flt = make_flt(q);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    constexpr uint32_t SUB = 32u * ST_RPL;
    for (uint64_t base = r0 + (uint64_t)warp * SUB; base < r1; base += (uint64_t)nwarps * SUB) {
        const uint64_t left = r1 - base;
        uint32_t valid = 0;
#pragma unroll
        for (int j = 0; j < ST_RPL; ++j) valid |= (uint32_t)((uint64_t)lane + 32 * j < left) << j;
        // all of the shape's columns for these rows in flight at once
        Eager<S> ev;
        ev.template fill<0>(query_cols<S>(q, base), (uint32_t)lane, valid);
        consume<S>(q, flt, t, ev, (uint32_t)lane, valid);
    }
    if constexpr (S::fast) {
        __syncthreads();
        const uint32_t* cnt = (const uint32_t*)smem;
        for (uint32_t gi = threadIdx.x; gi < G; gi += blockDim.x) {
            const uint64_t c = cnt[gi];
            if (!c) continue;
            atomicAdd((unsigned long long*)&B.acc[gi], (unsigned long long)c);
            flush_sums<S, 0>(B, cnt, G, gi, c);
        }
    }
}

// Defined after this header by the host: probe_tile<JS_id> for B.shape.
__device__ void dispatch_probe(const BatchQuery& B, uint64_t r0, uint64_t r1, unsigned char* smem);

}  // namespace tpj

extern "C" __global__ void __launch_bounds__(tpk::BATCH_THREADS)
    tpj_batch(const tpk::BatchQuery* __restrict__ qs, const tpk::BatchItem* __restrict__ items, uint32_t n_items,
              uint32_t n_q, unsigned* ctr, uint32_t* err, const uint64_t* __restrict__ wait) {
    using namespace tpk;
    using namespace tpj;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t cur;
    __shared__ int flag;
    __shared__ uint64_t first_row;
    const uint64_t wait_ns = *wait;
    unsigned* build_done = ctr + 1;
    unsigned* probe_done = ctr + 1 + n_q;
    for (;;) {
        if (threadIdx.x == 0) cur = atomicAdd(ctr, 1u);
        __syncthreads();
        const uint32_t i = cur;
        __syncthreads();
        if (i >= n_items) return;
        const BatchItem it = items[i];
        const BatchQuery& B = qs[it.q];
        const uint64_t t_claim = B.task_ns ? now_ns() : 0;
        if (it.kind == BI_BUILD) {
            for (uint64_t r = it.r0 + threadIdx.x; r < it.r1; r += blockDim.x) build_insert(B.b, r);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&build_done[it.q], 1u);
            }
        } else if (it.kind == BI_PROBE) {
            if (B.q.has_join && !wait_count(&build_done[it.q], B.build_items, wait_ns, err, &flag)) continue;
            dispatch_probe(B, it.r0, it.r1, smem);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&probe_done[it.q], 1u);
            }
        } else {
            if (!wait_count(&probe_done[it.q], B.probe_items, wait_ns, err, &flag)) continue;
            // groups [r0, r1): count them, wait for the ranges before to publish
            // where their rows end, publish this range's end, write the rows
            const uint32_t G = 1u << B.key_bits;
            const uint32_t g0 = (uint32_t)it.r0, g1 = (uint32_t)it.r1, k = g0 / FINAL_CHUNK;
            const uint32_t cnt = dense_range_count(B.acc, g0, g1);
            if (!wait_count(B.final_done, k, wait_ns, err, &flag)) continue;
            if (threadIdx.x == 0) {
                const uint64_t first = k ? *(volatile unsigned long long*)B.final_end : 0ull;
                first_row = first;
                *(volatile unsigned long long*)B.final_end = first + cnt;
                __threadfence();
                atomicAdd(B.final_done, 1u);
                if (g1 == G) *B.out.n_groups = first + cnt;
            }
            __syncthreads();
            dense_range_emit(B.acc, G, g0, g1, B.q.n_sum, B.out, B.fast != 0, first_row);
        }
        __syncthreads();
        if (B.task_ns && threadIdx.x == 0) atomicAdd(B.task_ns, (unsigned long long)(now_ns() - t_claim));
    }
}
