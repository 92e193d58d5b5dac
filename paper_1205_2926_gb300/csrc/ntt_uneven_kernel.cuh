// ntt_uneven_kernel.cuh -- the device side of the uneven batch: task,
// stage and work-item records, and the persistent kernel k_uneven<VAR> that
// runs them (lazy butterflies, Algorithms 3-4, or the NTL-style ones,
// Algorithm 2).  The host side (grouping, item order, launch) is
// ntt_uneven.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ntt_internal.hpp"
#include "ntt_kernels.cuh"

namespace ntt {

struct UStage {
    const uint32_t *ma, *mb;
    uint32_t units;  // CTA iterations (work items) of this stage
    uint32_t buf_chunks;
    int8_t logR, logS, logTV, logTA, row;
    uint8_t flags;
    uint16_t per_cta;
};

struct UTask {
    uint32_t *data;            // multi-pass task: the transform
    uint32_t *const *rowptrs;  // class task: one row address per transform
    const uint32_t *tw;
    uint64_t nrows;            // class task: number of transforms
    uint32_t p;
    uint32_t done_base;        // first completion counter of this task
    int8_t logL, nstages, dir;
    UStage st[kMaxPasses];
};

struct UItem {
    uint32_t task;
    uint32_t stage;
    uint32_t cta;  // CTA index within the stage
};

struct UCtl {
    unsigned int next;       // next item to take
    int status;              // NTT_OK or NTT_ERR_TIMEOUT
    int abort;               // set on timeout: every CTA stops
    unsigned int pad;
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *(volatile const int *)p; }

// Run-time dispatch on log2 R of a stage: run the rounds of one tile (the
// first round loads its words straight from global memory, the last stores
// them back).
template <int VAR, int DIR, bool ROW, int LO, int HI>
__device__ __forceinline__ void run_logr(int logR, const PassArgs<uint32_t> &a, uint32_t tile, uint4 *buf) {
    if (logR == LO) {
        tile_compute<uint32_t, DIR, VAR, LO, ROW>(a, tile, buf);
        return;
    }
    if constexpr (LO < HI) run_logr<VAR, DIR, ROW, LO + 1, HI>(logR, a, tile, buf);
}

__device__ __forceinline__ PassArgs<uint32_t> item_args(const UTask &t, const UStage &sg) {
    PassArgs<uint32_t> a;
    a.data = t.data;
    a.stride = 1ull << t.logL;
    a.batch = 1;
    a.logL = t.logL;
    a.logS = sg.logS;
    a.logTV = sg.logTV;
    a.logTA = sg.logTA;
    a.per_cta = sg.per_cta;
    a.ntiles = sg.units;
    a.buf_chunks = sg.buf_chunks;
    a.flags = sg.flags;
    a.tw = t.tw;
    a.ma = sg.ma;
    a.mb = sg.mb;
    a.p = t.p;
    a.J = 0;  // no Montgomery variant here
    a.rowptrs = t.rowptrs;
    a.nrows = t.rowptrs ? t.nrows : (1ull << (t.logL - sg.logR));
    return a;
}

// Run the rounds of a work item.
template <int VAR>
__device__ __forceinline__ void run_item(const UTask &t, const UStage &sg, uint32_t cta, uint4 *buf) {
    const PassArgs<uint32_t> a = item_args(t, sg);
    if (t.dir == DIR_FWD) {
        if (sg.row)
            run_logr<VAR, DIR_FWD, true, 3, kMaxRowLog>(sg.logR, a, cta, buf);
        else
            run_logr<VAR, DIR_FWD, false, 3, kMaxColLog>(sg.logR, a, cta, buf);
    } else {
        if (sg.row)
            run_logr<VAR, DIR_INV, true, 3, kMaxRowLog>(sg.logR, a, cta, buf);
        else
            run_logr<VAR, DIR_INV, false, 3, kMaxColLog>(sg.logR, a, cta, buf);
    }
}

// Completions item `it` needs before its tile may be read: every CTA
// iteration of the previous stage of its task.  A stall injected for testing
// asks for one completion more than will ever happen, so that the bounded
// wait must give up.
__device__ __forceinline__ const unsigned int *dep_counter(const UTask &t, const UItem &item, int stall_stage,
                                                           unsigned int *need, const unsigned int *done) {
    if (item.stage == 0) return nullptr;
    *need = t.st[item.stage - 1].units + (stall_stage == (int)item.stage ? 1u : 0u);
    return done + t.done_base + item.stage - 1;
}

// Persistent kernel over a queue of work items in dependency order.  Each
// CTA claims items with an atomic counter.  It claims its next item before
// computing the current one; when that item's dependencies are already met at
// claim time it starts on it right after, otherwise it waits for them
// (bounded) first.  Every item a CTA can wait for was claimed earlier and is
// processed before its owner blocks on a later one, so the queue always
// drains.  A wait that runs out of its budget sets NTT_ERR_TIMEOUT and the
// abort flag, and every CTA stops.  One tile buffer per CTA (32-bit tiles
// load their first round straight from global memory, so nothing is copied
// ahead) and 4 CTAs per SM: measured 14 % faster on the 4096-transform
// workload than two buffers at 3 CTAs per SM, although the 64-register budget
// spills (and 9 % faster than giving each pass shape its own non-inlined
// function, which spills less but passes its arguments through memory).
template <int VAR>
__global__ void __launch_bounds__(kThreads, 4) k_uneven(const UTask *__restrict__ tasks,
                                                         const UItem *__restrict__ items, uint32_t n_items,
                                                         unsigned int *done, UCtl *ctl, long long wait_budget,
                                                         int stall_stage) {
    extern __shared__ uint4 sm[];
    __shared__ unsigned int s_item;
    __shared__ int s_state;  // 1: dependencies met, 0: not yet, -1: stop
    // claim an item; with `block`, wait (bounded) until its dependencies are met
    auto claim = [&](bool block) -> unsigned int {
        if (threadIdx.x == 0) {
            const unsigned int it = ld_volatile(&ctl->abort) ? n_items : atomicAdd(&ctl->next, 1u);
            s_item = it;
            s_state = it >= n_items ? -1 : 1;
            if (it < n_items) {
                const UItem item = items[it];
                unsigned int need = 0;
                const unsigned int *cnt = dep_counter(tasks[item.task], item, stall_stage, &need, done);
                if (cnt && ld_acquire(cnt) < need) s_state = 0;
                if (s_state == 0 && block) {
                    const long long t0 = clock64();
                    while (ld_acquire(cnt) < need) {
                        if (ld_volatile(&ctl->abort) || clock64() - t0 > wait_budget) break;
                        __nanosleep(256);
                    }
                    if (ld_acquire(cnt) >= need) {
                        s_state = 1;
                    } else {
                        if (!ld_volatile(&ctl->abort)) atomicExch(&ctl->status, NTT_ERR_TIMEOUT);
                        atomicExch(&ctl->abort, 1);
                        s_state = -1;
                    }
                }
                __threadfence();
            }
        }
        __syncthreads();
        return s_item;
    };
    // the same wait for an item claimed earlier
    auto wait_ready = [&](unsigned int it) -> bool {
        if (threadIdx.x == 0) {
            const UItem item = items[it];
            unsigned int need = 0;
            const unsigned int *cnt = dep_counter(tasks[item.task], item, stall_stage, &need, done);
            s_state = 1;
            if (cnt) {
                const long long t0 = clock64();
                while (ld_acquire(cnt) < need) {
                    if (ld_volatile(&ctl->abort) || clock64() - t0 > wait_budget) break;
                    __nanosleep(256);
                }
                if (ld_acquire(cnt) < need) {
                    if (!ld_volatile(&ctl->abort)) atomicExch(&ctl->status, NTT_ERR_TIMEOUT);
                    atomicExch(&ctl->abort, 1);
                    s_state = -1;
                }
            }
            __threadfence();
        }
        __syncthreads();
        return s_state == 1;
    };
    unsigned int cur = claim(true);
    if (cur >= n_items || s_state != 1) return;
    for (;;) {
        const unsigned int nxt = claim(false);
        const bool have_next = nxt < n_items;
        const bool ready = have_next && s_state == 1;
        {
            const UItem item = items[cur];
            run_item<VAR>(tasks[item.task], tasks[item.task].st[item.stage], item.cta, sm);
        }
        __syncthreads();  // this item's last shared-memory reads before the next item's writes
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(done + tasks[items[cur].task].done_base + items[cur].stage, 1u);
        }
        if (!have_next) break;
        if (!ready && !wait_ready(nxt)) break;
        cur = nxt;
    }
}

// ----------------------------------------------------------------- host side

// The kernel of one butterfly variant, for the host side: its address (for
// attributes and occupancy) and a launcher.  Each variant is compiled in a
// translation unit of its own (ntt_uneven_<variant>.cu), in parallel.
using UnevenLaunchFn = cudaError_t (*)(unsigned grid, size_t smem, cudaStream_t st, const UTask *tasks,
                                       const UItem *items, uint32_t n_items, unsigned int *done, UCtl *ctl,
                                       long long wait_budget, int stall_stage);
struct UnevenKernel {
    const void *func;
    UnevenLaunchFn launch;
};

template <int VAR>
cudaError_t launch_uneven(unsigned grid, size_t smem, cudaStream_t st, const UTask *tasks, const UItem *items,
                          uint32_t n_items, unsigned int *done, UCtl *ctl, long long wait_budget, int stall_stage) {
    k_uneven<VAR><<<grid, kThreads, smem, st>>>(tasks, items, n_items, done, ctl, wait_budget, stall_stage);
    return cudaGetLastError();
}

template <int VAR>
UnevenKernel uneven_kernel();
template <>
UnevenKernel uneven_kernel<VAR_LAZY>();
template <>
UnevenKernel uneven_kernel<VAR_NTL>();

}  // namespace ntt
