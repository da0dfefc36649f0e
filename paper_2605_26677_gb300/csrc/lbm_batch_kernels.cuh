// lbm_batch_kernels.cuh -- batched step kernels: many lattices ("members",
// e.g. specimens of uneven size and material) advance one step in one
// persistent launch.
//
// The tasks of all members of a launch form one index space: member m owns
// global tasks [off[m], off[m+1]), off being the prefix sum of the members'
// (row, segment) task counts. A warp takes global task t (grid-stride, or
// claimed from a counter when the group runs in dynamic order), finds
// its member by binary search in off (copied to shared memory) and runs that
// member's task with that member's StepArgs, exactly the per-task code of the
// single-lattice kernel, so every member's populations evolve bit for bit as
// they would under its own launches. Status flags go to each member's own
// status word. The edge time factors are read through StepArgs::gdev, which
// the one-block kernel k_batch_time fills before each step.
#pragma once
#include "lbm_internal.h"
#include "lbm_step_core.cuh"

namespace tlv {

template <typename S, int LAW, int V, bool PACKED>
__device__ __forceinline__ void batch_loop(const BatchList &b, int *off, int *xq)
{
    using T = typename Prec<S>::R;
    constexpr bool XQ = !PACKED;  // side-edge rules deferred (unpacked kernels)
    for (int i = threadIdx.x; i <= b.n; i += blockDim.x) off[i] = b.off[i];
    __syncthreads();
    const StepArgs<T> *args = static_cast<const StepArgs<T> *>(b.args);
    const int lane = threadIdx.x & 31;
    const int ntask = off[b.n];
    XQueue q = XQ ? xq_make(xq) : XQueue{nullptr, nullptr, nullptr, 0};
    auto proc = [&](int x, int y, int mm) {
        const StepArgs<T> &a = args[mm];
        unsigned f = 0;
        xedge_node<LAW, S>(a, x, y, f);
        if (f) atomicOr(a.status, (int)f);
    };
    int m = 0;
    auto run = [&](int task) {
        // a warp's tasks grow except when it wraps from the last stripe to
        // the first (dynamic order): search from its member index onwards,
        // or from the start after a wrap
        int lo = (task >= off[m]) ? m : 0, hi = b.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= task)
                lo = mid;
            else
                hi = mid - 1;
        }
        m = lo;
        const StepArgs<T> &a = args[m];
        unsigned flags = 0;
        XPend xp{-1, 0};
        if constexpr (PACKED)
            step16_task<S, LAW, V, true>(a, task - off[m], lane, flags);
        else
            step_task<S, LAW, V, true, false, false, XQ>(a, task - off[m], lane, flags, &xp);
        flags = __reduce_or_sync(FULL_MASK, flags);
        if (flags && lane == 0) atomicOr(a.status, (int)flags);
        if constexpr (XQ) xq_push(q, xp, m, lane, proc);
    };
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b.ctr) {
        // dynamic: claim_tasks on the group's counters; the last block to
        // finish zeroes them for the next launch (every claim of the launch
        // has returned by then)
        claim_tasks<DYN_STRIPES>(b.ctr, ntask, lane, run);
        if constexpr (XQ)
            while (q.n > 0) xq_flush(q, lane, proc);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            unsigned *done = b.ctr + DYN_STRIPES * DYN_CTR_STRIDE;
            if (atomicAdd(done, 1u) == gridDim.x - 1) {
                for (int j = 0; j < DYN_STRIPES; ++j) b.ctr[j * DYN_CTR_STRIDE] = 0u;
                *done = 0u;
            }
        }
    } else {
        const int nw = gridDim.x * (blockDim.x >> 5);
        for (int task = gw; task < ntask; task += nw) run(task);
        if constexpr (XQ)
            while (q.n > 0) xq_flush(q, lane, proc);
    }
}

// unpacked vectors of V nodes (every storage type)
template <typename S, int LAW, int V>
__global__ void __launch_bounds__(128) k_batch(const BatchList b)
{
    extern __shared__ int off[];
    __shared__ int xq[4 * 3 * XQ_CAP];  // four warps' side-edge queues
    batch_loop<S, LAW, V, false>(b, off, xq);
}

// packed 16-bit vectors of 4 nodes (the single-lattice 16-bit kernel's form)
template <typename S, int LAW>
__global__ void __launch_bounds__(128, 3) k_batch16(const BatchList b)
{
    extern __shared__ int off[];
    batch_loop<S, LAW, 4, true>(b, off, nullptr);
}

// nodes per lane that the batched kernels are built for
template <typename S>
constexpr bool batch_vec_built(int vec)
{
    return sizeof(S) == 8 ? (vec == 1 || vec == 2) : sizeof(S) == 4 ? (vec == 1 || vec == 2 || vec == 4)
                                                                    : (vec == 2 || vec == 4);
}

template <typename S, int LAW>
const void *batch_kernel_law(int vec)
{
    if constexpr (sizeof(S) == 2) {
        if (vec == 4) return (const void *)k_batch16<S, LAW>;
        return (const void *)k_batch<S, LAW, 2>;
    } else if constexpr (sizeof(S) == 8) {
        if (vec == 1) return (const void *)k_batch<S, LAW, 1>;
        return (const void *)k_batch<S, LAW, 2>;
    } else {
        if (vec == 1) return (const void *)k_batch<S, LAW, 1>;
        if (vec == 2) return (const void *)k_batch<S, LAW, 2>;
        return (const void *)k_batch<S, LAW, 4>;
    }
}

// the kernel for (law, vec), or nullptr if it is not built
template <typename S>
const void *batch_kernel(int law, int vec)
{
    if (!batch_vec_built<S>(vec)) return nullptr;
    switch (law) {
    case LAW_SVK: return batch_kernel_law<S, LAW_SVK>(vec);
    case LAW_NH: return batch_kernel_law<S, LAW_NH>(vec);
    case LAW_LOGNH: return batch_kernel_law<S, LAW_LOGNH>(vec);
    case LAW_MR: return batch_kernel_law<S, LAW_MR>(vec);
    case LAW_YEOH: return batch_kernel_law<S, LAW_YEOH>(vec);
    case LAW_GENT: return batch_kernel_law<S, LAW_GENT>(vec);
    default: return nullptr;
    }
}

} // namespace tlv
