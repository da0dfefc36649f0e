// lbm_step_kernels.cuh -- the single-lattice step kernels (fused collide-
// stream, Sec. 3.7) and the node-form ghost refresh, as templates over the
// storage type and closure, with per-storage launch helpers. Each storage
// type is instantiated in its own translation unit (lbm_step_<type>.cu).
#pragma once
#include "lbm_internal.h"
#include "lbm_step_core.cuh"
#include "lbm_step16_staged.cuh"
#include "lbm_launch.cuh"

namespace tlv {
// Task order of the persistent step kernels. Static: warp w takes tasks w,
// w + W, w + 2W, ... Dynamic (DYN): warps claim tasks from counters in device
// memory (claim_tasks; the 16-bit kernels over one stripe or DYN_STRIPES, the
// others over DYN_STRIPES). Each launch uses one of two counter sets and zeroes
// the other, which the next launch in the stream uses; a launch starts only
// after the previous one has completed (griddepcontrol.wait), so every
// counter is zero when its launch begins.
template <int NS, typename Fn>
__device__ __forceinline__ void dyn_tasks(unsigned *ctr, unsigned *ctr_next, int ntask, int lane, Fn &&run)
{
    // all DYN_STRIPES counters of the next set, whatever NS: the launches of
    // a context may alternate between stripe counts
    if (blockIdx.x == 0 && threadIdx.x < DYN_STRIPES) ctr_next[threadIdx.x * DYN_CTR_STRIDE] = 0u;
    claim_tasks<NS>(ctr, ntask, lane, run);
}

template <typename S, int LAW, int VEC, bool FUSE, bool MATF = false, bool NOQ = false, bool DYN = false>
__global__ void __launch_bounds__(128) k_step(const StepArgs<typename Prec<S>::R> a)
{
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int ntask = a.L.ny * ((a.L.nx + 32 * VEC - 1) / (32 * VEC));  // < 2^31 (checked at creation)
    unsigned flags = 0;
    // FP64 with fused ghost writes: the side-edge rules go through the
    // warp's queue (FP64 specimen 5,050 -> 5,133 MLUPS). The FP32 kernels,
    // bound by memory, keep the inline rule: with the queue the clamped
    // specimen went 0.979 -> 0.976 and the 8192^2 lattice 1.009 -> 1.007.
    constexpr bool XQ = FUSE && sizeof(S) == 8;
    __shared__ int xq[XQ ? 4 * 3 * XQ_CAP : 1];
    XQueue q = XQ ? xq_make(xq) : XQueue{nullptr, nullptr, nullptr, 0};
    auto proc = [&](int x, int y, int) { xedge_node<LAW, S, MATF>(a, x, y, flags); };
    auto run = [&](int task) {
        XPend xp{-1, 0};
        step_task<S, LAW, VEC, FUSE, MATF, NOQ, XQ>(a, task, lane, flags, &xp);
        if constexpr (XQ) xq_push(q, xp, 0, lane, proc);
    };
    if constexpr (DYN)
        dyn_tasks<DYN_STRIPES>(a.ctr, a.ctr_next, ntask, lane, run);
    else
        for (int task = gw; task < ntask; task += nw) run(task);
    if constexpr (XQ)
        while (q.n > 0) xq_flush(q, lane, proc);
    flags = __reduce_or_sync(FULL_MASK, flags);
    if (flags && lane == 0) atomicOr(a.status, (int)flags);
}

// DYN: 0 static order, else dynamic claims over DYN stripes (1 or DYN_STRIPES)
template <typename S, int LAW, int V, bool FUSE, bool MATF = false, int DYN = 0>
__global__ void __launch_bounds__(128, 4) k_step16(const StepArgs<float> a)
{
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int ntask = a.L.ny * ((a.L.nx + 32 * V - 1) / (32 * V));
    unsigned flags = 0;
    if constexpr (DYN > 0)
        dyn_tasks<DYN>(a.ctr, a.ctr_next, ntask, lane,
                       [&](int task) { step16_task<S, LAW, V, FUSE, MATF>(a, task, lane, flags); });
    else
        for (int task = gw; task < ntask; task += nw) step16_task<S, LAW, V, FUSE, MATF>(a, task, lane, flags);
    flags = __reduce_or_sync(FULL_MASK, flags);
    if (flags && lane == 0) atomicOr(a.status, (int)flags);
}

// Ghost refresh in the node form (after initialization, a checkpoint load or
// new edge data): the same values the fused step writes, from the stored
// post-collision populations of the current buffer.
template <typename S, int LAW>
__global__ void __launch_bounds__(128) k_ghosts(const EdgeArgs a)
{
    using T = typename Prec<S>::R;
    S *f = static_cast<S *>(a.f);
    int e = 0;
    while (e < 3 && (int)blockIdx.x >= a.blk_end[e]) ++e;
    const int b0 = e ? a.blk_end[e - 1] : 0;
    const int s = ((int)blockIdx.x - b0) * blockDim.x + threadIdx.x;
    const int len = (e <= EDGE_RIGHT) ? a.L.ny : a.L.nx;
    if (s >= len) return;
    auto idx = [&](int q, int k, int x, int y) {
        return (long long)(q * 6 + k) * a.L.plane + (long long)(y + 1) * a.L.pitch + a.L.xoff + x;
    };
    int xb, yb, gx, gy;
    switch (e) {
    case EDGE_LEFT: xb = 0; yb = s; gx = -1; gy = s; break;
    case EDGE_RIGHT: xb = a.L.nx - 1; yb = s; gx = a.L.nx; gy = s; break;
    case EDGE_BOTTOM: xb = s; yb = 0; gx = s; gy = -1; break;
    default: xb = s; yb = a.L.ny - 1; gx = s; gy = a.L.ny; break;
    }
    const int d = edge_dmiss(e), md = edge_dout(e);
    const EdgeDesc &E = a.e[e];
    if (E.kind == BC_PERIODIC) {
        const int sx = (e == EDGE_LEFT) ? a.L.nx - 1 : (e == EDGE_RIGHT) ? 0 : s;
        const int sy = (e == EDGE_BOTTOM) ? a.L.ny - 1 : (e == EDGE_TOP) ? 0 : s;
#pragma unroll
        for (int k = 0; k < 6; ++k) f[idx(d, k, gx, gy)] = f[idx(d, k, sx, sy)];
        return;
    }
    T fq[4][6], U[6], fo[6], out[6];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 6; ++k) fq[q][k] = ld_r(f[idx(q, k, xb, yb)]);
    state_from_fstar(fq[0], fq[1], fq[2], fq[3], (T)a.hdtb1, (T)a.hdtb2, U);
#pragma unroll
    for (int k = 0; k < 6; ++k) fo[k] = fq[md][k];
    double val[2];
    edge_value(E, s, a.g[e], val);
    unsigned flags = 0;
    const LawP<T> m = law_cast<T>(law_at(a.m, (long long)yb * a.L.nx + xb));
    edge_ghost<LAW, T>(e, E.kind, fo, U, val, (T)a.c, m, out, flags);
    if (flags) atomicOr(a.status, (int)flags);
#pragma unroll
    for (int k = 0; k < 6; ++k) f[idx(d, k, gx, gy)] = to_store<S>(out[k]);
}

// ---------------------------------------------------------------- launchers
// One launch of the register step kernel with its variant fixed at compile
// time: fused ghost writes, per-node material (MATF), no u* update (NOQ:
// the adjoint's recomputed steps), and the task order (NS = 0 static, else
// dynamic claims over NS stripes).
template <typename S, int LAW, bool MATF, bool NOQ, int NS>
static cudaError_t launch_step_v(const StepArgs<typename Prec<S>::R> &a, bool fuse, int grid, cudaStream_t st)
{
    if constexpr (sizeof(S) == 2) {
        static_assert(!NOQ, "the 16-bit kernels always update u*");
        return fuse ? launch_pdl(k_step16<S, LAW, STEP16_V, true, MATF, NS>, grid, 128, 0, st, a)
                    : launch_pdl(k_step16<S, LAW, STEP16_V, false, MATF, NS>, grid, 128, 0, st, a);
    } else {
        static_assert(NS == 0 || NS == DYN_STRIPES, "FP32 and FP64 kernels claim over DYN_STRIPES stripes");
        constexpr int VEC = 16 / sizeof(S);  // 16-byte vectors (unpacked kernels)
        return fuse ? launch_pdl(k_step<S, LAW, VEC, true, MATF, NOQ, NS != 0>, grid, 128, 0, st, a)
                    : launch_pdl(k_step<S, LAW, VEC, false, MATF, NOQ, NS != 0>, grid, 128, 0, st, a);
    }
}

template <typename S, int LAW, bool MATF, bool NOQ>
static cudaError_t launch_step_o(const StepArgs<typename Prec<S>::R> &a, bool fuse, int grid, cudaStream_t st)
{
    if (!a.ctr2) return launch_step_v<S, LAW, MATF, NOQ, 0>(a, fuse, grid, st);
    // dynamic task claims: this launch takes the counter set the previous
    // dynamic launch zeroed (only dynamic launches touch the sets)
    StepArgs<typename Prec<S>::R> d = a;
    d.ctr = a.ctr2 + *a.ctr_par * DYN_SET_WORDS;
    d.ctr_next = a.ctr2 + (*a.ctr_par ^ 1) * DYN_SET_WORDS;
    *a.ctr_par ^= 1;
    if constexpr (sizeof(S) == 2)
        if (a.dyn_ns == 1) return launch_step_v<S, LAW, MATF, NOQ, 1>(d, fuse, grid, st);
    return launch_step_v<S, LAW, MATF, NOQ, DYN_STRIPES>(d, fuse, grid, st);
}

template <typename S, int LAW>
static cudaError_t launch_step_t(const StepArgs<typename Prec<S>::R> &a, bool fuse, int grid, cudaStream_t st)
{
    if (a.mufield) {
        // per-node material: SVK / NH / log-NH; the 16-bit formats on the register kernel
        if constexpr (LAW > LAW_LOGNH) {
            return cudaErrorNotSupported;
        } else if constexpr (sizeof(S) == 2) {
            if (!a.ustar) return cudaErrorInvalidValue;
            return launch_step_o<S, LAW, true, false>(a, fuse, grid, st);
        } else {
            // without u*: a step recomputed only for its populations (the
            // adjoint's checkpoint segments), 32 bytes per node less
            if (!a.ustar) return launch_step_o<S, LAW, true, true>(a, fuse, grid, st);
            return launch_step_o<S, LAW, true, false>(a, fuse, grid, st);
        }
    }
    if constexpr (sizeof(S) == 2) {
        cudaError_t e;
        if (launch_step16_staged<S, LAW>(a, fuse, grid, st, e)) return e;
    }
    return launch_step_o<S, LAW, false, false>(a, fuse, grid, st);
}

template <typename S>
static cudaError_t launch_step_s(int law, const void *args, bool fuse, int grid, cudaStream_t st)
{
    const auto &a = *static_cast<const StepArgs<typename Prec<S>::R> *>(args);
    switch (law) {
    case LAW_SVK: return launch_step_t<S, LAW_SVK>(a, fuse, grid, st);
    case LAW_NH: return launch_step_t<S, LAW_NH>(a, fuse, grid, st);
    case LAW_LOGNH: return launch_step_t<S, LAW_LOGNH>(a, fuse, grid, st);
    case LAW_MR: return launch_step_t<S, LAW_MR>(a, fuse, grid, st);
    case LAW_YEOH: return launch_step_t<S, LAW_YEOH>(a, fuse, grid, st);
    default: return launch_step_t<S, LAW_GENT>(a, fuse, grid, st);
    }
}

template <typename S>
static cudaError_t launch_ghosts_s(const EdgeArgs &a, int grid, cudaStream_t st)
{
    switch (a.m.law) {
    case LAW_SVK: k_ghosts<S, LAW_SVK><<<grid, 128, 0, st>>>(a); break;
    case LAW_NH: k_ghosts<S, LAW_NH><<<grid, 128, 0, st>>>(a); break;
    case LAW_LOGNH: k_ghosts<S, LAW_LOGNH><<<grid, 128, 0, st>>>(a); break;
    case LAW_MR: k_ghosts<S, LAW_MR><<<grid, 128, 0, st>>>(a); break;
    case LAW_YEOH: k_ghosts<S, LAW_YEOH><<<grid, 128, 0, st>>>(a); break;
    default: k_ghosts<S, LAW_GENT><<<grid, 128, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

// resident blocks per SM of the step kernel that will run (fused form)
template <typename S, int LAW>
static int step_blocks_t()
{
    int n = 0;
    cudaError_t e = cudaSuccess;
    if constexpr (sizeof(S) == 2) {
        int ns = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step16<S, LAW, STEP16_V, true>, 128, 0);
        if (e == cudaSuccess) e = step16_staged_blocks<S, LAW>(ns);
        if (e == cudaSuccess && ns < n) n = ns;
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<S, LAW, 16 / sizeof(S), true>, 128, 0);
    }
    return e == cudaSuccess ? n : 0;
}

template <typename S>
static int step_blocks_s(int law)
{
    switch (law) {
    case LAW_SVK: return step_blocks_t<S, LAW_SVK>();
    case LAW_NH: return step_blocks_t<S, LAW_NH>();
    case LAW_LOGNH: return step_blocks_t<S, LAW_LOGNH>();
    case LAW_MR: return step_blocks_t<S, LAW_MR>();
    case LAW_YEOH: return step_blocks_t<S, LAW_YEOH>();
    default: return step_blocks_t<S, LAW_GENT>();
    }
}

// per-storage entry points, defined in lbm_step_<type>.cu
#define TLV_STEP_ENTRY_POINTS(NAME, S)                                                                         \
    cudaError_t launch_step_##NAME(int law, const void *args, bool fuse, int grid, cudaStream_t st)           \
    {                                                                                                        \
        return launch_step_s<S>(law, args, fuse, grid, st);                                                  \
    }                                                                                                        \
    cudaError_t launch_ghosts_##NAME(const EdgeArgs &a, int grid, cudaStream_t st)                           \
    {                                                                                                        \
        return launch_ghosts_s<S>(a, grid, st);                                                              \
    }                                                                                                        \
    int step_blocks_##NAME(int law) { return step_blocks_s<S>(law); }

} // namespace tlv
