// lbm_step16_staged.cuh -- the 16-bit storage step kernel with its rows
// staged in shared memory by bulk asynchronous copies, and the choice
// between it and the register kernel (k_step16 in lbm_step_kernels.cuh).
#pragma once
#include "lbm_internal.h"
#include "lbm_step_core.cuh"
#include "lbm_bulk.cuh"
#include "lbm_launch.cuh"
#include <cstdlib>
#include <cstring>

namespace tlv {

// ---------------------------------------------------------------- staged 16-bit step
// With four packed nodes per lane, a warp of the register kernel (k_step16)
// keeps half the bytes of an FP32 task in flight, and at its register count
// 16 warps per SM leave HBM latency exposed. This variant stages each task's
// rows in shared memory with bulk asynchronous copies: one lane per warp
// issues them and an mbarrier per stage counts their bytes. A warp waits for
// stage j, moves it to registers, re-arms the stage with its task j + NS and
// only then collides, so NS tasks of every warp are in flight while it
// computes. Same tasks (row, 128-node segment), same arithmetic and same
// results as the register kernel.
//
// NS = 1 ships: the stage is re-armed as soon as its rows are in registers,
// so one task per warp is in flight while the warp computes, at four blocks
// (16 warps) per SM within the SM's shared memory.
//
// Stage layout in 16-bit elements, segment columns [x0s, x0s + 128):
//   per component k: q = 0 of row y, columns [x0s - 8, x0s + 128) (the
//   8-column halo holds column x0s - 1 and keeps the copy 16-byte aligned);
//   q = 2 of row y, [x0s, x0s + 136); q = 1 of row y - 1 and q = 3 of row
//   y + 1, [x0s, x0s + 128); then u* of row y, [x0s, x0s + 128), two FP64
//   planes. A ragged last segment copies whole 16-byte units up to what its
//   nodes read (the ghost column nx and at most 7 columns of row padding
//   beyond); the rest of the stage keeps stale values that only lanes
//   without real nodes read, and their results are never stored.
template <int NS>
struct Stage16 {
    static constexpr int SW = 128, HALO = 8, WARPS = 4;
    static constexpr int L02 = SW + HALO, L13 = SW;
    static constexpr int KSTRIDE = 2 * L02 + 2 * L13;  // elements per component
    static constexpr int POP_BYTES = 6 * KSTRIDE * 2;
    static constexpr int BYTES = POP_BYTES + 2 * SW * 8;
    static constexpr int BAR_BYTES = 128;
    static constexpr int SMEM = BAR_BYTES + WARPS * NS * BYTES;
    static constexpr int MIN_BLOCKS = NS == 1 ? 4 : 3;
    static_assert(WARPS * NS * 8 <= BAR_BYTES, "barriers fit their slot");
    static_assert(POP_BYTES % 32 == 0 && BYTES % 32 == 0 && (2 * L02) % 16 == 0 && (2 * L13) % 16 == 0,
                  "16-byte copy destinations, 32-byte u* vectors");
};

// inject_stall != 0 (a test of the bounded wait, see stall_test_once): the
// first task of warp 0 expects 16 bytes more than its copies deliver, so its
// stage never completes and the wait runs out.
template <typename S, int LAW, int NS, bool FUSE>
__global__ void __launch_bounds__(128, Stage16<NS>::MIN_BLOCKS) k_step16s(const StepArgs<float> a, int inject_stall)
{
    using G = Stage16<NS>;
    constexpr int V = 4, W = 2, SW = G::SW;
    static_assert(V == STEP16_V, "same tasks as the register kernel");
    using WV = Words<W>;
    using PD = Pack<double, 4>;
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_enter();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * G::WARPS + wid, nw = gridDim.x * G::WARPS;
    const int nx = a.L.nx, ny = a.L.ny;
    const int nseg = (nx + SW - 1) / SW;
    const int ntask = ny * nseg;
    const long long plane = a.L.plane;
    const int pitch = a.L.pitch;
    const unsigned short *__restrict__ fin = static_cast<const unsigned short *>(a.fin);
    unsigned short *__restrict__ fout = static_cast<unsigned short *>(a.fout);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem) + wid * NS;
    unsigned char *stages = smem + G::BAR_BYTES + wid * NS * G::BYTES;
    unsigned flags = 0;

    // lane 0: copy task `task`'s rows into stage s
    auto issue = [&](int task, int s) {
        int y, seg;
        task_coords(task, nseg, ny, y, seg);
        const int x0s = seg * SW;
        const unsigned rem = (unsigned)min(SW, nx - x0s);
        const unsigned n1 = (rem + 7) & ~7u, n0 = G::HALO + n1, n2 = (rem + 8) & ~7u, nu = (rem + 1) & ~1u;
        uint64_t *b = bar + s;
        const unsigned phantom = (inject_stall && task == gw && gw == 0) ? 16u : 0u;
        mbar_expect(b, 12u * (n0 + n2 + 2u * n1) + 16u * nu + phantom);
        const long long row = (long long)(y + 1) * pitch + a.L.xoff + x0s;
        unsigned short *d = reinterpret_cast<unsigned short *>(stages + s * G::BYTES);
#pragma unroll 1
        for (int k = 0; k < 6; ++k, d += G::KSTRIDE) {
            bulk_load(d, fin + (0 * 6 + k) * plane + row - G::HALO, 2 * n0, b);
            bulk_load(d + G::L02, fin + (2 * 6 + k) * plane + row, 2 * n2, b);
            bulk_load(d + 2 * G::L02, fin + (1 * 6 + k) * plane + row - pitch, 2 * n1, b);
            bulk_load(d + 2 * G::L02 + G::L13, fin + (3 * 6 + k) * plane + row + pitch, 2 * n1, b);
        }
        double *du = reinterpret_cast<double *>(stages + s * G::BYTES + G::POP_BYTES);
        const long long urow = (long long)y * a.L.upitch + x0s;
        bulk_load(du, a.ustar + urow, 8 * nu, b);
        bulk_load(du + SW, a.ustar + a.L.uplane + urow, 8 * nu, b);
    };

    if (lane == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(bar + s);
        mbar_init_fence();
        fence_async_smem();
        for (int s = 0; s < NS; ++s)
            if (gw + s * nw < ntask) issue(gw + s * nw, s);
    }
    __syncwarp();

    int j = 0;
    for (int task = gw; task < ntask; task += nw, ++j) {
        const int s = j % NS;
        const bool landed = mbar_wait(bar + s, (unsigned)(j / NS) & 1u);
        if (__any_sync(FULL_MASK, !landed)) {
            // the copy engine did not deliver within the bound: report, wait
            // (bounded) for this warp's copies still in flight, stop
            flags |= ST_STALL;
            for (int i = 0; i < NS; ++i)
                if (task + i * nw < ntask) mbar_wait(bar + (j + i) % NS, (unsigned)((j + i) / NS) & 1u);
            break;
        }
        int y, seg;
        task_coords(task, nseg, ny, y, seg);
        const int x0 = seg * SW + lane * V;
        const bool act = x0 < nx;
        const long long row = (long long)(y + 1) * pitch + a.L.xoff + x0;

        WV w[4][6];
        const unsigned *sw = reinterpret_cast<const unsigned *>(stages + s * G::BYTES);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const unsigned *b0 = sw + k * (G::KSTRIDE / 2);
            const unsigned *b2 = b0 + G::L02 / 2, *b1 = b0 + G::L02, *b3 = b0 + G::L02 + G::L13 / 2;
            // +x (Eq. 15): node x0 + e pulls column x0 + e - 1, element 4 lane + 7 + e of its row
            const unsigned a3 = b0[2 * lane + 3];
            const uint2 a45 = *reinterpret_cast<const uint2 *>(b0 + 2 * lane + 4);
            w[0][k].w[0] = __funnelshift_r(a3, a45.x, 16);
            w[0][k].w[1] = __funnelshift_r(a45.x, a45.y, 16);
            // -x: column x0 + e + 1, element 4 lane + 1 + e
            const uint2 c01 = *reinterpret_cast<const uint2 *>(b2 + 2 * lane);
            const unsigned c2 = b2[2 * lane + 2];
            w[2][k].w[0] = __funnelshift_r(c01.x, c01.y, 16);
            w[2][k].w[1] = __funnelshift_r(c01.y, c2, 16);
            // +y and -y: rows y - 1 and y + 1, same columns
            const uint2 d1 = *reinterpret_cast<const uint2 *>(b1 + 2 * lane);
            const uint2 d3 = *reinterpret_cast<const uint2 *>(b3 + 2 * lane);
            w[1][k].w[0] = d1.x;
            w[1][k].w[1] = d1.y;
            w[3][k].w[0] = d3.x;
            w[3][k].w[1] = d3.y;
        }
        const double *su = reinterpret_cast<const double *>(stages + s * G::BYTES + G::POP_BYTES);
        PD u[2];
        u[0] = *reinterpret_cast<const PD *>(su + 4 * lane);
        u[1] = *reinterpret_cast<const PD *>(su + SW + 4 * lane);
        // every lane has read stage s: hand it to the copy engine for task j + NS
        __syncwarp();
        if (lane == 0 && task + NS * nw < ntask) {
            fence_async_smem();
            issue(task + NS * nw, s);
        }

        float vel[2][V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
            float fq[4][6];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 6; ++k) fq[q][k] = unpack16(w[q][k].w[e >> 1], e & 1, S());
            collide_node<LAW, float>(fq, a, LawP<float>{a.lam, a.mu, a.p2, a.p3}, x0 + e < nx, flags, vel[0][e],
                                     vel[1][e]);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    unsigned &ww = w[q][k].w[e >> 1];
                    const unsigned b = bits16<S>(fq[q][k]);
                    ww = (e & 1) ? __byte_perm(ww, b, 0x5410) : __byte_perm(ww, b, 0x3254);
                }
        }

        if (act) {
            const bool full = x0 + V <= nx;
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    unsigned short *dst = fout + (q * 6 + k) * plane + row;
                    if (full) {
                        *reinterpret_cast<uint2 *>(dst) = make_uint2(w[q][k].w[0], w[q][k].w[1]);
                    } else {
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            const unsigned ww = w[q][k].w[e >> 1];
                            if (x0 + e < nx) dst[e] = (unsigned short)((e & 1) ? (ww >> 16) : (ww & 0xffffu));
                        }
                    }
                }
            // Eq. (22): u*^{n+1} = u*^n + dt v^n
            const long long urow = (long long)y * a.L.upitch + x0;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
#pragma unroll
                for (int e = 0; e < V; ++e) u[c].v[e] += a.dt * (double)vel[c][e];
                *reinterpret_cast<PD *>(a.ustar + c * a.L.uplane + urow) = u[c];
            }
            if (FUSE) lane_ghosts<LAW, S, V>(a, reinterpret_cast<S *>(fout), row, x0, y, flags);
        }
    }
    flags = __reduce_or_sync(FULL_MASK, flags);
    if (flags && lane == 0) atomicOr(a.status, (int)flags);
}

// Which 16-bit step kernel runs: LBM_STEP16 in the environment when set
// (step16_env_choice), else the context's own choice (StepArgs::k16), which
// the first lbm_step makes by timing both on the lattice. The register
// kernel is the faster one on most lattices measured (BF16 us per step,
// register / staged: 2048^2 periodic 98.9 / 105.4, 8192^2 periodic 1405 /
// 1586), the staged one on some (4096 x 2048 clamped 190.5 / 187.0).
static int step16_stages(int ctx_choice)
{
    const int e = step16_env_choice();
    return (e >= 0 ? e : ctx_choice) == 1 ? 1 : 0;
}

// The staged kernel's dynamic shared memory exceeds the 48 KB default: raise
// its limit once per device before its first occupancy query or launch.
template <typename S, int LAW, int NS, bool FUSE>
static cudaError_t step16s_prepare()
{
    static unsigned long long done = 0;  // one bit per device ordinal < 64
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (__atomic_load_n(&done, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(k_step16s<S, LAW, NS, FUSE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Stage16<NS>::SMEM);
    if (e == cudaSuccess) __atomic_fetch_or(&done, bit, __ATOMIC_ACQ_REL);
    return e;
}

// Test of the staged kernel's bounded wait: with LBM_STEP16_STALL_TEST=1 in
// the environment, the first staged launch of the process makes one warp's
// wait run out (about two seconds; the step then reports LBM_ERR_CUDA and its
// result is not valid). Every later launch runs normally.
static int stall_test_once()
{
    static const bool on = [] {
        const char *v = std::getenv("LBM_STEP16_STALL_TEST");
        return v && !std::strcmp(v, "1");
    }();
    static int used = 0;
    return on && __atomic_exchange_n(&used, 1, __ATOMIC_ACQ_REL) == 0 ? 1 : 0;
}

template <typename S, int LAW, int NS, bool FUSE>
static cudaError_t launch_step16s(const StepArgs<float> &a, int grid, cudaStream_t st)
{
    const cudaError_t e = step16s_prepare<S, LAW, NS, FUSE>();
    if (e != cudaSuccess) return e;
    return launch_pdl(k_step16s<S, LAW, NS, FUSE>, grid, 128, (size_t)Stage16<NS>::SMEM, st, a, stall_test_once());
}

// Launches the staged kernel when it is the selected one (true, status in
// err); false when the register kernel is to run.
template <typename S, int LAW>
static bool launch_step16_staged(const StepArgs<float> &a, bool fuse, int grid, cudaStream_t st, cudaError_t &err)
{
    if (step16_stages(a.k16) != 1) return false;
    err = fuse ? launch_step16s<S, LAW, 1, true>(a, grid, st) : launch_step16s<S, LAW, 1, false>(a, grid, st);
    return true;
}

// Resident blocks per SM of the staged kernel (fused form) in n, status in
// err. The grid is sized once for both 16-bit kernels, which either may run.
template <typename S, int LAW>
static cudaError_t step16_staged_blocks(int &n)
{
    cudaError_t err = step16s_prepare<S, LAW, 1, true>();
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step16s<S, LAW, 1, true>, 128, Stage16<1>::SMEM);
    return err;
}

} // namespace tlv
