// lbm_step.cu -- the per-step kernels of the TL vectorial D2Q4x6 LBM.
//
// One time step (Sec. 3.7) is two launches on the context's stream:
//   1. k_edges: for every edge node, the population that node will pull from
//      outside the domain is written into the ghost cell it pulls from:
//      periodic edges copy the opposite node's outgoing population; velocity
//      and traction edges apply the half-way rule f_d = D f*_{-d} + S_d(t +
//      dt/2) of Eqs. (23)-(25) (traction: Newton for F^b, Sec. 3.6.2).
//   2. k_step: fused pull-streaming + state recovery + P(F) + equilibrium +
//      BGK collision + displacement quadrature for every node, reading the
//      post-collision populations of step n-1 and writing those of step n.
// The stored state between steps is the post-collision f*^n, so streaming
// (Eq. 15) happens at the start of the next step as a pull.
#include "lbm_device.cuh"
#include "lbm_edges.cuh"
#include "lbm_internal.h"

namespace tlv {

template <typename T, int N>
struct alignas(sizeof(T) * N) Pack {
    T v[N];
};

#define FULL_MASK 0xffffffffu

// nodes per lane of the 16-bit storage kernel
#ifndef STEP16_V
#define STEP16_V 4
#endif

// ---------------------------------------------------------------- bulk step
// A warp owns VEC*32 consecutive nodes of one row (lane l: nodes x0..x0+VEC-1,
// x0 = seg*32*VEC + l*VEC) and loops over (row, segment) tasks. The +y and -y
// populations come from rows y-1 and y+1 at the same columns (aligned vector
// loads); the +x and -x populations come from the same row shifted by one
// column: each lane loads its own aligned vector and takes the missing end
// element from its neighbour lane by a shuffle (lane 0 / lane 31 load it).
//
// With FUSE the kernel also writes, into the ghost cells of fout, what the
// boundary nodes pull at the next step: everything that value depends on in
// the node form of Sec. 3.6 (f*_{-d} and U^n of the boundary node itself) is
// in the registers of the thread that owns the node. Periodic ghosts are the
// outgoing populations of the opposite edge's nodes.

// U^n of a node from its post-collision populations: sum_q f*_q = U + (dt/2) B
template <typename T>
__device__ __forceinline__ void state_from_fstar(const T f0[6], const T f1[6], const T f2[6], const T f3[6], T hb1,
                                                 T hb2, T U[6])
{
#pragma unroll
    for (int k = 0; k < 6; ++k) U[k] = (f0[k] + f2[k]) + (f1[k] + f3[k]);
    U[0] -= hb1;
    U[1] -= hb2;
}

// One node: Eq. (10) state recovery, P(F) (Appendix A), Eq. (7) fluxes,
// Eq. (12) equilibrium and Eq. (14) collision, in place on the four streamed
// populations f[q][k] (offsets). Returns the velocity v^n.
template <int LAW, typename T>
__device__ __forceinline__ void collide_node(T f[4][6], const StepArgs<T> &a, bool real, unsigned &flags, T &v1,
                                             T &v2)
{
    T U[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) U[k] = (f[0][k] + f[2][k]) + (f[1][k] + f[3][k]);
    U[0] += a.hdtb1;
    U[1] += a.hdtb2;
    T P11, P12, P21, P22, dJ;
    piola_ofs<LAW, T>(U[2], U[3], U[4], U[5], a.lam, a.mu, P11, P12, P21, P22, dJ);
    if (real) {
        if (!(dJ > T(-1))) flags |= ST_BAD_J;
        if (!(fabs(U[0]) + fabs(U[1]) + fabs(dJ) < T(INFINITY))) flags |= ST_NONFINITE;
    }
    v1 = U[0];
    v2 = U[1];
    // f^eq_q = U/4 + (1/2c)(i Phi_X + j Phi_Y)
    const T PhiX[6] = {-P11, -P21, -U[0], T(0), -U[1], T(0)};
    const T PhiY[6] = {-P12, -P22, T(0), -U[0], T(0), -U[1]};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const T qU = a.quarter * U[k];
        const T fx = a.inv2c * PhiX[k], fy = a.inv2c * PhiY[k];
        const T src = (k == 0) ? a.src1 : (k == 1) ? a.src2 : T(0);
        // f* = (1 - omega) f + omega f^eq + dt (2 - omega) w B
        f[0][k] = a.one_m_omega * f[0][k] + a.omega * (qU + fx) + src;
        f[2][k] = a.one_m_omega * f[2][k] + a.omega * (qU - fx) + src;
        f[1][k] = a.one_m_omega * f[1][k] + a.omega * (qU + fy) + src;
        f[3][k] = a.one_m_omega * f[3][k] + a.omega * (qU - fy) + src;
    }
}

// Ghost cells that node (x, y) is responsible for, from its post-collision
// populations f (compute type). Bottom ghost row (plane 1, y = -1), top ghost
// row (plane 3, y = ny), left ghost column (plane 0, x = -1), right ghost
// column (plane 2, x = nx), with the edge data of the step that will pull
// these values.
template <int LAW, typename S, typename T>
__device__ __forceinline__ void node_ghosts(const T f[4][6], int x, int y, const StepArgs<T> &a, S *fout,
                                            unsigned &flags)
{
    const int nx = a.L.nx, ny = a.L.ny;
    auto put = [&](int e, int gx, int gy, const T val[6]) {
        const int q = edge_dmiss(e);
        S *dst = fout + (long long)(q * 6) * a.L.plane + (long long)(gy + 1) * a.L.pitch + a.L.xoff + gx;
#pragma unroll
        for (int k = 0; k < 6; ++k) dst[k * a.L.plane] = to_store<S>(val[k]);
    };
    auto rule = [&](int e, int s, int gx, int gy) {
        T U[6], out[6];
        state_from_fstar(f[0], f[1], f[2], f[3], a.hdtb1, a.hdtb2, U);
        const double g = a.g[e] * (a.profile[e] ? a.profile[e][s] : 1.0);
        const double val[2] = {a.value[e][0] * g, a.value[e][1] * g};
        edge_ghost<LAW, T>(e, a.kind[e], f[edge_dout(e)], U, val, a.c, a.lam, a.mu, out, flags);
        put(e, gx, gy, out);
    };
    if (a.kind[EDGE_BOTTOM] == BC_PERIODIC) {
        if (y == ny - 1) put(EDGE_BOTTOM, x, -1, f[1]);
        if (y == 0) put(EDGE_TOP, x, ny, f[3]);
    } else {
        if (y == 0) rule(EDGE_BOTTOM, x, x, -1);
        if (y == ny - 1) rule(EDGE_TOP, x, x, ny);
    }
    if (a.kind[EDGE_LEFT] == BC_PERIODIC) {
        if (x == nx - 1) put(EDGE_LEFT, -1, y, f[0]);
        if (x == 0) put(EDGE_RIGHT, nx, y, f[2]);
    } else {
        if (x == 0) rule(EDGE_LEFT, y, -1, y);
        if (x == nx - 1) rule(EDGE_RIGHT, y, nx, y);
    }
}

// Task order shared by both step kernels: (row, segment) with the segments of
// row y rotated by y -- with a warp count that is a multiple of the number of
// segments, an unrotated order would give every edge segment (and its Newton
// solves) to the same few warps.
__device__ __forceinline__ void task_coords(int task, int nseg, int &y, int &seg)
{
    y = task / nseg;
    seg = (task - y * nseg + y) % nseg;
}

// After a lane has stored its nodes, the ghost cells its boundary nodes are
// responsible for are written from the stored post-collision values (read
// back by the same thread), so the edge work never adds to the register peak
// of the streaming loop, and it sees exactly the values the ghost-refresh
// kernel would read.
template <int LAW, typename S, int VEC>
__device__ __forceinline__ void lane_ghosts(const StepArgs<typename Prec<S>::R> &a, S *fout, long long row, int x0,
                                            int y, unsigned &flags)
{
    using T = typename Prec<S>::R;
    const int nx = a.L.nx, ny = a.L.ny;
    const bool edge_row = (y == 0 || y == ny - 1);
    if (!edge_row && x0 != 0 && !(x0 <= nx - 1 && nx - 1 < x0 + VEC)) return;
#pragma unroll 1
    for (int e = 0; e < VEC; ++e) {
        const int x = x0 + e;
        if (x >= nx) break;
        if (!edge_row && x != 0 && x != nx - 1) continue;
        T fq[4][6];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 6; ++k) fq[q][k] = ld_r(fout[(q * 6 + k) * a.L.plane + row + e]);
        node_ghosts<LAW, S, T>(fq, x, y, a, fout, flags);
    }
}

// FP64 and FP32 storage: VEC nodes per lane as 16-byte vectors, unpacked.
template <typename S, int LAW, int VEC, bool FUSE>
__global__ void __launch_bounds__(128) k_step(const StepArgs<typename Prec<S>::R> a)
{
    using T = typename Prec<S>::R;  // compute type
    using PK = Pack<S, VEC>;        // stored vector
    using PD = Pack<double, VEC>;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
    const int nw = gridDim.x * wpb;
    const int nx = a.L.nx, ny = a.L.ny;
    const int segw = 32 * VEC;
    const int nseg = (nx + segw - 1) / segw;
    const int ntask = ny * nseg;  // < 2^31 for every grid the library accepts
    const long long plane = a.L.plane;
    const int pitch = a.L.pitch;
    const S *__restrict__ fin = static_cast<const S *>(a.fin);
    S *__restrict__ fout = static_cast<S *>(a.fout);

    unsigned flags = 0;
    for (int task = gw; task < ntask; task += nw) {
        int y, seg;
        task_coords(task, nseg, y, seg);
        const int x0 = seg * segw + lane * VEC;
        const bool act = x0 < nx;   // lane owns at least one real node
        const bool ld0 = x0 <= nx;  // lane's vector holds a real node or the right ghost column
        const long long row = (long long)(y + 1) * pitch + a.L.xoff + x0;

        T f[4][6][VEC];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            PK c0 = {}, c1 = {}, c2 = {}, c3 = {};
            if (ld0) {
                c0 = *reinterpret_cast<const PK *>(fin + (0 * 6 + k) * plane + row);
                c2 = *reinterpret_cast<const PK *>(fin + (2 * 6 + k) * plane + row);
            }
            if (act) {
                c1 = *reinterpret_cast<const PK *>(fin + (1 * 6 + k) * plane + row - pitch);
                c3 = *reinterpret_cast<const PK *>(fin + (3 * 6 + k) * plane + row + pitch);
            }
            T left = __shfl_up_sync(FULL_MASK, ld_r(c0.v[VEC - 1]), 1);
            T right = __shfl_down_sync(FULL_MASK, ld_r(c2.v[0]), 1);
            if (act && lane == 0) left = ld_r(fin[(0 * 6 + k) * plane + row - 1]);
            if (act && lane == 31) right = ld_r(fin[(2 * 6 + k) * plane + row + VEC]);
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                f[0][k][e] = (e == 0) ? left : ld_r(c0.v[e - 1]);          // from x - 1 (Eq. 15)
                f[2][k][e] = (e == VEC - 1) ? right : ld_r(c2.v[e + 1]);   // from x + 1
                f[1][k][e] = ld_r(c1.v[e]);                                // from y - 1
                f[3][k][e] = ld_r(c3.v[e]);                                // from y + 1
            }
        }
        T vel[2][VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            T fq[4][6];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 6; ++k) fq[q][k] = f[q][k][e];
            collide_node<LAW, T>(fq, a, x0 + e < nx, flags, vel[0][e], vel[1][e]);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 6; ++k) f[q][k][e] = fq[q][k];
        }

        if (act) {
            const bool full = x0 + VEC <= nx;
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    S *dst = fout + (q * 6 + k) * plane + row;
                    if (full) {
                        PK o;
#pragma unroll
                        for (int e = 0; e < VEC; ++e) o.v[e] = to_store<S>(f[q][k][e]);
                        *reinterpret_cast<PK *>(dst) = o;
                    } else {
                        // ragged end: never write past node nx - 1 (column nx is a ghost cell)
#pragma unroll
                        for (int e = 0; e < VEC; ++e)
                            if (x0 + e < nx) dst[e] = to_store<S>(f[q][k][e]);
                    }
                }
            // Eq. (22): u*^{n+1} = u*^n + dt v^n (the two half steps of the paper)
            const long long urow = (long long)y * a.L.upitch + x0;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                PD u = *reinterpret_cast<const PD *>(a.ustar + c * a.L.uplane + urow);
#pragma unroll
                for (int e = 0; e < VEC; ++e) u.v[e] += a.dt * (double)vel[c][e];
                *reinterpret_cast<PD *>(a.ustar + c * a.L.uplane + urow) = u;
            }
            if (FUSE) lane_ghosts<LAW, S, VEC>(a, fout, row, x0, y, flags);
        }
    }
    flags = __reduce_or_sync(FULL_MASK, flags);
    if (flags && lane == 0) atomicOr(a.status, (int)flags);
}

// 16-bit storage (FP16, BF16): V = 4 or 8 nodes per lane, loaded as 8- or
// 16-byte vectors and kept packed in registers (two values per 32-bit word),
// so a lane holds half the registers of an unpacked vector. The one-column
// shifts of the +x and -x populations are funnel shifts of packed words; each
// node is unpacked, collided in FP32 and packed back in place.
__device__ __forceinline__ float unpack16(unsigned w, int hi, __half)
{
    return __half2float(__ushort_as_half((unsigned short)(hi ? (w >> 16) : (w & 0xffffu))));
}
__device__ __forceinline__ float unpack16(unsigned w, int hi, __nv_bfloat16)
{
    return __uint_as_float(hi ? (w & 0xffff0000u) : (w << 16));
}
template <typename S>
__device__ __forceinline__ unsigned bits16(float v);
template <>
__device__ __forceinline__ unsigned bits16<__half>(float v) { return __half_as_ushort(__float2half_rn(v)); }
template <>
__device__ __forceinline__ unsigned bits16<__nv_bfloat16>(float v)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

template <int W>
struct Words {
    unsigned w[W];
};

template <typename S, int LAW, int V, bool FUSE>
__global__ void __launch_bounds__(128, 4) k_step16(const StepArgs<float> a)
{
    constexpr int W = V / 2;  // 32-bit words per vector
    using WV = Words<W>;
    using PD = Pack<double, 4>;
    static_assert(V == 4 || V == 8, "4 or 8 nodes per lane");
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
    const int nw = gridDim.x * wpb;
    const int nx = a.L.nx, ny = a.L.ny;
    const int segw = 32 * V;
    const int nseg = (nx + segw - 1) / segw;
    const int ntask = ny * nseg;
    const long long plane = a.L.plane;
    const int pitch = a.L.pitch;
    const unsigned short *__restrict__ fin = static_cast<const unsigned short *>(a.fin);
    unsigned short *__restrict__ fout = static_cast<unsigned short *>(a.fout);
    auto ldv = [&](const unsigned short *p) {
        WV r;
        if constexpr (W == 2) {
            const uint2 t = *reinterpret_cast<const uint2 *>(p);
            r.w[0] = t.x;
            r.w[1] = t.y;
        } else {
            const uint4 t = *reinterpret_cast<const uint4 *>(p);
            r.w[0] = t.x;
            r.w[1] = t.y;
            r.w[2] = t.z;
            r.w[3] = t.w;
        }
        return r;
    };
    auto stv = [&](unsigned short *p, const WV &r) {
        if constexpr (W == 2)
            *reinterpret_cast<uint2 *>(p) = make_uint2(r.w[0], r.w[1]);
        else
            *reinterpret_cast<uint4 *>(p) = make_uint4(r.w[0], r.w[1], r.w[2], r.w[3]);
    };

    unsigned flags = 0;
    for (int task = gw; task < ntask; task += nw) {
        int y, seg;
        task_coords(task, nseg, y, seg);
        const int x0 = seg * segw + lane * V;
        const bool act = x0 < nx;
        const bool ld0 = x0 <= nx;
        const long long row = (long long)(y + 1) * pitch + a.L.xoff + x0;

        WV w[4][6];  // element e of plane (q, k) in half e & 1 of word e >> 1
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            WV c0 = {}, c1 = {}, c2 = {}, c3 = {};
            if (ld0) {
                c0 = ldv(fin + (0 * 6 + k) * plane + row);
                c2 = ldv(fin + (2 * 6 + k) * plane + row);
            }
            if (act) {
                c1 = ldv(fin + (1 * 6 + k) * plane + row - pitch);
                c3 = ldv(fin + (3 * 6 + k) * plane + row + pitch);
            }
            // +x: element e comes from x - 1, i.e. element e - 1 of this lane
            // (element V-1 of the previous lane for e = 0, carried in the high half)
            unsigned lw = __shfl_up_sync(FULL_MASK, c0.w[W - 1], 1);
            if (act && lane == 0) lw = (unsigned)fin[(0 * 6 + k) * plane + row - 1] << 16;
            w[0][k].w[0] = __funnelshift_l(lw, c0.w[0], 16);
#pragma unroll
            for (int i = 1; i < W; ++i) w[0][k].w[i] = __funnelshift_l(c0.w[i - 1], c0.w[i], 16);
            // -x: element e comes from x + 1 (element 0 of the next lane for e = V-1)
            unsigned rw = __shfl_down_sync(FULL_MASK, c2.w[0], 1);
            if (act && lane == 31) rw = (unsigned)fin[(2 * 6 + k) * plane + row + V];
#pragma unroll
            for (int i = 0; i < W - 1; ++i) w[2][k].w[i] = __funnelshift_r(c2.w[i], c2.w[i + 1], 16);
            w[2][k].w[W - 1] = __funnelshift_r(c2.w[W - 1], rw, 16);
            w[1][k] = c1;  // from y - 1
            w[3][k] = c3;  // from y + 1
        }
        // u* is read together with the populations so that its latency
        // overlaps theirs instead of following the collision
        const long long urow = (long long)y * a.L.upitch + x0;
        PD u[2][V / 4];
        if (act)
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int h = 0; h < V / 4; ++h) u[c][h] = *reinterpret_cast<const PD *>(a.ustar + c * a.L.uplane + urow + 4 * h);

        float vel[2][V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
            float fq[4][6];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 6; ++k) fq[q][k] = unpack16(w[q][k].w[e >> 1], e & 1, S());
            collide_node<LAW, float>(fq, a, x0 + e < nx, flags, vel[0][e], vel[1][e]);
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
                        stv(dst, w[q][k]);
                    } else {
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            const unsigned ww = w[q][k].w[e >> 1];
                            if (x0 + e < nx) dst[e] = (unsigned short)((e & 1) ? (ww >> 16) : (ww & 0xffffu));
                        }
                    }
                }
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int h = 0; h < V / 4; ++h) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) u[c][h].v[e] += a.dt * (double)vel[c][4 * h + e];
                    *reinterpret_cast<PD *>(a.ustar + c * a.L.uplane + urow + 4 * h) = u[c][h];
                }
            if (FUSE) lane_ghosts<LAW, S, V>(a, reinterpret_cast<S *>(fout), row, x0, y, flags);
        }
    }
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
    edge_ghost<LAW, T>(e, E.kind, fo, U, val, (T)a.c, (T)a.m.lam, (T)a.m.mu, out, flags);
    if (flags) atomicOr(a.status, (int)flags);
#pragma unroll
    for (int k = 0; k < 6; ++k) f[idx(d, k, gx, gy)] = to_store<S>(out[k]);
}

// ---------------------------------------------------------------- edges
template <typename T>
struct EdgeView {
    T *f;
    const Layout &L;
    __device__ long long idx(int q, int k, int x, int y) const
    {
        return (long long)(q * 6 + k) * L.plane + (long long)(y + 1) * L.pitch + L.xoff + x;
    }
};

// position (layer, p) on edge e -> node (x, y); layer 0 is the edge itself
__device__ __forceinline__ void edge_node(const Layout &L, int e, int layer, int p, int &x, int &y)
{
    switch (e) {
    case EDGE_LEFT: x = layer; y = p; break;
    case EDGE_RIGHT: x = L.nx - 1 - layer; y = p; break;
    case EDGE_BOTTOM: x = p; y = layer; break;
    default: x = p; y = L.ny - 1 - layer; break;
    }
}

// U^n at a node from the stored post-collision populations: sum_q f*_q =
// U + (dt/2) B (Eq. 14 summed over q with Eq. 10), offset form (v, G).
template <typename T>
__device__ void node_state(const EdgeView<T> &v, int x, int y, double hb1, double hb2, double U[6])
{
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) s += (double)ld_r(v.f[v.idx(q, k, x, y)]);
        U[k] = s;
    }
    U[0] -= hb1;
    U[1] -= hb2;
}

__device__ void piola_law(int law, const double G[4], double lam, double mu, double P[4], double &dJ)
{
    if (law == LAW_SVK)
        piola_ofs<LAW_SVK, double>(G[0], G[1], G[2], G[3], lam, mu, P[0], P[1], P[2], P[3], dJ);
    else if (law == LAW_NH)
        piola_ofs<LAW_NH, double>(G[0], G[1], G[2], G[3], lam, mu, P[0], P[1], P[2], P[3], dJ);
    else
        piola_ofs<LAW_LOGNH, double>(G[0], G[1], G[2], G[3], lam, mu, P[0], P[1], P[2], P[3], dJ);
}

// tangential derivative of v_i along edge e in layer `layer` at position s:
// central difference, wrap-around when the tangential direction is periodic,
// one-sided three-point stencil at the edge ends
template <typename T>
__device__ void edge_dv(const EdgeView<T> &v, const EdgeArgs &a, int e, int layer, int s, int len, int tper,
                        double dv[2])
{
    int p[3];
    double w[3];
    if (tper) {
        p[0] = (s - 1 + len) % len; p[1] = s; p[2] = (s + 1) % len;
        w[0] = -0.5; w[1] = 0.0; w[2] = 0.5;
    } else if (s == 0) {
        p[0] = 0; p[1] = 1; p[2] = 2;
        w[0] = -1.5; w[1] = 2.0; w[2] = -0.5;
    } else if (s == len - 1) {
        p[0] = len - 3; p[1] = len - 2; p[2] = len - 1;
        w[0] = 0.5; w[1] = -2.0; w[2] = 1.5;
    } else {
        p[0] = s - 1; p[1] = s; p[2] = s + 1;
        w[0] = -0.5; w[1] = 0.0; w[2] = 0.5;
    }
    dv[0] = dv[1] = 0.0;
    for (int j = 0; j < 3; ++j) {
        if (w[j] == 0.0) continue;
        int x, y;
        edge_node(a.L, e, layer, p[j], x, y);
        double U[6];
        node_state(v, x, y, a.hdtb1, a.hdtb2, U);
        dv[0] += w[j] * U[0];
        dv[1] += w[j] * U[1];
    }
    dv[0] /= a.dx;
    dv[1] /= a.dx;
}

// Sec. 3.6.2: boundary deformation gradient (offset form G^b = F^b - I) on a
// traction edge; Newton on r_i = N_a P_ia(F^b) - T_i for the normal column
// with a halving line search that rejects det F^b <= 0. Returns false if the
// residual did not reach the tolerance.
template <typename T>
__device__ bool traction_Fb(const EdgeView<T> &v, const EdgeArgs &a, int e, int s, int len, const double Tb[2],
                            double Gb[4])
{
    const int an = (e <= EDGE_RIGHT) ? 0 : 1;
    const int tc = 1 - an;
    const double Na = (e == EDGE_LEFT || e == EDGE_BOTTOM) ? -1.0 : 1.0;
    int x0, y0;
    edge_node(a.L, e, 0, s, x0, y0);
    double U0[6];
    node_state(v, x0, y0, a.hdtb1, a.hdtb2, U0);
    if (a.fb_mode == FB_EXTRAP2) {
        int x1, y1;
        edge_node(a.L, e, 1, s, x1, y1);
        double U1[6], dv0[2], dv1[2];
        node_state(v, x1, y1, a.hdtb1, a.hdtb2, U1);
        const int tper = (e <= EDGE_RIGHT) ? a.yper : a.xper;
        edge_dv(v, a, e, 0, s, len, tper, dv0);
        edge_dv(v, a, e, 1, s, len, tper, dv1);
        for (int i = 0; i < 2; ++i)
            Gb[i * 2 + tc] = 1.5 * U0[2 + i * 2 + tc] - 0.5 * U1[2 + i * 2 + tc] +
                             0.5 * a.dt * (1.5 * dv0[i] - 0.5 * dv1[i]);
    } else {
        for (int i = 0; i < 2; ++i) Gb[i * 2 + tc] = U0[2 + i * 2 + tc];
    }
    for (int i = 0; i < 2; ++i) Gb[i * 2 + an] = U0[2 + i * 2 + an];

    const double tmax = fmax(fabs(Tb[0]), fabs(Tb[1]));
    const double tol = 1e-13 * (tmax > 1.0 ? tmax : 1.0);
    double P[4], dJ, r[2];
    piola_law(a.m.law, Gb, a.m.lam, a.m.mu, P, dJ);
    r[0] = Na * P[0 * 2 + an] - Tb[0];
    r[1] = Na * P[1 * 2 + an] - Tb[1];
    for (int it = 0; it < 20; ++it) {
        if (fmax(fabs(r[0]), fabs(r[1])) <= tol) return true;
        const double F[4] = {1.0 + Gb[0], Gb[1], Gb[2], 1.0 + Gb[3]};
        double Jac[2][2];
        for (int k = 0; k < 2; ++k) {
            double dF[4] = {0.0, 0.0, 0.0, 0.0}, dP[4];
            dF[k * 2 + an] = 1.0;
            tangent_jvp(a.m.law, F, dF, a.m.lam, a.m.mu, dP);
            Jac[0][k] = Na * dP[0 * 2 + an];
            Jac[1][k] = Na * dP[1 * 2 + an];
        }
        const double det = Jac[0][0] * Jac[1][1] - Jac[0][1] * Jac[1][0];
        const double d0 = -(Jac[1][1] * r[0] - Jac[0][1] * r[1]) / det;
        const double d1 = -(-Jac[1][0] * r[0] + Jac[0][0] * r[1]) / det;
        const double rn = hypot(r[0], r[1]);
        double alpha = 1.0;
        bool accepted = false;
        for (int ls = 0; ls <= 10; ++ls) {
            double Gt[4] = {Gb[0], Gb[1], Gb[2], Gb[3]};
            Gt[0 * 2 + an] += alpha * d0;
            Gt[1 * 2 + an] += alpha * d1;
            const double Jt = (1.0 + Gt[0]) * (1.0 + Gt[3]) - Gt[1] * Gt[2];
            if (Jt > 0.0) {
                double Pt[4], dJt, rt[2];
                piola_law(a.m.law, Gt, a.m.lam, a.m.mu, Pt, dJt);
                rt[0] = Na * Pt[0 * 2 + an] - Tb[0];
                rt[1] = Na * Pt[1 * 2 + an] - Tb[1];
                if (hypot(rt[0], rt[1]) < rn) {
                    for (int m = 0; m < 4; ++m) Gb[m] = Gt[m];
                    r[0] = rt[0];
                    r[1] = rt[1];
                    accepted = true;
                    break;
                }
            }
            alpha *= 0.5;
        }
        if (!accepted) break;
    }
    return fmax(fabs(r[0]), fabs(r[1])) <= tol;
}

template <typename T>
__global__ void __launch_bounds__(128) k_edges(const EdgeArgs a)
{
    EdgeView<T> v{static_cast<T *>(a.f), a.L};
    int e = 0;
    while (e < 3 && (int)blockIdx.x >= a.blk_end[e]) ++e;
    const int b0 = e ? a.blk_end[e - 1] : 0;
    const int s = ((int)blockIdx.x - b0) * blockDim.x + threadIdx.x;
    const int len = (e <= EDGE_RIGHT) ? a.L.ny : a.L.nx;
    if (s >= len) return;
    const EdgeDesc &E = a.e[e];
    // boundary node (xb, yb), ghost cell (gx, gy), missing direction d = -N
    // and the outgoing direction -d = N at the same node
    int xb, yb, gx, gy, d, md;
    double N0, N1;
    switch (e) {
    case EDGE_LEFT: xb = 0; yb = s; gx = -1; gy = s; d = 0; md = 2; N0 = -1; N1 = 0; break;
    case EDGE_RIGHT: xb = a.L.nx - 1; yb = s; gx = a.L.nx; gy = s; d = 2; md = 0; N0 = 1; N1 = 0; break;
    case EDGE_BOTTOM: xb = s; yb = 0; gx = s; gy = -1; d = 1; md = 3; N0 = 0; N1 = -1; break;
    default: xb = s; yb = a.L.ny - 1; gx = s; gy = a.L.ny; d = 3; md = 1; N0 = 0; N1 = 1; break;
    }
    if (E.kind == BC_PERIODIC) {
        // the population leaving through the opposite edge re-enters here
        const int sx = (e == EDGE_LEFT) ? a.L.nx - 1 : (e == EDGE_RIGHT) ? 0 : s;
        const int sy = (e == EDGE_BOTTOM) ? a.L.ny - 1 : (e == EDGE_TOP) ? 0 : s;
#pragma unroll
        for (int k = 0; k < 6; ++k) v.f[v.idx(d, k, gx, gy)] = v.f[v.idx(d, k, sx, sy)];
        return;
    }
    // edge data at t^n + dt/2 (Eq. 23)
    double val[2];
    edge_value(E, s, a.g[e], val);
    double D[6], S[6];
    if (E.kind == BC_VELOCITY) {
        // Eq. (24); the F-components have D = +1, so the rest offset cancels
        D[0] = -1; D[1] = -1; D[2] = 1; D[3] = 1; D[4] = 1; D[5] = 1;
        S[0] = 0.5 * val[0];
        S[1] = 0.5 * val[1];
        S[2] = N0 * val[0] / a.c;
        S[3] = N1 * val[0] / a.c;
        S[4] = N0 * val[1] / a.c;
        S[5] = N1 * val[1] / a.c;
    } else {
        // Eq. (25) with D = -1 on the F-components: in offset form the source
        // becomes (F^b - I)/2 = G^b/2
        double Gb[4];
        if (!traction_Fb(v, a, e, s, len, val, Gb)) atomicOr(a.status, ST_NEWTON);
        D[0] = 1; D[1] = 1; D[2] = -1; D[3] = -1; D[4] = -1; D[5] = -1;
        S[0] = val[0] / a.c;
        S[1] = val[1] / a.c;
        for (int m = 0; m < 4; ++m) S[2 + m] = 0.5 * Gb[m];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
        v.f[v.idx(d, k, gx, gy)] = to_store<T>(D[k] * (double)ld_r(v.f[v.idx(md, k, xb, yb)]) + S[k]);
}

// ---------------------------------------------------------------- launchers
template <typename S, int LAW>
static cudaError_t launch_step_t(const StepArgs<typename Prec<S>::R> &a, bool fuse, int grid, cudaStream_t st)
{
    if constexpr (sizeof(S) == 2) {
        if (fuse)
            k_step16<S, LAW, STEP16_V, true><<<grid, 128, 0, st>>>(a);
        else
            k_step16<S, LAW, STEP16_V, false><<<grid, 128, 0, st>>>(a);
    } else {
        constexpr int VEC = 16 / sizeof(S);  // 16-byte vectors
        if (fuse)
            k_step<S, LAW, VEC, true><<<grid, 128, 0, st>>>(a);
        else
            k_step<S, LAW, VEC, false><<<grid, 128, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <typename S>
static cudaError_t launch_step_law(int law, const void *args, bool fuse, int grid, cudaStream_t st)
{
    const auto &a = *static_cast<const StepArgs<typename Prec<S>::R> *>(args);
    switch (law) {
    case LAW_SVK: return launch_step_t<S, LAW_SVK>(a, fuse, grid, st);
    case LAW_NH: return launch_step_t<S, LAW_NH>(a, fuse, grid, st);
    default: return launch_step_t<S, LAW_LOGNH>(a, fuse, grid, st);
    }
}

cudaError_t launch_step(int storage, int law, bool fuse, const void *args, int grid, cudaStream_t st)
{
    return with_storage(storage, [&](auto tag) {
        return launch_step_law<decltype(tag)>(law, args, fuse, grid, st);
    });
}

cudaError_t launch_edges(int storage, const EdgeArgs &a, int grid, cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    return with_storage(storage, [&](auto tag) {
        k_edges<decltype(tag)><<<grid, 128, 0, st>>>(a);
        return cudaGetLastError();
    });
}

cudaError_t launch_ghosts(int storage, const EdgeArgs &a, int grid, cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    return with_storage(storage, [&](auto tag) {
        using S = decltype(tag);
        switch (a.m.law) {
        case LAW_SVK: k_ghosts<S, LAW_SVK><<<grid, 128, 0, st>>>(a); break;
        case LAW_NH: k_ghosts<S, LAW_NH><<<grid, 128, 0, st>>>(a); break;
        default: k_ghosts<S, LAW_LOGNH><<<grid, 128, 0, st>>>(a); break;
        }
        return cudaGetLastError();
    });
}

int step_blocks_per_sm(int storage, int law)
{
    return with_storage(storage, [&](auto tag) {
        using S = decltype(tag);
        const void *fn;
        if constexpr (sizeof(S) == 2)
            fn = (law == LAW_SVK) ? (const void *)k_step16<S, LAW_SVK, STEP16_V, true>
                 : (law == LAW_NH) ? (const void *)k_step16<S, LAW_NH, STEP16_V, true>
                                   : (const void *)k_step16<S, LAW_LOGNH, STEP16_V, true>;
        else
            fn = (law == LAW_SVK) ? (const void *)k_step<S, LAW_SVK, 16 / sizeof(S), true>
                 : (law == LAW_NH) ? (const void *)k_step<S, LAW_NH, 16 / sizeof(S), true>
                                   : (const void *)k_step<S, LAW_LOGNH, 16 / sizeof(S), true>;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 128, 0) != cudaSuccess) n = 0;
        return n;
    });
}

int step_vec(int storage) { return storage == STORE_F64 ? 2 : storage == STORE_F32 ? 4 : STEP16_V; }

} // namespace tlv
