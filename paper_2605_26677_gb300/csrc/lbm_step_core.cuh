// lbm_step_core.cuh -- the per-task device code of the fused step (Sec. 3.7):
// one warp advances one (row, segment) task of one lattice by one step. The
// single-lattice kernels (lbm_step.cu) and the batched kernels
// (lbm_batch_kernels.cuh) loop over tasks and call these functions.
#pragma once
#include "lbm_device.cuh"
#include "lbm_edges.cuh"

namespace tlv {

template <typename T, int N>
struct alignas(sizeof(T) * N) Pack {
    T v[N];
};

#define FULL_MASK 0xffffffffu

// x is NaN or infinite: all exponent bits set, tested on the integer pipe
// (the FP64 pipe is the FP64 step's bottleneck)
__device__ __forceinline__ bool nonfinite(double x) { return (__double2hiint(x) & 0x7ff00000) == 0x7ff00000; }
__device__ __forceinline__ bool nonfinite(float x) { return (__float_as_int(x) & 0x7f800000) == 0x7f800000; }

// Dynamic task claims of one launch: the tasks [0, ntask) form NS contiguous
// stripes, stripe j claimed through counter ctr[j * DYN_CTR_STRIDE] (zero
// when the launch begins). A warp starts in the stripe of its global warp
// index modulo NS, claims one task ahead of the one it runs (the atomic's
// latency overlaps the task), and when a stripe runs out moves on to the
// next, cyclically, until it has found every stripe empty; a slower warp so
// takes fewer tasks and the launch ends evenly. Every task is run exactly
// once: each counter value is returned once, and no warp leaves before every
// stripe is empty. Several stripes divide the claims among several counters:
// with a single counter the 16-bit kernel on 8192^2 ran at 2.97e8 claims per
// second in five builds with different arithmetic (0.718 of the copy
// bandwidth against 0.91 in static order), so the one counter, not the
// kernel, set the pace. run(task) is called with the same task by all lanes
// of the warp.
template <int NS, typename Fn>
__device__ __forceinline__ void claim_tasks(unsigned *ctr, int ntask, int lane, Fn &&run)
{
    static_assert(NS >= 1 && NS <= DYN_STRIPES && (NS & (NS - 1)) == 0, "1 .. DYN_STRIPES stripes, a power of two");
    // the warp's k-th stripe (k = 0 .. NS - 1), starting from its
    // global warp index; recomputed where needed rather than kept in a
    // register (the 16-bit kernels run at their register limit)
    auto stripe = [](int k) {
        return ((int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) + k) & (NS - 1);
    };
    // stripe s holds tasks [s q + min(s, r), (s + 1) q + min(s + 1, r)),
    // q = ntask / NS, r = ntask % NS
    auto size = [&](int s) { return (unsigned)ntask / NS + ((unsigned)s < (unsigned)ntask % NS ? 1u : 0u); };
    auto start = [&](int s) { return (unsigned)s * ((unsigned)ntask / NS) + min((unsigned)s, (unsigned)ntask % NS); };
    int k = 0;
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(ctr + stripe(0) * DYN_CTR_STRIDE, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    for (;;) {
        if (t >= size(stripe(k))) {  // this stripe is empty: the next one
            if (++k == NS) break;
            if (lane == 0) t = atomicAdd(ctr + stripe(k) * DYN_CTR_STRIDE, 1u);
            t = __shfl_sync(0xffffffffu, t, 0);
            continue;
        }
        const int task = (int)(start(stripe(k)) + t);
        unsigned u = 0;
        if (lane == 0) u = atomicAdd(ctr + stripe(k) * DYN_CTR_STRIDE, 1u);  // the next claim, ahead
        run(task);
        t = __shfl_sync(0xffffffffu, u, 0);
    }
}

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
__device__ __forceinline__ void collide_node(T f[4][6], const StepArgs<T> &a, const LawP<T> &m, bool real,
                                             unsigned &flags, T &v1, T &v2)
{
    T U[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) U[k] = (f[0][k] + f[2][k]) + (f[1][k] + f[3][k]);
    U[0] += a.hdtb1;
    U[1] += a.hdtb2;
    T P11, P12, P21, P22, dJ;
    piola_ofs<LAW, T>(U[2], U[3], U[4], U[5], m, P11, P12, P21, P22, dJ);
    if (real) {
        if (!(dJ > T(-1))) flags |= ST_BAD_J;
        if (nonfinite(U[0]) | nonfinite(U[1]) | nonfinite(dJ)) flags |= ST_NONFINITE;
    }
    v1 = U[0];
    v2 = U[1];
    // f^eq_q = U/4 + (1/2c)(i Phi_X + j Phi_Y), and
    // f* = (1 - omega) f + omega f^eq + dt (2 - omega) w B, evaluated as
    //   t_q = (1 - omega) f_q + (omega/4 U + src)   (one FMA)
    //   f*_q = t_q +- (omega/2c) Phi                 (one FMA)
    // with omega/4 and omega/(2c) formed once on the host. The structural
    // zeros (Phi_X of F12 and F22, Phi_Y of F11 and F21, the source beyond
    // the velocity components) are skipped at compile time: under IEEE rules
    // the compiler may not drop a product with or a sum of a zero itself.
    const T PhiX[6] = {-P11, -P21, -U[0], T(0), -U[1], T(0)};
    const T PhiY[6] = {-P12, -P22, T(0), -U[0], T(0), -U[1]};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const bool hx = (k != 3 && k != 5), hy = (k != 2 && k != 4);
        const T aU = (k < 2) ? fma(a.wq, U[k], (k == 0) ? a.src1 : a.src2) : a.wq * U[k];
        const T t0 = fma(a.one_m_omega, f[0][k], aU);
        const T t2 = fma(a.one_m_omega, f[2][k], aU);
        const T t1 = fma(a.one_m_omega, f[1][k], aU);
        const T t3 = fma(a.one_m_omega, f[3][k], aU);
        f[0][k] = hx ? fma(a.wc, PhiX[k], t0) : t0;
        f[2][k] = hx ? fma(-a.wc, PhiX[k], t2) : t2;
        f[1][k] = hy ? fma(a.wc, PhiY[k], t1) : t1;
        f[3][k] = hy ? fma(-a.wc, PhiY[k], t3) : t3;
    }
}

// Ghost cells that node (x, y) is responsible for, from its post-collision
// populations f (compute type). Bottom ghost row (plane 1, y = -1), top ghost
// row (plane 3, y = ny), left ghost column (plane 0, x = -1), right ghost
// column (plane 2, x = nx), with the edge data of the step that will pull
// these values.
template <int LAW, typename S, typename T, bool SKIP_X = false>
__device__ __forceinline__ void node_ghosts(const T f[4][6], int x, int y, const StepArgs<T> &a, const LawP<T> &m,
                                            S *fout, unsigned &flags)
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
        const double g = (a.gdev ? a.gdev[e] : a.g[e]) * (a.profile[e] ? a.profile[e][s] : 1.0);
        const double val[2] = {a.value[e][0] * g, a.value[e][1] * g};
        edge_ghost<LAW, T>(e, a.kind[e], f[edge_dout(e)], U, val, a.c, m, out, flags);
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
    } else if (!SKIP_X) {
        if (x == 0) rule(EDGE_LEFT, y, -1, y);
        if (x == nx - 1) rule(EDGE_RIGHT, y, nx, y);
    }
}

// Deferred side-edge rules (XQ kernels): a node on a non-periodic x edge
// outside the two edge rows is not handled by its own lane while the warp's
// 31 other lanes wait; its coordinates go to the warp's queue in shared
// memory, and once 32 have gathered every lane of the warp takes one
// (xedge_flush). The rule reads the node's stored post-collision values, as
// the inline rule does, so the ghost values are the same bits.
struct XPend {
    int x, y;  // the lane's pending node, x = -1 for none
};

// The queue of one warp: XQ_CAP entries (x, y, member) in shared memory; a
// task adds at most two, and 32 are processed as soon as they are queued.
constexpr int XQ_CAP = 64;
struct XQueue {
    int *qx, *qy, *qm;
    int n;  // warp-uniform
};

__device__ __forceinline__ XQueue xq_make(int *base)
{
    int *qx = base + (threadIdx.x >> 5) * 3 * XQ_CAP;
    return XQueue{qx, qx + XQ_CAP, qx + 2 * XQ_CAP, 0};
}

// up to 32 queued nodes, one per lane (proc(x, y, m)); the rest moves to the
// front of the queue
template <typename Proc>
__device__ __forceinline__ void xq_flush(XQueue &q, int lane, Proc &&proc)
{
    __syncwarp();  // the queued nodes' stores, made by this warp's lanes, are visible
    const int nproc = q.n < 32 ? q.n : 32;
    if (lane < nproc) proc(q.qx[lane], q.qy[lane], q.qm[lane]);
    const int rest = q.n - nproc;
    int rx = 0, ry = 0, rm = 0;
    if (lane < rest) {
        rx = q.qx[nproc + lane];
        ry = q.qy[nproc + lane];
        rm = q.qm[nproc + lane];
    }
    __syncwarp();
    if (lane < rest) {
        q.qx[lane] = rx;
        q.qy[lane] = ry;
        q.qm[lane] = rm;
    }
    __syncwarp();
    q.n = rest;
}

// the lanes' pending nodes of one task (member m) into the queue
template <typename Proc>
__device__ __forceinline__ void xq_push(XQueue &q, const XPend &xp, int m, int lane, Proc &&proc)
{
    const unsigned bal = __ballot_sync(0xffffffffu, xp.x >= 0);
    if (!bal) return;
    if (xp.x >= 0) {
        const int pos = q.n + __popc(bal & ((1u << lane) - 1u));
        q.qx[pos] = xp.x;
        q.qy[pos] = xp.y;
        q.qm[pos] = m;
    }
    q.n += __popc(bal);
    if (q.n >= 32) xq_flush(q, lane, proc);
}

template <int LAW, typename S, bool MATF = false>
__device__ __forceinline__ void xedge_node(const StepArgs<typename Prec<S>::R> &a, int x, int y, unsigned &flags)
{
    using T = typename Prec<S>::R;
    S *fout = static_cast<S *>(a.fout);
    const long long row = (long long)(y + 1) * a.L.pitch + a.L.xoff + x;
    T fq[4][6];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 6; ++k) fq[q][k] = ld_r(fout[(q * 6 + k) * a.L.plane + row]);
    LawP<T> m{a.lam, a.mu, a.p2, a.p3};
    if (MATF) {
        m.mu = a.mufield[(long long)y * a.L.upitch + x];
        m.lam = a.lam_ratio * m.mu;
    }
    // an interior row: only the side-edge rules apply to the node
    const int nx = a.L.nx;
    const T *f0 = fq[0], *f1 = fq[1], *f2 = fq[2], *f3 = fq[3];
    T U[6], out[6];
    state_from_fstar(f0, f1, f2, f3, a.hdtb1, a.hdtb2, U);
    for (int side = 0; side < 2; ++side) {
        const int e = side == 0 ? EDGE_LEFT : EDGE_RIGHT;
        if ((side == 0 && x != 0) || (side == 1 && x != nx - 1)) continue;
        const double g = (a.gdev ? a.gdev[e] : a.g[e]) * (a.profile[e] ? a.profile[e][y] : 1.0);
        const double val[2] = {a.value[e][0] * g, a.value[e][1] * g};
        edge_ghost<LAW, T>(e, a.kind[e], fq[edge_dout(e)], U, val, a.c, m, out, flags);
        S *dst = fout + (long long)(edge_dmiss(e) * 6) * a.L.plane + (long long)(y + 1) * a.L.pitch + a.L.xoff +
                 (side == 0 ? -1 : nx);
#pragma unroll
        for (int k = 0; k < 6; ++k) dst[k * a.L.plane] = to_store<S>(out[k]);
    }
}

// Task order shared by the step kernels: (row, segment), rows in the order
// 0, ny - 1, 1, 2, ..., ny - 2, and the segments of row y rotated by y. The
// two edge rows, whose every lane runs edge rules (traction Newton solves),
// come first, so that their longer tasks overlap the later rounds of the
// persistent grid instead of forming its tail; without the rotation, a warp
// count that is a multiple of the segments per row would hand every edge
// segment of the side edges to the same few warps.
__device__ __forceinline__ void task_coords(int task, int nseg, int ny, int &y, int &seg)
{
    const int r = task / nseg;
    y = (r == 0 || ny < 2) ? r : (r == 1 ? ny - 1 : r - 1);
    seg = (task - r * nseg + y) % nseg;
}

// After a lane has stored its nodes, the ghost cells its boundary nodes are
// responsible for are written from the stored post-collision values (read
// back by the same thread), so the edge work never adds to the register peak
// of the streaming loop, and it sees exactly the values the ghost-refresh
// kernel would read.
template <int LAW, typename S, int VEC, bool MATF = false, bool XQ = false>
__device__ __forceinline__ void lane_ghosts(const StepArgs<typename Prec<S>::R> &a, S *fout, long long row, int x0,
                                            int y, unsigned &flags, XPend *xp = nullptr)
{
    using T = typename Prec<S>::R;
    const int nx = a.L.nx, ny = a.L.ny;
    const bool edge_row = (y == 0 || y == ny - 1);
    if (!edge_row && x0 != 0 && !(x0 <= nx - 1 && nx - 1 < x0 + VEC)) return;
    if constexpr (XQ) {
        // one side-edge node of an interior row is deferred to the warp's
        // queue; a lane holding both side nodes (nx <= VEC) keeps them
        if (!edge_row && a.kind[EDGE_LEFT] != BC_PERIODIC && !(x0 == 0 && nx - 1 < x0 + VEC)) {
            xp->x = (x0 == 0) ? 0 : nx - 1;
            xp->y = y;
            return;
        }
    }
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
        LawP<T> m{a.lam, a.mu, a.p2, a.p3};
        if (MATF) {
            m.mu = a.mufield[(long long)y * a.L.upitch + x];
            m.lam = a.lam_ratio * m.mu;
        }
        node_ghosts<LAW, S, T>(fq, x, y, a, m, fout, flags);
    }
}

// FP64 and FP32 storage: VEC nodes per lane as 16-byte vectors, unpacked.
// One (row, segment) task of lattice `a`, executed by a whole warp.
// NOQ: no displacement quadrature (states recomputed only for their
// populations, as the adjoint's checkpoint segments are).
template <typename S, int LAW, int VEC, bool FUSE, bool MATF = false, bool NOQ = false, bool XQ = false>
__device__ __forceinline__ void step_task(const StepArgs<typename Prec<S>::R> &a, int task, int lane,
                                          unsigned &flags, XPend *xp = nullptr)
{
    using T = typename Prec<S>::R;  // compute type
    using PK = Pack<S, VEC>;        // stored vector
    using PD = Pack<double, VEC>;
    const int nx = a.L.nx;
    const int segw = 32 * VEC;
    const int nseg = (nx + segw - 1) / segw;
    const long long plane = a.L.plane;
    const int pitch = a.L.pitch;
    const S *__restrict__ fin = static_cast<const S *>(a.fin);
    S *__restrict__ fout = static_cast<S *>(a.fout);
    {
        int y, seg;
        task_coords(task, nseg, a.L.ny, y, seg);
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
        T muv[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) muv[e] = a.mu;
        if (MATF && act) {
            const Pack<T, VEC> m = *reinterpret_cast<const Pack<T, VEC> *>(a.mufield + (long long)y * a.L.upitch + x0);
#pragma unroll
            for (int e = 0; e < VEC; ++e) muv[e] = m.v[e];
        }
        T vel[2][VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            T fq[4][6];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 6; ++k) fq[q][k] = f[q][k][e];
            const LawP<T> m{MATF ? a.lam_ratio * muv[e] : a.lam, muv[e], a.p2, a.p3};
            collide_node<LAW, T>(fq, a, m, x0 + e < nx, flags, vel[0][e], vel[1][e]);
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
            if constexpr (!NOQ) {
                const long long urow = (long long)y * a.L.upitch + x0;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    PD u = *reinterpret_cast<const PD *>(a.ustar + c * a.L.uplane + urow);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) u.v[e] += a.dt * (double)vel[c][e];
                    *reinterpret_cast<PD *>(a.ustar + c * a.L.uplane + urow) = u;
                }
            }
            if (FUSE) lane_ghosts<LAW, S, VEC, MATF, XQ>(a, fout, row, x0, y, flags, xp);
        }
    }
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

template <typename S, int LAW, int V, bool FUSE, bool MATF = false>
__device__ __forceinline__ void step16_task(const StepArgs<float> &a, int task, int lane, unsigned &flags)
{
    constexpr int W = V / 2;  // 32-bit words per vector
    using WV = Words<W>;
    using PD = Pack<double, 4>;
    static_assert(V == 4 || V == 8, "4 or 8 nodes per lane");
    const int nx = a.L.nx;
    const int segw = 32 * V;
    const int nseg = (nx + segw - 1) / segw;
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

    {
        int y, seg;
        task_coords(task, nseg, a.L.ny, y, seg);
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
        // per-node mu (material field, compute-type plane in the u* layout);
        // read only by the MATF kernels
        float muv[V];
        if (MATF && act)
#pragma unroll
            for (int h = 0; h < V / 4; ++h) {
                const Pack<float, 4> m = *reinterpret_cast<const Pack<float, 4> *>(a.mufield + urow + 4 * h);
#pragma unroll
                for (int e = 0; e < 4; ++e) muv[4 * h + e] = m.v[e];
            }
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
            collide_node<LAW, float>(fq, a, MATF ? LawP<float>{a.lam_ratio * muv[e], muv[e], a.p2, a.p3} : LawP<float>{a.lam, a.mu, a.p2, a.p3}, x0 + e < nx, flags, vel[0][e],
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
            if (FUSE) lane_ghosts<LAW, S, V, MATF>(a, reinterpret_cast<S *>(fout), row, x0, y, flags);
        }
    }
}

} // namespace tlv
