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

template <typename T, int LAW, int VEC, bool FUSE>
__global__ void __launch_bounds__(128) k_step(const StepArgs<T> a)
{
    using PK = Pack<T, VEC>;
    using PD = Pack<double, VEC>;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const long long gw = (long long)blockIdx.x * wpb + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * wpb;
    const int nx = a.L.nx, ny = a.L.ny;
    const int segw = 32 * VEC;
    const int nseg = (nx + segw - 1) / segw;
    const long long ntask = (long long)ny * nseg;
    const long long plane = a.L.plane;
    const int pitch = a.L.pitch;
    const T *__restrict__ fin = a.fin;
    T *__restrict__ fout = a.fout;
    const long long n_in = *a.step_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.step_out = n_in + 1;
    // edge data for the next step's pull is sampled at t^{n} + dt/2 (Eq. 23)
    const double th = ((double)n_in + 1.5) * a.dt;

    unsigned flags = 0;
    for (long long task = gw; task < ntask; task += nw) {
        const int y = (int)(task / nseg);
        // the segments of row y are taken in an order rotated by y: with a warp
        // count that is a multiple of nseg, an unrotated order would give every
        // edge segment (and its Newton solves) to the same few warps
        const int seg = (int)((task - (long long)y * nseg + y) % nseg);
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
            T left = __shfl_up_sync(FULL_MASK, c0.v[VEC - 1], 1);
            T right = __shfl_down_sync(FULL_MASK, c2.v[0], 1);
            if (act && lane == 0) left = fin[(0 * 6 + k) * plane + row - 1];
            if (act && lane == 31) right = fin[(2 * 6 + k) * plane + row + VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                f[0][k][e] = (e == 0) ? left : c0.v[e - 1];          // from x - 1 (Eq. 15)
                f[2][k][e] = (e == VEC - 1) ? right : c2.v[e + 1];   // from x + 1
                f[1][k][e] = c1.v[e];                                // from y - 1
                f[3][k][e] = c3.v[e];                                // from y + 1
            }
        }

        T vel[2][VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            // Eq. (10): U = sum_q f_q + (dt/2) B (offsets: F-components give G = F - I)
            T U[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) U[k] = (f[0][k][e] + f[2][k][e]) + (f[1][k][e] + f[3][k][e]);
            U[0] += a.hdtb1;
            U[1] += a.hdtb2;
            T P11, P12, P21, P22, dJ;
            piola_ofs<LAW, T>(U[2], U[3], U[4], U[5], a.lam, a.mu, P11, P12, P21, P22, dJ);
            if (x0 + e < nx) {
                if (!(dJ > T(-1))) flags |= ST_BAD_J;
                if (!(fabs(U[0]) + fabs(U[1]) + fabs(dJ) < T(INFINITY))) flags |= ST_NONFINITE;
            }
            vel[0][e] = U[0];
            vel[1][e] = U[1];
            // Eq. (7) fluxes, Eq. (12) equilibrium: f^eq_q = U/4 + (1/2c)(i Phi_X + j Phi_Y)
            const T PhiX[6] = {-P11, -P21, -U[0], T(0), -U[1], T(0)};
            const T PhiY[6] = {-P12, -P22, T(0), -U[0], T(0), -U[1]};
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const T qU = a.quarter * U[k];
                const T fx = a.inv2c * PhiX[k], fy = a.inv2c * PhiY[k];
                const T src = (k == 0) ? a.src1 : (k == 1) ? a.src2 : T(0);
                // Eq. (14): f* = (1 - omega) f + omega f^eq + dt (2 - omega) w B
                f[0][k][e] = a.one_m_omega * f[0][k][e] + a.omega * (qU + fx) + src;
                f[2][k][e] = a.one_m_omega * f[2][k][e] + a.omega * (qU - fx) + src;
                f[1][k][e] = a.one_m_omega * f[1][k][e] + a.omega * (qU + fy) + src;
                f[3][k][e] = a.one_m_omega * f[3][k][e] + a.omega * (qU - fy) + src;
            }
        }

        if (act) {
            const bool full = x0 + VEC <= nx;
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    T *dst = fout + (q * 6 + k) * plane + row;
                    if (full) {
                        PK o;
#pragma unroll
                        for (int e = 0; e < VEC; ++e) o.v[e] = f[q][k][e];
                        *reinterpret_cast<PK *>(dst) = o;
                    } else {
                        // ragged end: never write past node nx - 1 (column nx is a ghost cell)
#pragma unroll
                        for (int e = 0; e < VEC; ++e)
                            if (x0 + e < nx) dst[e] = f[q][k][e];
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

            if (FUSE) {
                // ---- bottom ghost row (plane q=1, row y = -1) and top ghost row
                // (plane q=3, row y = ny): whole vectors, one per lane
                const bool ypers = a.kind[EDGE_BOTTOM] == BC_PERIODIC;
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const int e_id = side == 0 ? EDGE_BOTTOM : EDGE_TOP;
                    const int qd = side == 0 ? 1 : 3;          // missing direction
                    const int qo = side == 0 ? 3 : 1;          // outgoing direction -d
                    const int yb = side == 0 ? 0 : ny - 1;     // boundary row
                    const int ysrc = side == 0 ? ny - 1 : 0;   // periodic source row
                    const long long grow = (long long)(side == 0 ? 0 : ny + 1) * pitch + a.L.xoff + x0;
                    T *dst = fout + (long long)(qd * 6) * plane + grow;
                    if (ypers) {
                        if (y == ysrc)
#pragma unroll
                            for (int k = 0; k < 6; ++k) {
                                PK o;
#pragma unroll
                                for (int e = 0; e < VEC; ++e) o.v[e] = f[qd][k][e];
                                *reinterpret_cast<PK *>(dst + k * plane) = o;
                            }
                    } else if (y == yb) {
                        T g[6][VEC];
#pragma unroll
                        for (int e = 0; e < VEC; ++e) {
                            T out[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
                            if (x0 + e < nx) {
                                T fo[6], f0[6], f1[6], f2[6], f3[6], U[6];
#pragma unroll
                                for (int k = 0; k < 6; ++k) {
                                    fo[k] = f[qo][k][e];
                                    f0[k] = f[0][k][e]; f1[k] = f[1][k][e]; f2[k] = f[2][k][e]; f3[k] = f[3][k][e];
                                }
                                state_from_fstar(f0, f1, f2, f3, a.hdtb1, a.hdtb2, U);
                                double val[2];
                                const double gt = timefn(a.timefn[e_id], a.tp[e_id], th) *
                                                  (a.profile[e_id] ? a.profile[e_id][x0 + e] : 1.0);
                                val[0] = a.value[e_id][0] * gt;
                                val[1] = a.value[e_id][1] * gt;
                                edge_ghost<LAW, T>(e_id, a.kind[e_id], fo, U, val, a.c, a.lam, a.mu, out, flags);
                            }
#pragma unroll
                            for (int k = 0; k < 6; ++k) g[k][e] = out[k];
                        }
#pragma unroll
                        for (int k = 0; k < 6; ++k) {
                            PK o;
#pragma unroll
                            for (int e = 0; e < VEC; ++e) o.v[e] = g[k][e];
                            *reinterpret_cast<PK *>(dst + k * plane) = o;
                        }
                    }
                }
                // ---- left ghost column (plane 0, x = -1) and right ghost column
                // (plane 2, x = nx): one element of one lane per row
                const bool xpers = a.kind[EDGE_LEFT] == BC_PERIODIC;
                const long long rbase = (long long)(y + 1) * pitch + a.L.xoff;
                const int elast = nx - 1 - x0;  // element of node nx - 1 in this lane, if any
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const int e_id = side == 0 ? EDGE_LEFT : EDGE_RIGHT;
                    const int qd = side == 0 ? 0 : 2, qo = side == 0 ? 2 : 0;
                    const int gx = side == 0 ? -1 : nx;
                    // element holding the boundary node (left: x = 0, right: x = nx-1)
                    // and, for periodic edges, the source node on the opposite side
                    const int eb = side == 0 ? (x0 == 0 ? 0 : -1) : (elast >= 0 && elast < VEC ? elast : -1);
                    const int es = side == 0 ? (elast >= 0 && elast < VEC ? elast : -1) : (x0 == 0 ? 0 : -1);
                    T *dst = fout + (long long)(qd * 6) * plane + rbase + gx;
                    if (xpers) {
#pragma unroll
                        for (int e = 0; e < VEC; ++e)
                            if (e == es)
#pragma unroll
                                for (int k = 0; k < 6; ++k) dst[k * plane] = f[qd][k][e];
                    } else {
#pragma unroll
                        for (int e = 0; e < VEC; ++e)
                            if (e == eb) {
                                T fo[6], f0[6], f1[6], f2[6], f3[6], U[6], out[6];
#pragma unroll
                                for (int k = 0; k < 6; ++k) {
                                    fo[k] = f[qo][k][e];
                                    f0[k] = f[0][k][e]; f1[k] = f[1][k][e]; f2[k] = f[2][k][e]; f3[k] = f[3][k][e];
                                }
                                state_from_fstar(f0, f1, f2, f3, a.hdtb1, a.hdtb2, U);
                                double val[2];
                                const double gt = timefn(a.timefn[e_id], a.tp[e_id], th) *
                                                  (a.profile[e_id] ? a.profile[e_id][y] : 1.0);
                                val[0] = a.value[e_id][0] * gt;
                                val[1] = a.value[e_id][1] * gt;
                                edge_ghost<LAW, T>(e_id, a.kind[e_id], fo, U, val, a.c, a.lam, a.mu, out, flags);
#pragma unroll
                                for (int k = 0; k < 6; ++k) dst[k * plane] = out[k];
                            }
                    }
                }
            }
        }
    }
    flags = __reduce_or_sync(FULL_MASK, flags);
    if (flags && lane == 0) atomicOr(a.status, (int)flags);
}

// Ghost refresh in the node form (after initialization, a checkpoint load or
// new edge data): the same values the fused step writes, from the stored
// post-collision populations of the current buffer.
template <typename T, int LAW>
__global__ void __launch_bounds__(128) k_ghosts(const EdgeArgs a)
{
    T *f = static_cast<T *>(a.f);
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
        for (int k = 0; k < 6; ++k) fq[q][k] = f[idx(q, k, xb, yb)];
    state_from_fstar(fq[0], fq[1], fq[2], fq[3], (T)a.hdtb1, (T)a.hdtb2, U);
#pragma unroll
    for (int k = 0; k < 6; ++k) fo[k] = fq[md][k];
    double val[2];
    edge_value(E, s, ((double)(*a.step) + 0.5) * a.dt, val);
    unsigned flags = 0;
    edge_ghost<LAW, T>(e, E.kind, fo, U, val, (T)a.c, (T)a.m.lam, (T)a.m.mu, out, flags);
    if (flags) atomicOr(a.status, (int)flags);
#pragma unroll
    for (int k = 0; k < 6; ++k) f[idx(d, k, gx, gy)] = out[k];
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
        for (int q = 0; q < 4; ++q) s += (double)v.f[v.idx(q, k, x, y)];
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
    // edge data at t^n + dt/2 (Eq. 23); *step counts the steps already taken
    const double th = ((double)(*a.step) + 0.5) * a.dt;
    const double g = timefn(E.timefn, E.tp, th) * (E.profile ? E.profile[s] : 1.0);
    const double val[2] = {E.value[0] * g, E.value[1] * g};
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
    for (int k = 0; k < 6; ++k) v.f[v.idx(d, k, gx, gy)] = (T)(D[k] * (double)v.f[v.idx(md, k, xb, yb)] + S[k]);
}

// ---------------------------------------------------------------- launchers
template <typename T, int LAW, int VEC>
static cudaError_t launch_step_t(const StepArgs<T> &a, bool fuse, int grid, cudaStream_t st)
{
    if (fuse)
        k_step<T, LAW, VEC, true><<<grid, 128, 0, st>>>(a);
    else
        k_step<T, LAW, VEC, false><<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_step_law(int law, const StepArgs<T> &a, bool fuse, int grid, cudaStream_t st)
{
    constexpr int VEC = 16 / sizeof(T);
    switch (law) {
    case LAW_SVK: return launch_step_t<T, LAW_SVK, VEC>(a, fuse, grid, st);
    case LAW_NH: return launch_step_t<T, LAW_NH, VEC>(a, fuse, grid, st);
    default: return launch_step_t<T, LAW_LOGNH, VEC>(a, fuse, grid, st);
    }
}

cudaError_t launch_step(int storage_bytes, int law, bool fuse, const void *args, int grid, cudaStream_t st)
{
    if (storage_bytes == 8)
        return launch_step_law<double>(law, *static_cast<const StepArgs<double> *>(args), fuse, grid, st);
    return launch_step_law<float>(law, *static_cast<const StepArgs<float> *>(args), fuse, grid, st);
}

cudaError_t launch_edges(int storage_bytes, const EdgeArgs &a, int grid, cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    if (storage_bytes == 8)
        k_edges<double><<<grid, 128, 0, st>>>(a);
    else
        k_edges<float><<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_ghosts_t(const EdgeArgs &a, int grid, cudaStream_t st)
{
    switch (a.m.law) {
    case LAW_SVK: k_ghosts<T, LAW_SVK><<<grid, 128, 0, st>>>(a); break;
    case LAW_NH: k_ghosts<T, LAW_NH><<<grid, 128, 0, st>>>(a); break;
    default: k_ghosts<T, LAW_LOGNH><<<grid, 128, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_ghosts(int storage_bytes, const EdgeArgs &a, int grid, cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    return storage_bytes == 8 ? launch_ghosts_t<double>(a, grid, st) : launch_ghosts_t<float>(a, grid, st);
}

int step_blocks_per_sm(int storage_bytes, int law)
{
    int n = 0;
    const void *fn;
    if (storage_bytes == 8)
        fn = (law == LAW_SVK) ? (const void *)k_step<double, LAW_SVK, 2, true>
             : (law == LAW_NH) ? (const void *)k_step<double, LAW_NH, 2, true>
                               : (const void *)k_step<double, LAW_LOGNH, 2, true>;
    else
        fn = (law == LAW_SVK) ? (const void *)k_step<float, LAW_SVK, 4, true>
             : (law == LAW_NH) ? (const void *)k_step<float, LAW_NH, 4, true>
                               : (const void *)k_step<float, LAW_LOGNH, 4, true>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 128, 0) != cudaSuccess) n = 0;
    return n;
}

int step_vec(int storage_bytes) { return 16 / storage_bytes; }

} // namespace tlv
