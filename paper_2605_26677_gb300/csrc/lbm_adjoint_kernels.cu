// lbm_adjoint_kernels.cu -- kernels of the discrete adjoint of the step
// (Sec. 3.7) for a sensor-displacement loss, with respect to the per-node
// shear modulus mu(X) (lambda = lam_ratio mu) and the initial velocity v0.
//
// Notation (offset storage as in the forward kernels): f*^n is the stored
// post-collision state after n steps, a^n = dL/df*^n (same layout), ubar =
// dL/du* (the displacement accumulator), gmu = dL/dmu.
//
// Forward step n -> n+1 at node x: f_q(x) = pull_q(f*^n) (Eq. 15; edge pulls
// read the half-way ghosts, Eqs. 23-25), U = sum_q f_q + (dt/2) B (Eq. 10),
// f*^{n+1}_q = (1 - w) f_q + w f^eq_q(U; lambda(x), mu(x)) + src (Eq. 14),
// u* += dt v. Its transpose, given a = a^{n+1}(x):
//   g   = w [ S/4 + (1/2c)(A_X^T (a_0 - a_2) + A_Y^T (a_1 - a_3)) ] + dt ubar e_v
//   h_q = (1 - w) a_q + g                       (= dL/df_q(x), every q)
//   gmu += w (1/2c) [ (a_0 - a_2) . dPhi_X/dmu + (a_1 - a_3) . dPhi_Y/dmu ]
// with S = sum_q a_q. A_X = dPhi_X/dU holds the tangent C = dP/dF (Eq. 4);
// C has major symmetry (P derives from W), so A^T acts on F through the same
// Jacobian action C : M as the forward (Eq. 8). P is linear in (lambda, mu)
// for SVK, NH and log-NH, so dP/dmu along lambda = r mu is P(F; r, 1).
// The pull becomes a push: a^n_q(x - e_q) = h_q(x). At the edges the same
// kernel applies the transposed half-way rules (velocity: a^n_{-d} = D h_d;
// traction: the same plus the implicit-function-theorem derivative of the
// Newton solve for F^b, which depends on the boundary node's tangential
// column and mu, evaluated at the F^b the forward stored in the ghost cell;
// periodic: h_d goes back to the node it was copied from).
#include "lbm_launch.cuh"
#include "lbm_init_core.cuh"
#include "lbm_step_core.cuh"

namespace tlv {

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ void ghost_cell(int e, int s, int nx, int ny, int &gx, int &gy)
{
    switch (e) {
    case EDGE_LEFT: gx = -1; gy = s; break;
    case EDGE_RIGHT: gx = nx; gy = s; break;
    case EDGE_BOTTOM: gx = s; gy = -1; break;
    default: gx = s; gy = ny; break;
    }
}

__device__ __forceinline__ bool on_traction(const int kind[4], int x, int y, int nx, int ny)
{
    return (x == 0 && kind[EDGE_LEFT] == BC_TRACTION) || (x == nx - 1 && kind[EDGE_RIGHT] == BC_TRACTION) ||
           (y == 0 && kind[EDGE_BOTTOM] == BC_TRACTION) || (y == ny - 1 && kind[EDGE_TOP] == BC_TRACTION);
}

// Traction edge e at a node with converged G^b (Sec. 3.6.2): the ghost's
// F-part S_F = G^b / 2 got the cotangent hd[2..5]. The normal column n of G^b
// solves r(n; t, mu) = N_a P_ia(G^b) - T_i = 0 with the tangential column t
// taken from the node, so (implicit function theorem) dn/dt = -Jn^{-1} Jt and
// dn/dmu = -Jn^{-1} dr/dmu. Adds the node's cotangent of G (tangential
// column) to ug and returns the mu-cotangent in dmu.
template <int LAW, typename T>
__device__ __forceinline__ void traction_ift(int e, const T Gb[4], const T hd[6], T mu, T lam_ratio, T ug[4], T &dmu)
{
    const LawP<T> mp{lam_ratio * mu, mu, T(0), T(0)};
    const int an = (e <= EDGE_RIGHT) ? 0 : 1, tc = 1 - an;
    const T Na = (e == EDGE_LEFT || e == EDGE_BOTTOM) ? T(-1) : T(1);
    T Jn[2][2], Jt[2][2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        T dF[4] = {T(0), T(0), T(0), T(0)}, dP[4];
        dF[j * 2 + an] = T(1);
        jvp_ofs<LAW, T>(Gb, dF, mp, dP);
        Jn[0][j] = Na * dP[0 * 2 + an];
        Jn[1][j] = Na * dP[1 * 2 + an];
        dF[j * 2 + an] = T(0);
        dF[j * 2 + tc] = T(1);
        jvp_ofs<LAW, T>(Gb, dF, mp, dP);
        Jt[0][j] = Na * dP[0 * 2 + an];
        Jt[1][j] = Na * dP[1 * 2 + an];
    }
    const T Gbb[4] = {T(0.5) * hd[2], T(0.5) * hd[3], T(0.5) * hd[4], T(0.5) * hd[5]};
    // z = -Jn^{-T} Gbb_normal
    const T det = Jn[0][0] * Jn[1][1] - Jn[0][1] * Jn[1][0];
    const T r0 = -Gbb[0 * 2 + an], r1 = -Gbb[1 * 2 + an];
    const T z0 = (Jn[1][1] * r0 - Jn[1][0] * r1) / det;
    const T z1 = (-Jn[0][1] * r0 + Jn[0][0] * r1) / det;
#pragma unroll
    for (int j = 0; j < 2; ++j) ug[j * 2 + tc] += Gbb[j * 2 + tc] + z0 * Jt[0][j] + z1 * Jt[1][j];
    T Pm[4], dJ;
    piola_ofs<LAW, T>(Gb[0], Gb[1], Gb[2], Gb[3], LawP<T>{lam_ratio, T(1), T(0), T(0)}, Pm[0], Pm[1], Pm[2], Pm[3],
                      dJ);
    dmu = z0 * Na * Pm[0 * 2 + an] + z1 * Na * Pm[1 * 2 + an];
}

// ---------------------------------------------------------------- main
// The part of an adjoint task after its inputs are in registers: U^{n+1}
// recovered from the pulled f*^n (U), a^{n+1} at the lane's nodes (h, which
// is overwritten by the cotangents h_q), mu, ubar and the dL/dmu accumulator
// of the lane's nodes. Adds the traction nodes' carried cotangent, applies
// the transposed collision, pushes a^n to the pulling neighbours, applies
// the transposed edge rules and stores dL/dmu.
template <typename S, int LAW, int VEC>
__device__ __forceinline__ void adj_finish(const AdjArgs<typename Prec<S>::R> &a, int y, int x0, int lane,
                                           typename Prec<S>::R (&U)[6][VEC], typename Prec<S>::R (&h)[4][6][VEC],
                                           const Pack<typename Prec<S>::R, VEC> &mu,
                                           const Pack<typename Prec<S>::R, VEC> &ub0,
                                           const Pack<typename Prec<S>::R, VEC> &ub1, Pack<double, VEC> gm)
{
    using T = typename Prec<S>::R;
    using PK = Pack<S, VEC>;
    using PD = Pack<double, VEC>;
    const int nx = a.L.nx, ny = a.L.ny;
    const long long plane = a.L.plane;
    const int pitch = a.L.pitch;
    const S *__restrict__ fin = static_cast<const S *>(a.fin);
    S *__restrict__ aout = static_cast<S *>(a.aout);
    const bool act = x0 < nx;
    const long long row = (long long)(y + 1) * pitch + a.L.xoff + x0;
    const long long urow = (long long)y * a.L.upitch + x0;
    // the traction edges' cotangent of U at their nodes, left by the
    // previous (later-in-time) step for every q
    if (act) {
#pragma unroll
        for (int e = 0; e < VEC; ++e)
            if (x0 + e < nx && on_traction(a.kind, x0 + e, y, nx, ny))
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const T u = a.tug_in[m * a.L.uplane + urow + e];
#pragma unroll
                    for (int q = 0; q < 4; ++q) h[q][2 + m][e] += u;
                }
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        T Sa[6], bX[6], bY[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            Sa[k] = (h[0][k][e] + h[2][k][e]) + (h[1][k][e] + h[3][k][e]);
            bX[k] = h[0][k][e] - h[2][k][e];
            bY[k] = h[1][k][e] - h[3][k][e];
        }
        const T G[4] = {U[2][e], U[3][e], U[4][e], U[5][e]};
        const T M[4] = {bX[0], bY[0], bX[1], bY[1]};  // cotangent of (P11, P12, P21, P22)
        const LawP<T> mp{a.lam_ratio * mu.v[e], mu.v[e], T(0), T(0)};
        const LawP<T> unit{a.lam_ratio, T(1), T(0), T(0)};  // d(lambda, mu)/dmu
        T CM[4], Pm[4], dJ;
        jvp_ofs<LAW, T>(G, M, mp, CM);
        piola_ofs<LAW, T>(G[0], G[1], G[2], G[3], unit, Pm[0], Pm[1], Pm[2], Pm[3], dJ);
        T g[6];
        g[0] = a.wq * Sa[0] - a.wi2c * (bX[2] + bY[3]) + a.dtT * ub0.v[e];
        g[1] = a.wq * Sa[1] - a.wi2c * (bX[4] + bY[5]) + a.dtT * ub1.v[e];
#pragma unroll
        for (int j = 0; j < 4; ++j) g[2 + j] = a.wq * Sa[2 + j] - a.wi2c * CM[j];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 6; ++k) h[q][k][e] = a.one_m_omega * h[q][k][e] + g[k];
        // the step's dL/dmu term is formed in the compute type and only
        // accumulated over the run in FP64 (on GB300 FP64 instructions are
        // scarce: forming it in FP64 kept the FP64 pipe 42% busy)
        if (x0 + e < nx) {
            if constexpr (sizeof(T) == 4)
                gm.v[e] -= (double)(a.wi2c * (M[0] * Pm[0] + M[1] * Pm[1] + M[2] * Pm[2] + M[3] * Pm[3]));
            else
                gm.v[e] -= a.wi2c_d * (M[0] * Pm[0] + M[1] * Pm[1] + M[2] * Pm[2] + M[3] * Pm[3]);
        }
    }

    // pushes: a^n_q(x - e_q) = h_q(x); what would leave the domain is
    // handled by the edge rules below
    const bool full = act && x0 + VEC <= nx;
    const bool ylo = (y == 0), yhi = (y == ny - 1);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        // q = 1 to row y - 1 and q = 3 to row y + 1, inside the domain
        if (act) {
            S *d1 = aout + (1 * 6 + k) * plane + row - pitch;
            S *d3 = aout + (3 * 6 + k) * plane + row + pitch;
            if (full) {
                PK o1, o3;
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    o1.v[e] = to_store<S>(h[1][k][e]);
                    o3.v[e] = to_store<S>(h[3][k][e]);
                }
                if (!ylo) *reinterpret_cast<PK *>(d1) = o1;
                if (!yhi) *reinterpret_cast<PK *>(d3) = o3;
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (x0 + e < nx) {
                        if (!ylo) d1[e] = to_store<S>(h[1][k][e]);
                        if (!yhi) d3[e] = to_store<S>(h[3][k][e]);
                    }
            }
        }
        // q = 0 to column x - 1: position p = x0 + e takes h_0(p + 1), p <= nx - 2
        {
            const T nxt = __shfl_down_sync(FULL_MASK, h[0][k][0], 1);
            S *d0 = aout + (0 * 6 + k) * plane + row;
            bool all = true;
#pragma unroll
            for (int e = 0; e < VEC; ++e) all = all && (x0 + e <= nx - 2) && !(lane == 31 && e == VEC - 1);
            if (all) {
                PK o;
#pragma unroll
                for (int e = 0; e < VEC; ++e) o.v[e] = to_store<S>(e < VEC - 1 ? h[0][k][e + 1] : nxt);
                *reinterpret_cast<PK *>(d0) = o;
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (x0 + e <= nx - 2 && !(lane == 31 && e == VEC - 1))
                        d0[e] = to_store<S>(e < VEC - 1 ? h[0][k][e + 1] : nxt);
            }
            if (lane == 0 && act && x0 >= 1) d0[-1] = to_store<S>(h[0][k][0]);  // the previous segment's last position
        }
        // q = 2 to column x + 1: position p = x0 + e takes h_2(p - 1), 1 <= p <= nx - 1
        {
            const T prv = __shfl_up_sync(FULL_MASK, h[2][k][VEC - 1], 1);
            S *d2 = aout + (2 * 6 + k) * plane + row;
            bool all = true;
#pragma unroll
            for (int e = 0; e < VEC; ++e) all = all && (x0 + e >= 1) && (x0 + e <= nx - 1) && !(lane == 0 && e == 0);
            if (all) {
                PK o;
#pragma unroll
                for (int e = 0; e < VEC; ++e) o.v[e] = to_store<S>(e == 0 ? prv : h[2][k][e - 1]);
                *reinterpret_cast<PK *>(d2) = o;
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (x0 + e >= 1 && x0 + e <= nx - 1 && !(lane == 0 && e == 0))
                        d2[e] = to_store<S>(e == 0 ? prv : h[2][k][e - 1]);
            }
            if (lane == 31 && x0 + VEC <= nx - 1) d2[VEC] = to_store<S>(h[2][k][VEC - 1]);  // the next segment's first
        }
    }

    // Edge rules, transposed (Eqs. 23-25), at the lane's boundary nodes.
    // The node x_b pulled f_d(x_b) = D f*_{-d}(x_b) + S_d(U^n(x_b)) (or, on a
    // periodic edge, the opposite node's f*_d), so its h_d goes to
    // a^n_{-d}(x_b) with D (or back to that opposite node). A traction
    // edge adds the implicit-function derivative of F^b, which reaches
    // every q of x_b through U^n = sum_q f*^n_q: its F-part is left in
    // tug_out for the next step to add, and its mu-part goes to dL/dmu.
    // No other thread writes the cells written here.
    if (act && (ylo || yhi || x0 == 0 || x0 + VEC >= nx)) {
        T ug[VEC][4];
        bool tr[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            tr[e] = false;
#pragma unroll
            for (int m = 0; m < 4; ++m) ug[e][m] = T(0);
        }
#pragma unroll
        for (int ed = 0; ed < 4; ++ed) {
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int x = x0 + e;
                if (x >= nx) continue;
                const bool on = (ed == EDGE_LEFT) ? x == 0 : (ed == EDGE_RIGHT) ? x == nx - 1 : (ed == EDGE_BOTTOM) ? ylo : yhi;
                if (!on) continue;
                const int d = edge_dmiss(ed), md = edge_dout(ed);
                T hd[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) hd[k] = h[d][k][e];
                if (a.kind[ed] == BC_PERIODIC) {
                    const int tx = (ed == EDGE_LEFT) ? nx - 1 : (ed == EDGE_RIGHT) ? 0 : x;
                    const int ty = (ed == EDGE_BOTTOM) ? ny - 1 : (ed == EDGE_TOP) ? 0 : y;
                    const long long cell = (long long)(ty + 1) * pitch + a.L.xoff + tx;
#pragma unroll
                    for (int k = 0; k < 6; ++k) aout[(d * 6 + k) * plane + cell] = to_store<S>(hd[k]);
                    continue;
                }
                const T sv = (a.kind[ed] == BC_VELOCITY) ? T(-1) : T(1);  // D on (v1, v2); -sv on F
#pragma unroll
                for (int k = 0; k < 6; ++k) aout[(md * 6 + k) * plane + row + e] = to_store<S>((k < 2 ? sv : -sv) * hd[k]);
                if (a.kind[ed] != BC_TRACTION) continue;
                tr[e] = true;
                // the forward stored ghost = -f*_{-d} + G^b / 2 on the F-components
                int gx, gy;
                ghost_cell(ed, (ed <= EDGE_RIGHT) ? y : x, nx, ny, gx, gy);
                const long long gcell = (long long)(gy + 1) * pitch + a.L.xoff + gx;
                T Gb[4];
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    Gb[m] = T(2) * (ld_r(fin[(d * 6 + 2 + m) * plane + gcell]) + ld_r(fin[(md * 6 + 2 + m) * plane + row + e]));
                T dmu;
                traction_ift<LAW, T>(ed, Gb, hd, mu.v[e], a.lam_ratio, ug[e], dmu);
                gm.v[e] += (double)dmu;
            }
        }
#pragma unroll
        for (int e = 0; e < VEC; ++e)
            if (tr[e])
#pragma unroll
                for (int m = 0; m < 4; ++m) a.tug_out[m * a.L.uplane + urow + e] = ug[e][m];
    }
    if (act) *reinterpret_cast<PD *>(a.gmu + urow) = gm;
}

// FP32: every load of a task is issued before the shifts and sums that use
// them (about 13.6 KB per warp in flight at once; 127 registers, 4 blocks
// per SM), which cut the backward step by 3% against loading and summing
// one component at a time. FP64 keeps the component-at-a-time order: its
// loads would need twice the registers.
// NS: 0 static task order, else dynamic claims over NS stripes (claim_tasks)
template <typename S, int LAW, int VEC, int NS = 0>
__global__ void __launch_bounds__(128, sizeof(S) == 4 ? 4 : 1) k_adj(const AdjArgs<typename Prec<S>::R> a)
{
    constexpr bool EARLY = sizeof(S) == 4;
    pdl_enter();
    using T = typename Prec<S>::R;
    using PK = Pack<S, VEC>;
    using PT = Pack<T, VEC>;
    using PD = Pack<double, VEC>;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int nx = a.L.nx, ny = a.L.ny;
    const int segw = 32 * VEC;
    const int nseg = (nx + segw - 1) / segw;
    const int ntask = ny * nseg;
    const long long plane = a.L.plane;
    const int pitch = a.L.pitch;
    const S *__restrict__ fin = static_cast<const S *>(a.fin);
    const S *__restrict__ ain = static_cast<const S *>(a.ain);

    auto body = [&](int task) {
        int y, seg;
        task_coords(task, nseg, ny, y, seg);
        const int x0 = seg * segw + lane * VEC;
        const bool act = x0 < nx;
        const bool ld0 = x0 <= nx;
        const long long row = (long long)(y + 1) * pitch + a.L.xoff + x0;
        const long long urow = (long long)y * a.L.upitch + x0;

        T U[6][VEC];
        T h[4][6][VEC];
        PT mu = {}, ub0 = {}, ub1 = {};
        PD gm = {};
        if constexpr (EARLY) {
            // every load of the task first, so that all of them are in flight
            // together, then the shifts and sums
            PK c0[6], c1[6], c2[6], c3[6], av[4][6];
            T lft[6], rgt[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                c0[k] = PK{};
                c1[k] = PK{};
                c2[k] = PK{};
                c3[k] = PK{};
                lft[k] = T(0);
                rgt[k] = T(0);
                if (ld0) {
                    c0[k] = *reinterpret_cast<const PK *>(fin + (0 * 6 + k) * plane + row);
                    c2[k] = *reinterpret_cast<const PK *>(fin + (2 * 6 + k) * plane + row);
                }
                if (act) {
                    c1[k] = *reinterpret_cast<const PK *>(fin + (1 * 6 + k) * plane + row - pitch);
                    c3[k] = *reinterpret_cast<const PK *>(fin + (3 * 6 + k) * plane + row + pitch);
                    if (lane == 0) lft[k] = ld_r(fin[(0 * 6 + k) * plane + row - 1]);
                    if (lane == 31) rgt[k] = ld_r(fin[(2 * 6 + k) * plane + row + VEC]);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    av[q][k] = PK{};
                    if (act) av[q][k] = *reinterpret_cast<const PK *>(ain + (q * 6 + k) * plane + row);
                }
            if (act) {
                mu = *reinterpret_cast<const PT *>(a.mufield + urow);
                ub0 = *reinterpret_cast<const PT *>(a.ubar + urow);
                ub1 = *reinterpret_cast<const PT *>(a.ubar + a.L.uplane + urow);
                gm = *reinterpret_cast<const PD *>(a.gmu + urow);
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                T left = __shfl_up_sync(FULL_MASK, ld_r(c0[k].v[VEC - 1]), 1);
                T right = __shfl_down_sync(FULL_MASK, ld_r(c2[k].v[0]), 1);
                if (act && lane == 0) left = lft[k];
                if (act && lane == 31) right = rgt[k];
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const T f0 = (e == 0) ? left : ld_r(c0[k].v[e - 1]);
                    const T f2 = (e == VEC - 1) ? right : ld_r(c2[k].v[e + 1]);
                    U[k][e] = (f0 + f2) + (ld_r(c1[k].v[e]) + ld_r(c3[k].v[e]));
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 6; ++k)
#pragma unroll
                    for (int e = 0; e < VEC; ++e) h[q][k][e] = ld_r(av[q][k].v[e]);
        } else {
            // U^{n+1} of the lane's nodes from the pulled populations
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
                    const T f0 = (e == 0) ? left : ld_r(c0.v[e - 1]);
                    const T f2 = (e == VEC - 1) ? right : ld_r(c2.v[e + 1]);
                    U[k][e] = (f0 + f2) + (ld_r(c1.v[e]) + ld_r(c3.v[e]));
                }
            }
            // a^{n+1} at the lane's own nodes; h overwrites it in place
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    PK v = {};
                    if (act) v = *reinterpret_cast<const PK *>(ain + (q * 6 + k) * plane + row);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) h[q][k][e] = ld_r(v.v[e]);
                }
            if (act) {
                mu = *reinterpret_cast<const PT *>(a.mufield + urow);
                ub0 = *reinterpret_cast<const PT *>(a.ubar + urow);
                ub1 = *reinterpret_cast<const PT *>(a.ubar + a.L.uplane + urow);
                gm = *reinterpret_cast<const PD *>(a.gmu + urow);
            }
        }
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            U[0][e] += a.hdtb1;
            U[1][e] += a.hdtb2;
        }
        adj_finish<S, LAW, VEC>(a, y, x0, lane, U, h, mu, ub0, ub1, gm);
    };
    if constexpr (NS > 0) {
        if (blockIdx.x == 0 && threadIdx.x < DYN_STRIPES) a.ctr_next[threadIdx.x * DYN_CTR_STRIDE] = 0u;
        claim_tasks<NS>(a.ctr, ntask, lane, body);
    } else {
        for (int task = gw; task < ntask; task += nw) body(task);
    }
}

// ---------------------------------------------------------------- sensors
// u^n at the sensors, exactly as the read-out computes it
template <typename S>
__global__ void k_adj_record(const RecordArgs a)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.nsens) return;
    const S *f = static_cast<const S *>(a.f);
    const int x = a.sens[2 * s], y = a.sens[2 * s + 1];
    const long long base = (long long)(y + 1) * a.L.pitch + a.L.xoff + x;
    const long long ui = (long long)y * a.L.upitch + x;
    for (int c = 0; c < 2; ++c) {
        double sum = 0.0;
        for (int q = 0; q < 4; ++q) sum += (double)ld_r(f[(long long)(q * 6 + c) * a.L.plane + base]);
        const double v = sum - 0.5 * a.dt * (c == 0 ? a.b1 : a.b2);
        a.out[2 * s + c] = a.ustar[c * a.L.uplane + ui] - 0.5 * a.dt * v;
    }
}

// loss terms of recorded step n: r = u^n - d at each sensor; u^n = u* - (dt/2) v^n
template <typename S>
__global__ void k_adj_inject(const InjectArgs<typename Prec<S>::R> a)
{
    using T = typename Prec<S>::R;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.nsens) return;
    S *f = static_cast<S *>(a.aout);
    const int x = a.sens[2 * s], y = a.sens[2 * s + 1];
    const long long base = (long long)(y + 1) * a.L.pitch + a.L.xoff + x;
    const long long ui = (long long)y * a.L.upitch + x;
    for (int c = 0; c < 2; ++c) {
        const double r = a.rec[2 * s + c] - a.tgt[2 * s + c];
        a.ubar[c * a.L.uplane + ui] += (T)r;
        for (int q = 0; q < 4; ++q) {
            const long long i = (long long)(q * 6 + c) * a.L.plane + base;
            f[i] = to_store<S>(ld_r(f[i]) + (T)(-0.5 * a.dt * r));
        }
    }
}

// ---------------------------------------------------------------- init
// Transpose of the step-0 collision and of f^0 = f^eq(U0) - (dt/2) D f^eq
// (Eqs. 16-21) at each node, in FP64. f^0 is linear in v0 and affine in
// (lambda, mu); its mu-derivative along lambda = r mu is f^0(r, 1) - f^0(0, 0).
// The cotangents of the finite-difference gradients of v0 go to ghat for the
// transposed stencil of k_adj_init_fd.
template <typename S>
__global__ void __launch_bounds__(128) k_adj_init(const AdjInitArgs a)
{
    using T = typename Prec<S>::R;
    const InitArgs &ia = a.ia;
    const int nx = ia.L.nx, ny = ia.L.ny;
    const long long N = (long long)nx * ny;
    const S *a0 = static_cast<const S *>(a.a0);
    const T *ubar = static_cast<const T *>(a.ubar);
    const int ci[4] = {1, 0, -1, 0}, cj[4] = {0, 1, 0, -1};
    const double c = ia.c, dt = ia.dt, w = ia.omega, wi2c = w * 0.5 / c;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % nx), y = (int)(n / nx);
        double f0[4][6];
        const LawP<double> mp = law_at(ia.m, n);
        init_node(ia, x, y, mp, f0);
        double Un[6];
        for (int k = 0; k < 6; ++k) Un[k] = f0[0][k] + f0[1][k] + f0[2][k] + f0[3][k];
        Un[0] += 0.5 * dt * ia.b1;
        Un[1] += 0.5 * dt * ia.b2;
        const double Fn[4] = {Un[2], Un[3], Un[4], Un[5]};
        const double Gn[4] = {Un[2] - 1.0, Un[3], Un[4], Un[5] - 1.0};
        const long long ui = (long long)y * ia.L.upitch + x;
        double h[4][6], Sa[6], bX[6], bY[6];
        for (int q = 0; q < 4; ++q)
            for (int k = 0; k < 6; ++k) h[q][k] = (double)ld_r(a0[pidx(ia.L, q, k, x, y)]);
        if (on_traction(a.kind, x, y, nx, ny))
            for (int m = 0; m < 4; ++m) {
                const double u = (double)static_cast<const T *>(a.tug)[m * ia.L.uplane + ui];
                for (int q = 0; q < 4; ++q) h[q][2 + m] += u;
            }
        for (int k = 0; k < 6; ++k) {
            Sa[k] = (h[0][k] + h[2][k]) + (h[1][k] + h[3][k]);
            bX[k] = h[0][k] - h[2][k];
            bY[k] = h[1][k] - h[3][k];
        }
        const double ub[2] = {(double)ubar[ui], (double)ubar[ia.L.uplane + ui]};
        const double M[4] = {bX[0], bY[0], bX[1], bY[1]};
        double CM[4], Pm[4], dJ;
        const LawP<double> unit{ia.m.lam_ratio, 1.0, 0.0, 0.0};  // d(lambda, mu)/dmu
        tangent_jvp(ia.m.law, Fn, M, mp, CM);
        piola_any(ia.m.law, Gn, unit, Pm, dJ);
        double g[6];
        g[0] = 0.25 * w * Sa[0] - wi2c * (bX[2] + bY[3]) + dt * ub[0];
        g[1] = 0.25 * w * Sa[1] - wi2c * (bX[4] + bY[5]) + dt * ub[1];
        for (int j = 0; j < 4; ++j) g[2 + j] = 0.25 * w * Sa[2 + j] - wi2c * CM[j];
        for (int q = 0; q < 4; ++q)
            for (int k = 0; k < 6; ++k) h[q][k] = (1.0 - w) * h[q][k] + g[k];
        // mu: the step-0 collision and f^0 itself
        double gm = -wi2c * (M[0] * Pm[0] + M[1] * Pm[1] + M[2] * Pm[2] + M[3] * Pm[3]);
        {
            double fR[4][6], fZ[4][6];
            init_node(ia, x, y, unit, fR);
            init_node(ia, x, y, LawP<double>{0.0, 0.0, 0.0, 0.0}, fZ);
            for (int q = 0; q < 4; ++q)
                for (int k = 0; k < 6; ++k) gm += h[q][k] * (fR[q][k] - fZ[q][k]);
        }
        a.gmu[ui] += gm;
        // v0: f^eq(U0) at the node, and u*^0 = u0 - (dt/2) v0 + dt v^0
        double gv[2] = {-0.5 * dt * ub[0], -0.5 * dt * ub[1]};
        for (int q = 0; q < 4; ++q) {
            gv[0] += 0.25 * (h[q][0] - (2.0 / c) * (ci[q] * h[q][2] + cj[q] * h[q][3]));
            gv[1] += 0.25 * (h[q][1] - (2.0 / c) * (ci[q] * h[q][4] + cj[q] * h[q][5]));
        }
        a.gv0[n] = gv[0];
        a.gv0[N + n] = gv[1];
        // v0 through the gradients in D_q (order 2): Db_q = -(dt/2) h_q
        double gh[4] = {0.0, 0.0, 0.0, 0.0};  // d/d(dX v1, dX v2, dY v1, dY v2)
        if (ia.order == 2) {
            double F0[4];
            for (int m = 0; m < 4; ++m) F0[m] = ia.U0[(2 + m) * N + n];
            for (int q = 0; q < 4; ++q) {
                const double i = ci[q], j = cj[q];
                double Db[6], Zb[6], dPb[4], CdP[4];
                for (int k = 0; k < 6; ++k) Db[k] = -0.5 * dt * h[q][k];
                for (int k = 0; k < 6; ++k) Zb[k] = 0.25 * Db[k];
                Zb[0] += -0.25 * (2.0 * i / c) * Db[2] - 0.25 * (2.0 * j / c) * Db[3];
                Zb[1] += -0.25 * (2.0 * i / c) * Db[4] - 0.25 * (2.0 * j / c) * Db[5];
                dPb[0] = -0.25 * (2.0 / c) * i * Db[0];
                dPb[1] = -0.25 * (2.0 / c) * j * Db[0];
                dPb[2] = -0.25 * (2.0 / c) * i * Db[1];
                dPb[3] = -0.25 * (2.0 / c) * j * Db[1];
                tangent_jvp(ia.m.law, F0, dPb, mp, CdP);  // C^T = C
                for (int m = 0; m < 4; ++m) Zb[2 + m] += CdP[m];
                gh[0] += c * i * Zb[0] + Zb[2];
                gh[1] += c * i * Zb[1] + Zb[4];
                gh[2] += c * j * Zb[0] + Zb[3];
                gh[3] += c * j * Zb[1] + Zb[5];
            }
        }
        for (int m = 0; m < 4; ++m) a.ghat[m * N + n] = gh[m];
    }
}

// transpose of the second-order differences of Sec. 3.4 (central inside,
// wrap-around when periodic, one-sided three-point stencils at the ends)
__device__ __forceinline__ double fd_t(const double *g, int nx, int ny, int x, int y, int dir, int per, double dx)
{
    const int n = dir == 0 ? nx : ny;
    const int i = dir == 0 ? x : y;
    auto at = [&](int j) { return dir == 0 ? g[(long long)y * nx + j] : g[(long long)j * nx + x]; };
    double s = 0.0;
    if (per) {
        s = at((i - 1 + n) % n) - at((i + 1) % n);
    } else {
        if (i - 1 >= 1 && i - 1 <= n - 2) s += at(i - 1);
        if (i + 1 >= 1 && i + 1 <= n - 2) s -= at(i + 1);
        if (i == 0) s += -3.0 * at(0);
        if (i == 1) s += 4.0 * at(0);
        if (i == 2) s += -1.0 * at(0);
        if (i == n - 1) s += 3.0 * at(n - 1);
        if (i == n - 2) s += -4.0 * at(n - 1);
        if (i == n - 3) s += 1.0 * at(n - 1);
    }
    return s / (2.0 * dx);
}

__global__ void k_adj_init_fd(const AdjInitArgs a)
{
    const InitArgs &ia = a.ia;
    const int nx = ia.L.nx, ny = ia.L.ny;
    const long long N = (long long)nx * ny;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % nx), y = (int)(n / nx);
        for (int c = 0; c < 2; ++c)
            a.gv0[c * N + n] += fd_t(a.ghat + c * N, nx, ny, x, y, 0, ia.xper, ia.dx) +
                                fd_t(a.ghat + (2 + c) * N, nx, ny, x, y, 1, ia.yper, ia.dx);
    }
}

__global__ void k_plane_to_compact(const double *plane, double *out, Layout L)
{
    const long long N = (long long)L.nx * L.ny;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % L.nx), y = (int)(n / L.nx);
        out[n] = plane[(long long)y * L.upitch + x];
    }
}

// ---------------------------------------------------------------- launchers
static int grid_for(long long n, int block, int cap = 8192)
{
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    return (int)(g < cap ? g : cap);
}

// nodes per lane of the adjoint kernel (FP64, FP32 storage)
#ifndef ADJ_VEC32
#define ADJ_VEC32 2
#endif
template <typename S>
constexpr int adj_vec()
{
    return sizeof(S) == 8 ? 2 : ADJ_VEC32;
}

template <typename S, int LAW>
static cudaError_t launch_adj_t(const void *args, int grid, cudaStream_t st)
{
    using T = typename Prec<S>::R;
    const auto &a = *static_cast<const AdjArgs<T> *>(args);
    if constexpr (sizeof(S) == 4) {
        if (a.ctr && a.dyn_ns == 1) return launch_pdl(k_adj<S, LAW, adj_vec<S>(), 1>, grid, 128, 0, st, a);
        if (a.ctr) return launch_pdl(k_adj<S, LAW, adj_vec<S>(), DYN_STRIPES>, grid, 128, 0, st, a);
    }
    return launch_pdl(k_adj<S, LAW, adj_vec<S>()>, grid, 128, 0, st, a);
}

template <typename S>
static cudaError_t launch_adj_s(int law, const void *args, int grid, cudaStream_t st)
{
    switch (law) {
    case LAW_SVK: return launch_adj_t<S, LAW_SVK>(args, grid, st);
    case LAW_NH: return launch_adj_t<S, LAW_NH>(args, grid, st);
    default: return launch_adj_t<S, LAW_LOGNH>(args, grid, st);
    }
}

int adj_vec_for(int storage) { return storage == STORE_F64 ? adj_vec<double>() : adj_vec<float>(); }

cudaError_t launch_adj(int storage, int law, const void *args, int grid, cudaStream_t st)
{
    if (storage == STORE_F64) return launch_adj_s<double>(law, args, grid, st);
    if (storage == STORE_F32) return launch_adj_s<float>(law, args, grid, st);
    return cudaErrorNotSupported;
}

int adj_blocks_per_sm(int storage, int law)
{
    const void *fn;
    if (storage == STORE_F64)
        fn = law == LAW_SVK ? (const void *)k_adj<double, LAW_SVK, 2>
             : law == LAW_NH ? (const void *)k_adj<double, LAW_NH, 2> : (const void *)k_adj<double, LAW_LOGNH, 2>;
    else
        fn = law == LAW_SVK ? (const void *)k_adj<float, LAW_SVK, adj_vec<float>()>
             : law == LAW_NH ? (const void *)k_adj<float, LAW_NH, adj_vec<float>()>
                             : (const void *)k_adj<float, LAW_LOGNH, adj_vec<float>()>;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 128, 0) != cudaSuccess) n = 0;
    return n;
}

cudaError_t launch_adj_record(int storage, const RecordArgs &a, cudaStream_t st)
{
    if (a.nsens <= 0) return cudaSuccess;
    const int grid = (a.nsens + 127) / 128;
    if (storage == STORE_F64)
        k_adj_record<double><<<grid, 128, 0, st>>>(a);
    else
        k_adj_record<float><<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adj_inject(int storage, const void *args, cudaStream_t st)
{
    if (storage == STORE_F64) {
        const auto &a = *static_cast<const InjectArgs<double> *>(args);
        if (a.nsens > 0) k_adj_inject<double><<<(a.nsens + 127) / 128, 128, 0, st>>>(a);
    } else {
        const auto &a = *static_cast<const InjectArgs<float> *>(args);
        if (a.nsens > 0) k_adj_inject<float><<<(a.nsens + 127) / 128, 128, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_init(int storage, const AdjInitArgs &a, cudaStream_t st)
{
    const long long N = (long long)a.ia.L.nx * a.ia.L.ny;
    const int grid = grid_for(N, 128);
    if (storage == STORE_F64)
        k_adj_init<double><<<grid, 128, 0, st>>>(a);
    else
        k_adj_init<float><<<grid, 128, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adj_init_fd<<<grid_for(N, 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_plane_to_compact(const double *plane, double *out, const Layout &L, cudaStream_t st)
{
    const long long N = (long long)L.nx * L.ny;
    k_plane_to_compact<<<grid_for(N, 256), 256, 0, st>>>(plane, out, L);
    return cudaGetLastError();
}

} // namespace tlv
