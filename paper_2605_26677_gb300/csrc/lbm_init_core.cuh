// lbm_init_core.cuh -- per-node pieces of the second-order initialization
// (Sec. 3.4, Eqs. 16-21) shared by the init kernel and the adjoint's init
// step, in a compute type R: FP64 for FP64 storage and for the adjoint, FP32
// for FP32 and 16-bit storage (whose populations are rounded to FP32 or
// less anyway, and whose every step computes in FP32).
#pragma once
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace tlv {

__device__ __forceinline__ long long pidx(const Layout &L, int q, int k, int x, int y)
{
    return (long long)(q * 6 + k) * L.plane + (long long)(y + 1) * L.pitch + L.xoff + x;
}


// Second-order difference of a compact field along x (dir 0) or y (dir 1):
// central inside, wrap-around when periodic, one-sided three-point stencil at
// a non-periodic end (Sec. 3.4). h = 1 / (2 dx), computed once by the caller
// (a multiply instead of an FP64 divide per difference).
__device__ inline double fd(const double *a, int nx, int ny, int x, int y, int dir, int per, double h)
{
    const int n = dir == 0 ? nx : ny;
    const int i = dir == 0 ? x : y;
    auto at = [&](int j) { return dir == 0 ? a[(long long)y * nx + j] : a[(long long)j * nx + x]; };
    if (per) return (at((i + 1) % n) - at((i - 1 + n) % n)) * h;
    if (i == 0) return (-3.0 * at(0) + 4.0 * at(1) - at(2)) * h;
    if (i == n - 1) return (3.0 * at(n - 1) - 4.0 * at(n - 2) + at(n - 3)) * h;
    return (at(i + 1) - at(i - 1)) * h;
}

// f^eq_q(U) - f^eq_q(U_rest) of Eq. (12): U_ofs = U - U_rest (v, F - I), P the
// stress; f^eq is linear in U and in P, and P(I) = 0.
template <typename R>
__device__ __forceinline__ void feq_ofs(const R U[6], const R P[4], R c, R feq[4][6])
{
    const R PhiX[6] = {-P[0], -P[2], -U[0], R(0), -U[1], R(0)};
    const R PhiY[6] = {-P[1], -P[3], R(0), -U[0], R(0), -U[1]};
    const int ci[4] = {1, 0, -1, 0}, cj[4] = {0, 1, 0, -1};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 6; ++k) feq[q][k] = R(0.25) * (U[k] + (R(2) / c) * (ci[q] * PhiX[k] + cj[q] * PhiY[k]));
}

// f^0 - f_rest at node (x, y) in compute type R (f_rest = U_rest / 4: 1/4 in
// the F11 and F22 components, 0 elsewhere): f^eq(U0) and, for order 2, the
// correction -(dt/2) D_q f^eq of Eqs. (16)-(21), with the node's parameters.
// Returns false if det F0 <= 0.
template <typename R>
__device__ inline bool init_node_ofs(const InitArgs &a, int x, int y, const LawP<R> &m, R f[4][6])
{
    const int nx = a.L.nx, ny = a.L.ny;
    const long long N = (long long)nx * ny, n = (long long)y * nx + x;
    const int ci[4] = {1, 0, -1, 0}, cj[4] = {0, 1, 0, -1};
    const R c = (R)a.c, dt = (R)a.dt;
    R U[6];  // U0 - U_rest
#pragma unroll
    for (int k = 0; k < 6; ++k) U[k] = (R)(a.U0[k * N + n] - ((k == 2 || k == 5) ? 1.0 : 0.0));
    const R G[4] = {U[2], U[3], U[4], U[5]};
    const R F[4] = {R(1) + U[2], U[3], U[4], R(1) + U[5]};
    R P[4], dJ;
    piola_any_t<R>(a.m.law, G, m, P, dJ);
    feq_ofs<R>(U, P, c, f);
    if (a.order == 2) {
        R gX[6], gY[6], dPX[4], dPY[4];
        const double h = 0.5 / a.dx;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            gX[k] = (R)fd(a.U0 + k * N, nx, ny, x, y, 0, a.xper, h);
            gY[k] = (R)fd(a.U0 + k * N, nx, ny, x, y, 1, a.yper, h);
        }
        // d_alpha P = C : d_alpha F (text after Eq. 18), as Jacobian actions (Eq. 8)
        tangent_jvp_t<R>(a.m.law, F, gX + 2, m, dPX);
        tangent_jvp_t<R>(a.m.law, F, gY + 2, m, dPY);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const R i = (R)ci[q], j = (R)cj[q];
            R Z[6], dP[4];
            // Eq. (18): Z_q = D_q U0 with d_t U0 taken from the continuum system
            Z[0] = (R)a.b1 + dPX[0] + dPY[1] + c * i * gX[0] + c * j * gY[0];
            Z[1] = (R)a.b2 + dPX[2] + dPY[3] + c * i * gX[1] + c * j * gY[1];
            Z[2] = gX[0] + c * i * gX[2] + c * j * gY[2];
            Z[3] = gY[0] + c * i * gX[3] + c * j * gY[3];
            Z[4] = gX[1] + c * i * gX[4] + c * j * gY[4];
            Z[5] = gY[1] + c * i * gX[5] + c * j * gY[5];
            tangent_jvp_t<R>(a.m.law, F, Z + 2, m, dP); // Eq. (20)
            // Eq. (21): D_q f^eq = (f^eq)'(U0) Z_q, then Eq. (16)
            const R Dq[6] = {R(0.25) * (Z[0] - (R(2) / c) * (i * dP[0] + j * dP[1])),
                             R(0.25) * (Z[1] - (R(2) / c) * (i * dP[2] + j * dP[3])),
                             R(0.25) * (Z[2] - (R(2) * i / c) * Z[0]),
                             R(0.25) * (Z[3] - (R(2) * j / c) * Z[0]),
                             R(0.25) * (Z[4] - (R(2) * i / c) * Z[1]),
                             R(0.25) * (Z[5] - (R(2) * j / c) * Z[1])};
#pragma unroll
            for (int k = 0; k < 6; ++k) f[q][k] -= R(0.5) * dt * Dq[k];
        }
    }
    return dJ > R(-1);
}

// f^0 at node (x, y) in full (not offset) form, FP64
__device__ inline bool init_node(const InitArgs &a, int x, int y, const LawP<double> &m, double f[4][6])
{
    const bool ok = init_node_ofs<double>(a, x, y, m, f);
    for (int q = 0; q < 4; ++q) {
        f[q][2] += 0.25;
        f[q][5] += 0.25;
    }
    return ok;
}

} // namespace tlv
