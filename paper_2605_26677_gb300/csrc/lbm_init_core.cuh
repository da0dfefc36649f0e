// lbm_init_core.cuh -- per-node pieces of the second-order initialization
// (Sec. 3.4, Eqs. 16-21) shared by the init kernel and the adjoint's init
// step. FP64 whatever the storage.
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
// a non-periodic end (Sec. 3.4).
__device__ inline double fd(const double *a, int nx, int ny, int x, int y, int dir, int per, double dx)
{
    const int n = dir == 0 ? nx : ny;
    const int i = dir == 0 ? x : y;
    auto at = [&](int j) { return dir == 0 ? a[(long long)y * nx + j] : a[(long long)j * nx + x]; };
    if (per) return (at((i + 1) % n) - at((i - 1 + n) % n)) / (2.0 * dx);
    if (i == 0) return (-3.0 * at(0) + 4.0 * at(1) - at(2)) / (2.0 * dx);
    if (i == n - 1) return (3.0 * at(n - 1) - 4.0 * at(n - 2) + at(n - 3)) / (2.0 * dx);
    return (at(i + 1) - at(i - 1)) / (2.0 * dx);
}

// f^eq_q(U) of Eq. (12) in full (not offset) form
__device__ __forceinline__ void feq_full(const double U[6], const double P[4], double c, double feq[4][6])
{
    const double PhiX[6] = {-P[0], -P[2], -U[0], 0.0, -U[1], 0.0};
    const double PhiY[6] = {-P[1], -P[3], 0.0, -U[0], 0.0, -U[1]};
    const int ci[4] = {1, 0, -1, 0}, cj[4] = {0, 1, 0, -1};
    for (int q = 0; q < 4; ++q)
        for (int k = 0; k < 6; ++k) feq[q][k] = 0.25 * (U[k] + (2.0 / c) * (ci[q] * PhiX[k] + cj[q] * PhiY[k]));
}

// f^0 at node (x, y) in full (not offset) form: f^eq(U0) and, for order 2,
// the correction -(dt/2) D_q f^eq of Eqs. (16)-(21), with the node's
// parameters. Returns false if det F0 <= 0.
__device__ inline bool init_node(const InitArgs &a, int x, int y, const LawP<double> &m, double f[4][6])
{
    const int nx = a.L.nx, ny = a.L.ny;
    const long long N = (long long)nx * ny, n = (long long)y * nx + x;
    const int ci[4] = {1, 0, -1, 0}, cj[4] = {0, 1, 0, -1};
    const double c = a.c, dt = a.dt;
    double U[6];
    for (int k = 0; k < 6; ++k) U[k] = a.U0[k * N + n];
    const double F[4] = {U[2], U[3], U[4], U[5]};
    const double G[4] = {U[2] - 1.0, U[3], U[4], U[5] - 1.0};
    double P[4], dJ;
    piola_any(a.m.law, G, m, P, dJ);
    feq_full(U, P, c, f);
    if (a.order == 2) {
        double gX[6], gY[6], dPX[4], dPY[4];
        for (int k = 0; k < 6; ++k) {
            gX[k] = fd(a.U0 + k * N, nx, ny, x, y, 0, a.xper, a.dx);
            gY[k] = fd(a.U0 + k * N, nx, ny, x, y, 1, a.yper, a.dx);
        }
        // d_alpha P = C : d_alpha F (text after Eq. 18), as Jacobian actions (Eq. 8)
        tangent_jvp(a.m.law, F, gX + 2, m, dPX);
        tangent_jvp(a.m.law, F, gY + 2, m, dPY);
        for (int q = 0; q < 4; ++q) {
            const double i = ci[q], j = cj[q];
            double Z[6], dP[4];
            // Eq. (18): Z_q = D_q U0 with d_t U0 taken from the continuum system
            Z[0] = a.b1 + dPX[0] + dPY[1] + c * i * gX[0] + c * j * gY[0];
            Z[1] = a.b2 + dPX[2] + dPY[3] + c * i * gX[1] + c * j * gY[1];
            Z[2] = gX[0] + c * i * gX[2] + c * j * gY[2];
            Z[3] = gY[0] + c * i * gX[3] + c * j * gY[3];
            Z[4] = gX[1] + c * i * gX[4] + c * j * gY[4];
            Z[5] = gY[1] + c * i * gX[5] + c * j * gY[5];
            tangent_jvp(a.m.law, F, Z + 2, m, dP); // Eq. (20)
            // Eq. (21): D_q f^eq = (f^eq)'(U0) Z_q, then Eq. (16)
            const double Dq[6] = {0.25 * (Z[0] - (2.0 / c) * (i * dP[0] + j * dP[1])),
                                  0.25 * (Z[1] - (2.0 / c) * (i * dP[2] + j * dP[3])),
                                  0.25 * (Z[2] - (2.0 * i / c) * Z[0]),
                                  0.25 * (Z[3] - (2.0 * j / c) * Z[0]),
                                  0.25 * (Z[4] - (2.0 * i / c) * Z[1]),
                                  0.25 * (Z[5] - (2.0 * j / c) * Z[1])};
            for (int k = 0; k < 6; ++k) f[q][k] -= 0.5 * dt * Dq[k];
        }
    }
    return dJ > -1.0;
}

} // namespace tlv
