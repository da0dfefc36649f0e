// lbm_edges.cuh -- half-way edge reconstruction shared by the fused step
// kernel and the ghost-refresh kernel (Sec. 3.6, Eqs. 23-25).
//
// For a boundary node x_b of edge e the missing incoming direction is d = -N;
// the value it pulls at the next step is f_d = D f*_{-d}(x_b) + S_d(t + dt/2),
// written into the ghost cell x_b + N of plane d. In offset storage (values
// minus f_rest = (0, 0, 1/4, 0, 0, 1/4)) the velocity rule keeps S as is (its
// F-components have D = +1) and the traction rule's F-source becomes
// (F^b - I)/2 = G^b/2 (D = -1 on the F-components).
#pragma once
#include "lbm_device.cuh"

namespace tlv {

// missing direction d and outgoing direction -d = N per edge
__host__ __device__ constexpr int edge_dmiss(int e) { return e == EDGE_LEFT ? 0 : e == EDGE_RIGHT ? 2 : e == EDGE_BOTTOM ? 1 : 3; }
__host__ __device__ constexpr int edge_dout(int e) { return e == EDGE_LEFT ? 2 : e == EDGE_RIGHT ? 0 : e == EDGE_BOTTOM ? 3 : 1; }

// Newton tolerance on the traction residual: the paper's FP64 setting
// 1e-13 max(1, |T|); in FP32 the offset stress has a rounding floor of about
// eps |P| ~ 6e-8 (|T| + mu |G^b|), and 4e-6 times that scale is reachable.
template <typename R>
__device__ __forceinline__ R newton_tol(R tmax, R mu, R gmax);
template <>
__device__ __forceinline__ double newton_tol<double>(double tmax, double, double)
{
    return 1e-13 * (tmax > 1.0 ? tmax : 1.0);
}
template <>
__device__ __forceinline__ float newton_tol<float>(float tmax, float mu, float gmax)
{
    return 4e-6f * (tmax + mu * gmax) + 1e-30f;
}

// dP = C : dF (Eq. 8) in precision R, from G = F - I
template <int LAW, typename R>
__device__ __forceinline__ void jvp_ofs(const R G[4], const R dF[4], const LawP<R> &m, R dP[4])
{
    if (LAW >= LAW_MR) {
        jvp_inv<LAW, R>(G, dF, m, dP);
        return;
    }
    const R lam = m.lam, mu = m.mu;
    const R F[4] = {R(1) + G[0], G[1], G[2], R(1) + G[3]};
    if (LAW == LAW_SVK) {
        const R E11 = G[0] + R(0.5) * (G[0] * G[0] + G[2] * G[2]);
        const R E22 = G[3] + R(0.5) * (G[1] * G[1] + G[3] * G[3]);
        const R E12 = R(0.5) * (G[1] + G[2] + G[0] * G[1] + G[2] * G[3]);
        const R trE = E11 + E22;
        const R S11 = lam * trE + R(2) * mu * E11, S22 = lam * trE + R(2) * mu * E22, S12 = R(2) * mu * E12;
        const R dE11 = dF[0] * F[0] + dF[2] * F[2];
        const R dE22 = dF[1] * F[1] + dF[3] * F[3];
        const R dE12 = R(0.5) * (dF[0] * F[1] + dF[2] * F[3] + F[0] * dF[1] + F[2] * dF[3]);
        const R dtr = dE11 + dE22;
        const R dS11 = lam * dtr + R(2) * mu * dE11, dS22 = lam * dtr + R(2) * mu * dE22, dS12 = R(2) * mu * dE12;
        dP[0] = dF[0] * S11 + dF[1] * S12 + F[0] * dS11 + F[1] * dS12;
        dP[1] = dF[0] * S12 + dF[1] * S22 + F[0] * dS12 + F[1] * dS22;
        dP[2] = dF[2] * S11 + dF[3] * S12 + F[2] * dS11 + F[3] * dS12;
        dP[3] = dF[2] * S12 + dF[3] * S22 + F[2] * dS12 + F[3] * dS22;
        return;
    }
    const R dJ = G[0] + G[3] + (G[0] * G[3] - G[1] * G[2]);
    const R J = R(1) + dJ;
    const R invJ = R(1) / J;
    const R H[4] = {F[3] * invJ, -F[2] * invJ, -F[1] * invJ, F[0] * invJ};
    const R HdF = H[0] * dF[0] + H[1] * dF[1] + H[2] * dF[2] + H[3] * dF[3];
    R a, b;
    if (LAW == LAW_NH) {
        a = lam * J * J;
        b = mu - R(0.5) * lam * dJ * (R(2) + dJ);
    } else {
        a = lam;
        b = mu - lam * log1p(dJ);
    }
    // (H dF^T H)_iA = sum_{B,k} H_iB dF_kB H_kA
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int A = 0; A < 2; ++A) {
            R s = R(0);
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int B = 0; B < 2; ++B) s += H[i * 2 + B] * dF[k * 2 + B] * H[k * 2 + A];
            dP[i * 2 + A] = mu * dF[i * 2 + A] + a * HdF * H[i * 2 + A] + b * s;
        }
}

// Sec. 3.6.2 in the paper's (node) form: G^b takes its tangential column from
// the boundary node; its normal column solves N_a P_ia(F^b) = T_i by Newton
// (at most 20 steps, halving line search that rejects det F^b <= 0 and keeps
// only decreasing |r|). G holds F - I at the node; the result replaces it.
// Returns false if the tolerance was not reached.
template <int LAW, typename R>
__device__ bool traction_newton(int e, R G[4], const R Tb[2], const LawP<R> &m)
{
    const R mus = shear_scale<LAW, R>(m);
    const int an = (e <= EDGE_RIGHT) ? 0 : 1;
    const R Na = (e == EDGE_LEFT || e == EDGE_BOTTOM) ? R(-1) : R(1);
    R P[4], dJ, r[2];
    piola_ofs<LAW, R>(G[0], G[1], G[2], G[3], m, P[0], P[1], P[2], P[3], dJ);
    r[0] = Na * P[0 * 2 + an] - Tb[0];
    r[1] = Na * P[1 * 2 + an] - Tb[1];
    const R tmax = fmax(fabs(Tb[0]), fabs(Tb[1]));
    for (int it = 0; it < 20; ++it) {
        const R gmax = fmax(fmax(fabs(G[0]), fabs(G[1])), fmax(fabs(G[2]), fabs(G[3])));
        if (fmax(fabs(r[0]), fabs(r[1])) <= newton_tol<R>(tmax, mus, gmax)) return true;
        R Jac[2][2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            R dF[4] = {R(0), R(0), R(0), R(0)}, dP[4];
            dF[k * 2 + an] = R(1);
            jvp_ofs<LAW, R>(G, dF, m, dP);
            Jac[0][k] = Na * dP[0 * 2 + an];
            Jac[1][k] = Na * dP[1 * 2 + an];
        }
        const R det = Jac[0][0] * Jac[1][1] - Jac[0][1] * Jac[1][0];
        const R d0 = -(Jac[1][1] * r[0] - Jac[0][1] * r[1]) / det;
        const R d1 = -(-Jac[1][0] * r[0] + Jac[0][0] * r[1]) / det;
        // Euclidean norms through hypot: squaring residuals of order 1e-23 (nodes
        // still at rest) underflows in FP32 and would stall the line search
        const R rn = hypot(r[0], r[1]);
        R alpha = R(1);
        bool accepted = false;
        for (int ls = 0; ls <= 10; ++ls) {
            R Gt[4] = {G[0], G[1], G[2], G[3]};
            Gt[0 * 2 + an] += alpha * d0;
            Gt[1 * 2 + an] += alpha * d1;
            R Pt[4], dJt;
            piola_ofs<LAW, R>(Gt[0], Gt[1], Gt[2], Gt[3], m, Pt[0], Pt[1], Pt[2], Pt[3], dJt);
            if (dJt > R(-1)) {
                const R rt0 = Na * Pt[0 * 2 + an] - Tb[0], rt1 = Na * Pt[1 * 2 + an] - Tb[1];
                if (hypot(rt0, rt1) < rn) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) G[m] = Gt[m];
                    r[0] = rt0;
                    r[1] = rt1;
                    accepted = true;
                    break;
                }
            }
            alpha *= R(0.5);
        }
        if (!accepted) break;
    }
    const R gmax = fmax(fmax(fabs(G[0]), fabs(G[1])), fmax(fabs(G[2]), fabs(G[3])));
    return fmax(fabs(r[0]), fabs(r[1])) <= newton_tol<R>(tmax, mus, gmax);
}

// Ghost value of a velocity or traction edge in the node form. fo: f*_{-d}
// at the boundary node (offsets); U: (v, G) at the node at t^n; val: edge data
// at t^n + dt/2. Writes out[6]; sets ST_NEWTON in flags on failure.
template <int LAW, typename R>
__device__ __forceinline__ void edge_ghost(int e, int kind, const R fo[6], const R U[6], const double val[2],
                                           R c, const LawP<R> &m, R out[6], unsigned &flags)
{
    const R N0 = (e == EDGE_LEFT) ? R(-1) : (e == EDGE_RIGHT) ? R(1) : R(0);
    const R N1 = (e == EDGE_BOTTOM) ? R(-1) : (e == EDGE_TOP) ? R(1) : R(0);
    const R v0 = (R)val[0], v1 = (R)val[1];
    if (kind == BC_VELOCITY) {
        // Eq. (24): D = diag(-1,-1,1,1,1,1), S = (vD/2, N1 vD1/c, N2 vD1/c, N1 vD2/c, N2 vD2/c)
        out[0] = -fo[0] + R(0.5) * v0;
        out[1] = -fo[1] + R(0.5) * v1;
        out[2] = fo[2] + N0 * v0 / c;
        out[3] = fo[3] + N1 * v0 / c;
        out[4] = fo[4] + N0 * v1 / c;
        out[5] = fo[5] + N1 * v1 / c;
    } else {
        // Eq. (25): D = diag(1,1,-1,-1,-1,-1), S = (T/c, F^b/2)
        R G[4] = {U[2], U[3], U[4], U[5]};
        const R Tb[2] = {v0, v1};
        if (!traction_newton<LAW, R>(e, G, Tb, m)) flags |= ST_NEWTON;
        out[0] = fo[0] + v0 / c;
        out[1] = fo[1] + v1 / c;
#pragma unroll
        for (int m = 0; m < 4; ++m) out[2 + m] = -fo[2 + m] + R(0.5) * G[m];
    }
}

// edge data for position s of edge E with time factor g
__device__ __forceinline__ void edge_value(const EdgeDesc &E, int s, double g, double val[2])
{
    const double f = g * (E.profile ? E.profile[s] : 1.0);
    val[0] = E.value[0] * f;
    val[1] = E.value[1] * f;
}

} // namespace tlv
