// lbm_step.cu -- the edge kernel of the extrapolated F^b form and the
// dispatch of the single-lattice step kernels of the TL vectorial D2Q4x6 LBM
// (the kernels themselves: lbm_step_kernels.cuh, one storage type per
// translation unit).
//
// One time step (Sec. 3.7) is one launch of k_step (k_step16 for 16-bit
// storage): fused pull-streaming (Eq. 15) + state recovery (Eq. 10) + P(F) +
// equilibrium (Eq. 12) + BGK collision with the trapezoidal source (Eq. 14) +
// displacement quadrature (Eq. 22) for every node, reading the post-collision
// populations of step n-1 and writing those of step n. In the node form of
// F^b the same launch writes the ghost cells the boundary nodes pull at the
// next step (half-way rules, Eqs. 23-25); k_ghosts rebuilds them when they are
// stale. The extrapolated form of F^b needs neighbouring nodes and runs
// k_edges (FP64 Newton) before every step instead.
// The stored state between steps is the post-collision f*^n, so streaming
// happens at the start of the next step as a pull.
#include "lbm_internal.h"
#include "lbm_step_core.cuh"

namespace tlv {
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
    const LawP<double> m = law_at(a.m, (long long)y0 * a.L.nx + x0);
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
    piola_any(a.m.law, Gb, m, P, dJ);
    r[0] = Na * P[0 * 2 + an] - Tb[0];
    r[1] = Na * P[1 * 2 + an] - Tb[1];
    for (int it = 0; it < 20; ++it) {
        if (fmax(fabs(r[0]), fabs(r[1])) <= tol) return true;
        const double F[4] = {1.0 + Gb[0], Gb[1], Gb[2], 1.0 + Gb[3]};
        double Jac[2][2];
        for (int k = 0; k < 2; ++k) {
            double dF[4] = {0.0, 0.0, 0.0, 0.0}, dP[4];
            dF[k * 2 + an] = 1.0;
            tangent_jvp(a.m.law, F, dF, m, dP);
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
                piola_any(a.m.law, Gt, m, Pt, dJt);
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

// ---------------------------------------------------------------- dispatch
#define TLV_DECLARE(NAME)                                                                                  \
    cudaError_t launch_step_##NAME(int law, const void *args, bool fuse, int grid, cudaStream_t st);       \
    cudaError_t launch_ghosts_##NAME(const EdgeArgs &a, int grid, cudaStream_t st);                       \
    int step_blocks_##NAME(int law);
TLV_DECLARE(f64)
TLV_DECLARE(f32)
TLV_DECLARE(bf16)
TLV_DECLARE(f16)

cudaError_t launch_step(int storage, int law, bool fuse, const void *args, int grid, cudaStream_t st)
{
    switch (storage) {
    case STORE_F64: return launch_step_f64(law, args, fuse, grid, st);
    case STORE_BF16: return launch_step_bf16(law, args, fuse, grid, st);
    case STORE_F16: return launch_step_f16(law, args, fuse, grid, st);
    default: return launch_step_f32(law, args, fuse, grid, st);
    }
}

cudaError_t launch_ghosts(int storage, const EdgeArgs &a, int grid, cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    switch (storage) {
    case STORE_F64: return launch_ghosts_f64(a, grid, st);
    case STORE_BF16: return launch_ghosts_bf16(a, grid, st);
    case STORE_F16: return launch_ghosts_f16(a, grid, st);
    default: return launch_ghosts_f32(a, grid, st);
    }
}

int step_blocks_per_sm(int storage, int law)
{
    switch (storage) {
    case STORE_F64: return step_blocks_f64(law);
    case STORE_BF16: return step_blocks_bf16(law);
    case STORE_F16: return step_blocks_f16(law);
    default: return step_blocks_f32(law);
    }
}

cudaError_t launch_edges(int storage, const EdgeArgs &a, int grid, cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    return with_storage(storage, [&](auto tag) {
        k_edges<decltype(tag)><<<grid, 128, 0, st>>>(a);
        return cudaGetLastError();
    });
}

int step_vec(int storage) { return storage == STORE_F64 ? 2 : storage == STORE_F32 ? 4 : STEP16_V; }

} // namespace tlv
