// lbm_device.cuh -- device-side layout, parameter blocks and pointwise
// physics of the total-Lagrangian vectorial D2Q4x6 LBM (Feng & Chu).
//
// Population storage (both buffers): 24 planes p = q*6 + k (direction q of
// Sec. 3.1, state component k of Eq. 5), each (ny + 2) rows x pitch elements.
// Row 0 and row ny + 1 are ghost rows (y = -1, y = ny); column xoff - 1 and
// column xoff + nx are ghost columns (x = -1, x = nx). Node (x, y) lives at
//   p * plane + (y + 1) * pitch + xoff + x.
// xoff is 128 bytes, so every row of real nodes starts on a 128-byte line.
// Before each step the ghost cells hold the value each boundary node pulls
// from outside the domain (written by the previous step's fused kernel, or by
// the ghost or edge kernel), so the bulk kernel is a uniform pull over all
// nodes.
//
// Stored values are offsets from the rest equilibrium f_rest =
// (0, 0, 1/4, 0, 0, 1/4) (Eq. 12 at F = I, v = 0, where P(I) = 0), so the sum
// over q of the F-components gives G = F - I directly.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace tlv {

// ---------------------------------------------------------------- storage
// Populations are stored as S (double, float, __half or __nv_bfloat16) and
// computed in Prec<S>::R: double for double storage, float otherwise.
enum { STORE_F64 = 0, STORE_F32 = 1, STORE_BF16 = 2, STORE_F16 = 3 };

template <typename S>
struct Prec {
    using R = float;
};
template <>
struct Prec<double> {
    using R = double;
};

__device__ __forceinline__ double ld_r(double v) { return v; }
__device__ __forceinline__ float ld_r(float v) { return v; }
__device__ __forceinline__ float ld_r(__half v) { return __half2float(v); }
__device__ __forceinline__ float ld_r(__nv_bfloat16 v) { return __bfloat162float(v); }

// round to the storage type (nearest even)
template <typename S>
__device__ __forceinline__ S to_store(double v);
template <>
__device__ __forceinline__ double to_store<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_store<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __half to_store<__half>(double v) { return __double2half(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

template <typename S>
__device__ __forceinline__ S to_store(float v);
template <>
__device__ __forceinline__ float to_store<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half to_store<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Call fn with a value of the storage type selected by `storage`.
template <typename Fn>
__host__ auto with_storage(int storage, Fn fn)
{
    switch (storage) {
    case STORE_F64: return fn(double(0));
    case STORE_BF16: return fn(__nv_bfloat16());
    case STORE_F16: return fn(__half());
    default: return fn(float(0));
    }
}

enum { EDGE_LEFT = 0, EDGE_RIGHT = 1, EDGE_BOTTOM = 2, EDGE_TOP = 3 };
enum { BC_PERIODIC = 0, BC_VELOCITY = 1, BC_TRACTION = 2 };
enum { LAW_SVK = 0, LAW_NH = 1, LAW_LOGNH = 2, LAW_MR = 3, LAW_YEOH = 4, LAW_GENT = 5 };
enum { TF_CONST = 0, TF_LINEAR_RAMP = 1, TF_SIN2_RAMP = 2, TF_SIN_PULSE = 3, TF_RICKER = 4, TF_TABLE = 5 };
enum { FB_NODE = 0, FB_EXTRAP2 = 1 };
enum { ST_BAD_J = 1, ST_NEWTON = 2, ST_NONFINITE = 4, ST_STALL = 8 };  // ST_STALL: a bounded wait gave up

struct Layout {
    long long plane;  // elements per population plane
    int pitch;        // elements per row
    int xoff;         // column of node x = 0
    int nx, ny;
    long long uplane; // doubles per u* plane
    int upitch;       // doubles per u* row (no ghost rows or columns)
};

// Closure parameters as the law lists them (Appendix A): lam = lambda and
// mu, p2, p3 the law's own (SVK, NH, log-NH: mu; MR: c10, c01; Yeoh: c1,
// c2, c3; Gent: mu, Jm).
template <typename R>
struct LawP {
    R lam, mu, p2, p3;
};

struct Material {
    int law;
    double lam, mu, p2, p3;
    const double *mufield;  // per-node mu (compact, node y * nx + x) or nullptr (SVK, NH, log-NH)
    double lam_ratio;       // lambda = lam_ratio * mu where mufield is set
};

// parameters of node n (compact index)
__host__ __device__ __forceinline__ LawP<double> law_at(const Material &m, long long n)
{
    if (m.mufield) {
        const double mu = m.mufield[n];
        return LawP<double>{m.lam_ratio * mu, mu, 0.0, 0.0};
    }
    return LawP<double>{m.lam, m.mu, m.p2, m.p3};
}

template <typename R>
__host__ __device__ __forceinline__ LawP<R> law_cast(const LawP<double> &m)
{
    return LawP<R>{(R)m.lam, (R)m.mu, (R)m.p2, (R)m.p3};
}

// small-strain shear modulus of the law (a stress scale for tolerances)
template <int LAW, typename R>
__host__ __device__ __forceinline__ R shear_scale(const LawP<R> &m)
{
    return LAW == LAW_MR ? R(2) * (m.mu + m.p2) : LAW == LAW_YEOH ? R(2) * m.mu : m.mu;
}

struct EdgeDesc {
    int kind, timefn;
    double value[2];
    double tp[4];
    const double *profile; // device, one factor per edge node, or nullptr
};

// omega and 1 - omega of the collision (Eq. 14) in the compute type T, as a
// pair whose sum is exactly 1: with the two rounded on their own (for
// omega = 1.95 in FP32 they sum to 1 + 6e-8) every step would scale the
// node's state by that sum, an error that grows linearly with the step count
// instead of as a random walk. One of the pair is rounded, the other is its
// exact complement (Sterbenz: 1 - x is exact in T for x in [1/2, 2]).
template <typename T>
__host__ __device__ inline void relax_pair(double w, T &omega, T &one_m_omega)
{
    if (w >= 0.5) {
        omega = (T)w;
        one_m_omega = T(1) - omega;
    } else {
        one_m_omega = (T)(1.0 - w);
        omega = T(1) - one_m_omega;
    }
}

// T is the compute type; the populations are stored as the kernel's S
template <typename T>
struct StepArgs {
    const void *fin;             // post-collision populations f*^{n-1}, ghosts filled
    void *fout;                  // post-collision populations f*^n
    double *__restrict__ ustar;  // u*, advanced by dt v^n; nullptr (FP64, FP32 storage with a
                                 // material field: the adjoint's recomputed steps) skips it
    int *status;                 // latched ST_* bits
    Layout L;
    T omega, one_m_omega;        // the pair of relax_pair
    T wq, wc;                    // omega / 4 and omega / (2c) of the collision
    T hdtb1, hdtb2;              // (dt/2) b
    T src1, src2;                // dt (2 - omega) b / 8  (Eq. 14, w = 1/8)
    T lam, mu, c;
    T p2, p3;                    // third and fourth closure parameters (MR, Yeoh, Gent)
    const T *mufield;            // per-node mu in the u* plane layout, read by the MATF kernels
    T lam_ratio;                 // lambda = lam_ratio * mu there
    double dt;
    // edge rules, used when the kernel also writes the ghost cells of fout:
    // value * g * profile[s], g = g(t^n + dt/2) evaluated once on the host
    int kind[4];
    double value[4][2], g[4];
    const double *gdev;          // if set, the time factors are read here instead of g
    const double *profile[4];
    int k16;                     // 16-bit storage: step kernel chosen for the context (0 register,
                                 // 1 staged); read by the host launcher only
    // dynamic task claims (uniform material, register kernels): ctr2 the
    // context's two counter sets (2 x DYN_SET_WORDS words) or nullptr,
    // ctr_par the host-side index of the set the next dynamic launch takes
    // (read by the launcher); ctr / ctr_next that launch's set and the one it
    // zeroes
    unsigned *ctr2;
    int *ctr_par;
    int dyn_ns;                  // stripes of the claims: 1 or DYN_STRIPES (16-bit kernels;
                                 // the others always use DYN_STRIPES)
    unsigned *ctr, *ctr_next;
};

// Dynamic task claims (see claim_tasks): the task list is split into
// DYN_STRIPES contiguous stripes, each with its own claim counter, and the
// counters sit DYN_CTR_STRIDE words (256 bytes) apart so that no two share a
// cache line. One set of counters is DYN_SET_WORDS words.
constexpr int DYN_STRIPES = 4;
constexpr int DYN_CTR_STRIDE = 64;
constexpr int DYN_SET_WORDS = DYN_STRIPES * DYN_CTR_STRIDE;

// A batch of lattices for one persistent launch
constexpr int BATCH_MAX_MEMBERS = 4096;
struct BatchList {
    const void *args;  // StepArgs<R>[n]
    const int *off;    // n + 1 prefix sums of the members' task counts
    unsigned *ctr;     // dynamic task order: DYN_STRIPES claim counters and a
                       // finished-blocks counter, DYN_CTR_STRIDE words apart,
                       // all zero when the launch begins; nullptr: static order
    int n;
};

// Edge time factors of a batch: the host tabulates g(t) of every member's
// edges for the steps of one call (the same function and arguments as the
// single-lattice path), and before each step a one-block kernel copies row k
// of the table to the slot the members' StepArgs::gdev point at.
struct BatchTime {
    const double *tab;  // [K][n4]
    int *k;             // next row
    double *g;          // [n4]
    int n4;
    int rows;           // K
};

struct EdgeArgs {
    void *f;                  // populations of the current step (storage type)
    Layout L;
    EdgeDesc e[4];
    int blk_end[4];           // cumulative block counts per edge
    Material m;
    double c, dt, dx, hdtb1, hdtb2;
    int fb_mode, xper, yper;
    double g[4];              // time factor of each edge's data for the coming pull
    int *status;
};

// ---------------------------------------------------------------- pointwise
using ::expm1;  // the overloads below add Dual versions to these
using ::log1p;

// Forward-mode dual numbers v + d eps (eps^2 = 0): the Jacobian action of a
// closure written once for the value type is its evaluation on duals.
template <typename R>
struct Dual {
    R v, d;
    __host__ __device__ Dual() {}
    __host__ __device__ Dual(R x) : v(x), d(R(0)) {}
    __host__ __device__ Dual(R x, R y) : v(x), d(y) {}
};
template <typename R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, Dual<R> b) { return {a.v + b.v, a.d + b.d}; }
template <typename R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, Dual<R> b) { return {a.v - b.v, a.d - b.d}; }
template <typename R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a) { return {-a.v, -a.d}; }
template <typename R> __device__ __forceinline__ Dual<R> operator*(Dual<R> a, Dual<R> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <typename R> __device__ __forceinline__ Dual<R> operator/(Dual<R> a, Dual<R> b)
{
    const R q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
template <typename R> __device__ __forceinline__ Dual<R> operator*(R a, Dual<R> b) { return {a * b.v, a * b.d}; }
template <typename R> __device__ __forceinline__ Dual<R> operator+(R a, Dual<R> b) { return {a + b.v, b.d}; }
template <typename R> __device__ __forceinline__ Dual<R> operator-(R a, Dual<R> b) { return {a - b.v, -b.d}; }
template <typename R> __device__ __forceinline__ Dual<R> operator*(Dual<R> a, R b) { return {a.v * b, a.d * b}; }
template <typename R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, R b) { return {a.v + b, a.d}; }
template <typename R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, R b) { return {a.v - b, a.d}; }
template <typename R> __device__ __forceinline__ Dual<R> operator/(Dual<R> a, R b) { return {a.v / b, a.d / b}; }
template <typename R> __device__ __forceinline__ Dual<R> operator/(R a, Dual<R> b)
{
    const R q = a / b.v;
    return {q, -q * b.d / b.v};
}
template <typename R> __device__ __forceinline__ Dual<R> log1p(Dual<R> a) { return {::log1p(a.v), a.d / (R(1) + a.v)}; }
template <typename R> __device__ __forceinline__ Dual<R> expm1(Dual<R> a)
{
    const R e = ::expm1(a.v);
    return {e, (R(1) + e) * a.d};
}

// Closures built on the isochoric invariants (Eqs. A.2-A.3, A.7-A.9), from
// G = F - I in a form without cancellation at F = I: with tc = tr C - 2,
// J - 1 = dJ, J^{-2/3} = 1 + j23 and J^{-4/3} = 1 + j43 (expm1 of the scaled
// log1p), I1 = 3 + tc, I2 = 3 + dJ (2 + dJ) + tc (C33 = 1):
//   dI1bar/dF = (1 + j23) [2 (F - H) - (2/3) tc H]
//   dI2bar/dF = (1 + j43) [2 (F - H) + ((2/3) dJ (2 + dJ) - (4/3) tc) H]
//   P = s1 dI1bar/dF + s2 dI2bar/dF + lambda log J H,
// s1 = c10, s2 = c01 (MR); s1 = c1 + 2 c2 A + 3 c3 A^2 (Yeoh); s1 = mu / (2 (1 - A / Jm))
// (Gent), A = I1bar - 3 = 3 j23 + tc + j23 tc. V is R or Dual<R>.
template <int LAW, typename V, typename R>
__device__ __forceinline__ void piola_inv(const V G[4], const LawP<R> &m, V P[4], V &dJ)
{
    dJ = G[0] + G[3] + (G[0] * G[3] - G[1] * G[2]);
    const V J = R(1) + dJ;
    const V invJ = V(R(1)) / J;
    const V FmH[4] = {(G[0] - G[3] + dJ * (R(1) + G[0])) * invJ, (G[1] * J + G[2]) * invJ,
                      (G[2] * J + G[1]) * invJ, (G[3] - G[0] + dJ * (R(1) + G[3])) * invJ};
    const V H[4] = {(R(1) + G[3]) * invJ, -(G[2] * invJ), -(G[1] * invJ), (R(1) + G[0]) * invJ};
    const V tc = R(2) * (G[0] + G[3]) + (G[0] * G[0] + G[1] * G[1]) + (G[2] * G[2] + G[3] * G[3]);
    const V lJ = log1p(dJ);
    const V j23 = expm1(R(-2.0 / 3.0) * lJ);
    const V A = R(3) * j23 + tc + j23 * tc;
    V s1;
    if (LAW == LAW_MR)
        s1 = V(m.mu);
    else if (LAW == LAW_YEOH)
        s1 = m.mu + (R(2) * m.p2) * A + (R(3) * m.p3) * (A * A);
    else
        s1 = m.mu / (R(2) * (R(1) - A / V(m.p2)));
    const V c1 = R(2.0 / 3.0) * tc;
    const V vol = m.lam * lJ;
    for (int k = 0; k < 4; ++k) P[k] = s1 * ((R(1) + j23) * (R(2) * FmH[k] - c1 * H[k])) + vol * H[k];
    if (LAW == LAW_MR) {
        const V j43 = expm1(R(-4.0 / 3.0) * lJ);
        const V c2 = R(2.0 / 3.0) * (dJ * (R(2) + dJ)) - R(4.0 / 3.0) * tc;
        for (int k = 0; k < 4; ++k) P[k] = P[k] + m.p2 * ((R(1) + j43) * (R(2) * FmH[k] + c2 * H[k]));
    }
}

// First Piola stress from G = F - I (Appendix A), written so that the rest
// state does not cancel catastrophically: J - 1 = G11 + G22 + G11 G22 - G12 G21.
// 1 / x rounded to nearest (the value R(1) / x has under IEEE rules) by the
// reciprocal intrinsics, which need fewer instructions than a division
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

// Returns J - 1 in dJ.
template <int LAW, typename R>
__device__ __forceinline__ void piola_ofs(R G11, R G12, R G21, R G22, const LawP<R> &m, R &P11, R &P12,
                                          R &P21, R &P22, R &dJ)
{
    const R lam = m.lam, mu = m.mu;
    if (LAW >= LAW_MR) {
        const R G[4] = {G11, G12, G21, G22};
        R P[4];
        piola_inv<LAW, R, R>(G, m, P, dJ);
        P11 = P[0];
        P12 = P[1];
        P21 = P[2];
        P22 = P[3];
        return;
    }
    dJ = G11 + G22 + (G11 * G22 - G12 * G21);
    if (LAW == LAW_SVK) {
        // Eq. (A.4): P = F S, S = lambda tr(E) I + 2 mu E, E = (G + G^T + G^T G) / 2
        const R E11 = G11 + R(0.5) * (G11 * G11 + G21 * G21);
        const R E22 = G22 + R(0.5) * (G12 * G12 + G22 * G22);
        const R E12 = R(0.5) * (G12 + G21 + G11 * G12 + G21 * G22);
        const R trE = E11 + E22;
        const R S11 = lam * trE + R(2) * mu * E11, S22 = lam * trE + R(2) * mu * E22, S12 = R(2) * mu * E12;
        P11 = (R(1) + G11) * S11 + G12 * S12;
        P12 = (R(1) + G11) * S12 + G12 * S22;
        P21 = G21 * S11 + (R(1) + G22) * S12;
        P22 = G21 * S12 + (R(1) + G22) * S22;
    } else {
        // Eq. (A.5) / (A.6): P = mu (F - H) + a H, H = F^{-T} = cof(F) / J,
        // a = (lambda/2)(J^2 - 1) (NH) or lambda log J (log-NH)
        const R J = R(1) + dJ;
        const R invJ = rcp_rn(J);
        R a;
        if (LAW == LAW_NH)
            a = R(0.5) * lam * dJ * (R(2) + dJ);
        else
            a = lam * log1p(dJ);
        // mu / J and a / J formed once: P = (mu/J)(J F - cof F) + (a/J) cof F
        const R mJ = mu * invJ, aJ = a * invJ;
        P11 = mJ * (G11 - G22 + dJ * (R(1) + G11)) + aJ * (R(1) + G22);
        P12 = mJ * (G12 * J + G21) - aJ * G21;
        P21 = mJ * (G21 * J + G12) - aJ * G12;
        P22 = mJ * (G22 - G11 + dJ * (R(1) + G22)) + aJ * (R(1) + G11);
    }
}

// dP = C : dF for the invariant-based closures, by dual numbers
template <int LAW, typename R>
__device__ __forceinline__ void jvp_inv(const R G[4], const R dF[4], const LawP<R> &m, R dP[4])
{
    Dual<R> Gd[4], Pd[4], dJ;
    for (int k = 0; k < 4; ++k) Gd[k] = Dual<R>(G[k], dF[k]);
    piola_inv<LAW, Dual<R>, R>(Gd, m, Pd, dJ);
    for (int k = 0; k < 4; ++k) dP[k] = Pd[k].d;
}

// Stress of any law chosen at run time, from G = F - I, in compute type R
template <typename R>
__device__ inline void piola_any_t(int law, const R G[4], const LawP<R> &m, R P[4], R &dJ)
{
    switch (law) {
    case LAW_SVK: piola_ofs<LAW_SVK, R>(G[0], G[1], G[2], G[3], m, P[0], P[1], P[2], P[3], dJ); break;
    case LAW_NH: piola_ofs<LAW_NH, R>(G[0], G[1], G[2], G[3], m, P[0], P[1], P[2], P[3], dJ); break;
    case LAW_LOGNH: piola_ofs<LAW_LOGNH, R>(G[0], G[1], G[2], G[3], m, P[0], P[1], P[2], P[3], dJ); break;
    case LAW_MR: piola_ofs<LAW_MR, R>(G[0], G[1], G[2], G[3], m, P[0], P[1], P[2], P[3], dJ); break;
    case LAW_YEOH: piola_ofs<LAW_YEOH, R>(G[0], G[1], G[2], G[3], m, P[0], P[1], P[2], P[3], dJ); break;
    default: piola_ofs<LAW_GENT, R>(G[0], G[1], G[2], G[3], m, P[0], P[1], P[2], P[3], dJ); break;
    }
}

// FP64 stress of any law chosen at run time, from G = F - I
__device__ inline void piola_any(int law, const double G[4], const LawP<double> &m, double P[4], double &dJ)
{
    piola_any_t<double>(law, G, m, P, dJ);
}

// Strain energy W(F) of the same laws (diagnostics only), from G = F - I.
__device__ __forceinline__ double energy_ofs(int law, double G11, double G12, double G21, double G22,
                                             const LawP<double> &m)
{
    const double lam = m.lam, mu = m.mu;
    const double dJ = G11 + G22 + (G11 * G22 - G12 * G21);
    if (law == LAW_SVK) {
        const double E11 = G11 + 0.5 * (G11 * G11 + G21 * G21);
        const double E22 = G22 + 0.5 * (G12 * G12 + G22 * G22);
        const double E12 = 0.5 * (G12 + G21 + G11 * G12 + G21 * G22);
        const double trE = E11 + E22;
        return 0.5 * lam * trE * trE + mu * (E11 * E11 + 2.0 * E12 * E12 + E22 * E22);
    }
    // tr C - 2 = 2 (G11 + G22) + |G|^2
    const double trCm2 = 2.0 * (G11 + G22) + G11 * G11 + G12 * G12 + G21 * G21 + G22 * G22;
    const double lJ = log1p(dJ);
    if (law == LAW_NH) return 0.5 * mu * (trCm2 - 2.0 * lJ) + 0.25 * lam * (dJ * (2.0 + dJ) - 2.0 * lJ);
    if (law == LAW_LOGNH) return 0.5 * mu * (trCm2 - 2.0 * lJ) + 0.5 * lam * lJ * lJ;
    // Eqs. (A.7)-(A.9) with the variables of piola_inv
    const double j23 = expm1(-2.0 / 3.0 * lJ);
    const double A = 3.0 * j23 + trCm2 + j23 * trCm2;
    const double vol = 0.5 * lam * lJ * lJ;
    if (law == LAW_MR) {
        const double j43 = expm1(-4.0 / 3.0 * lJ);
        const double s = dJ * (2.0 + dJ) + trCm2;
        return mu * A + m.p2 * (3.0 * j43 + s + j43 * s) + vol;
    }
    if (law == LAW_YEOH) return mu * A + m.p2 * A * A + m.p3 * A * A * A + vol;
    return -0.5 * mu * m.p2 * log1p(-A / m.p2) + vol;
}


// Jacobian-vector product dP = C : dF of the tangent of Eq. (4) (Eq. 8), in
// compute type R.
template <typename R>
__device__ __forceinline__ void tangent_jvp_t(int law, const R F[4], const R dF[4], const LawP<R> &m, R dP[4])
{
    const R lam = m.lam, mu = m.mu;
    if (law >= LAW_MR) {
        const R G[4] = {F[0] - R(1.0), F[1], F[2], F[3] - R(1.0)};
        if (law == LAW_MR)
            jvp_inv<LAW_MR, R>(G, dF, m, dP);
        else if (law == LAW_YEOH)
            jvp_inv<LAW_YEOH, R>(G, dF, m, dP);
        else
            jvp_inv<LAW_GENT, R>(G, dF, m, dP);
        return;
    }
    if (law == LAW_SVK) {
        // dP = dF S + F dS, dS = lambda tr(dE) I + 2 mu dE, dE = (dF^T F + F^T dF) / 2
        const R E11 = R(0.5) * (F[0] * F[0] + F[2] * F[2] - R(1.0));
        const R E22 = R(0.5) * (F[1] * F[1] + F[3] * F[3] - R(1.0));
        const R E12 = R(0.5) * (F[0] * F[1] + F[2] * F[3]);
        const R trE = E11 + E22;
        const R S11 = lam * trE + R(2.0) * mu * E11, S22 = lam * trE + R(2.0) * mu * E22, S12 = R(2.0) * mu * E12;
        const R dE11 = dF[0] * F[0] + dF[2] * F[2];
        const R dE22 = dF[1] * F[1] + dF[3] * F[3];
        const R dE12 = R(0.5) * (dF[0] * F[1] + dF[2] * F[3] + F[0] * dF[1] + F[2] * dF[3]);
        const R dtr = dE11 + dE22;
        const R dS11 = lam * dtr + R(2.0) * mu * dE11, dS22 = lam * dtr + R(2.0) * mu * dE22, dS12 = R(2.0) * mu * dE12;
        dP[0] = dF[0] * S11 + dF[1] * S12 + F[0] * dS11 + F[1] * dS12;
        dP[1] = dF[0] * S12 + dF[1] * S22 + F[0] * dS12 + F[1] * dS22;
        dP[2] = dF[2] * S11 + dF[3] * S12 + F[2] * dS11 + F[3] * dS12;
        dP[3] = dF[2] * S12 + dF[3] * S22 + F[2] * dS12 + F[3] * dS22;
        return;
    }
    // NH:    dP = mu dF + lambda J^2 (H : dF) H + [mu - (lambda/2)(J^2 - 1)] H dF^T H
    // logNH: dP = mu dF + lambda     (H : dF) H + [mu - lambda log J]        H dF^T H
    const R J = F[0] * F[3] - F[1] * F[2];
    const R iJ = R(1) / J;
    const R H[4] = {F[3] * iJ, -F[2] * iJ, -F[1] * iJ, F[0] * iJ};
    const R HdF = H[0] * dF[0] + H[1] * dF[1] + H[2] * dF[2] + H[3] * dF[3];
    R a, b;
    if (law == LAW_NH) {
        a = lam * J * J;
        b = mu - R(0.5) * lam * (J * J - R(1.0));
    } else {
        a = lam;
        b = mu - lam * log(J);
    }
    // (H dF^T H)_iA = sum_{B,k} H_iB dF_kB H_kA
    R M[4];
    for (int i = 0; i < 2; ++i)
        for (int A = 0; A < 2; ++A) {
            R s = R(0);
            for (int k = 0; k < 2; ++k)
                for (int B = 0; B < 2; ++B) s += H[i * 2 + B] * dF[k * 2 + B] * H[k * 2 + A];
            M[i * 2 + A] = s;
        }
    for (int m = 0; m < 4; ++m) dP[m] = mu * dF[m] + a * HdF * H[m] + b * M[m];
}

// Jacobian-vector product dP = C : dF of the tangent of Eq. (4) (Eq. 8), FP64.
__device__ __forceinline__ void tangent_jvp(int law, const double F[4], const double dF[4], const LawP<double> &m,
                                            double dP[4])
{
    tangent_jvp_t<double>(law, F, dF, m, dP);
}


// Boundary-data time function g(t) (shapes of Eqs. 33, 35 and Sec. 5.4),
// evaluated on the host once per step and edge.
__host__ __device__ inline double timefn(int kind, const double *tp, double t)
{
    const double pi = 3.14159265358979323846;
    switch (kind) {
    case TF_CONST: return 1.0;
    case TF_LINEAR_RAMP: return t < tp[0] ? t / tp[0] : 1.0;
    case TF_SIN2_RAMP: {
        if (t >= tp[0]) return 1.0;
        const double s = sin(pi * t / (2.0 * tp[0]));
        return s * s;
    }
    case TF_SIN_PULSE: return t < tp[0] ? sin(pi * t / tp[0]) : 0.0;
    case TF_RICKER: {
        if (t > tp[2]) return 0.0;
        const double z = (t - tp[1]) / tp[0];
        return 2.0 / (sqrt(3.0 * tp[0]) * pow(pi, 0.25)) * (1.0 - z * z) * exp(-0.5 * z * z);
    }
    default: return 0.0;
    }
}

} // namespace tlv
