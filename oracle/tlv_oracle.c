/*
 * tlv_oracle.c -- FP64 CPU oracle for the total-Lagrangian vectorial LBM
 * (D2Q4 x 6) of Feng & Chu.
 *
 * TEST INFRASTRUCTURE. This file is the parity reference for the CUDA library:
 * plain loops over the whole lattice, one phase of the paper's time step at a
 * time (Sec. 3.7), IEEE binary64, compiled with -ffp-contract=off and no
 * fast-math. Only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg load it. It shares no code with the CUDA sources.
 *
 * Threads: the per-node loops of the initialization, of the phases of a step
 * and of the read-outs run their nodes (rows, or flat node ranges) across
 * OpenMP threads when the library is built with OpenMP. Each node's
 * arithmetic is the same whatever the thread count and no sum runs across
 * nodes, so every result is bit-identical for any number of threads; the
 * edge phase and the reference adjoint stay serial.
 *
 * Readings of points the paper leaves open (each listed in the design notes):
 *  - nodes are cell centred, so a half-way wall lies dx/2 outside the first
 *    and last node of a non-periodic direction (Sec. 3.6);
 *  - Neumann boundary deformation gradient F^b (Sec. 3.6.2). Two forms of
 *    the tangential column are provided:
 *      ORC_FB_NODE (default): F^b_iT = F_iT(x0, t^n), the value at the
 *        boundary node itself. With the boundary manufactured solution of
 *        Sec. 4.2 evaluated at t = 0.05 this form reproduces all six
 *        mixed-boundary errors of Table 2 to the printed digits, so it is
 *        taken as the form behind the paper's results;
 *      ORC_FB_EXTRAP2: F^b_iT = 1.5 F_iT(x0) - 0.5 F_iT(x1)
 *        + (dt/2)(1.5 dT v_i(x0) - 0.5 dT v_i(x1)), the linear extrapolation
 *        to the wall shifted half a step by the kinematic identity of Eq. (2),
 *        so that F^b = F(X_b, t + dt/2) + O(dt^2) as Eq. (B.20) asks.
 *    The normal column starts from F_iN(x0, t^n) and is found by Newton on
 *    P(F^b) N = T with a halving line search that rejects det F^b <= 0;
 *  - boundary data (v_D, T) are sampled at t^n + dt/2 (Eq. 23); F^b uses U^n;
 *  - no body-force term is added to the boundary sources S_d;
 *  - at a corner each missing link belongs to exactly one edge and uses that
 *    edge's rule; tangential derivatives are one-sided at the edge ends.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "tlv_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sec. 3.1: the D2Q4 directions (i, j) */
static const int CI[4] = {1, 0, -1, 0};
static const int CJ[4] = {0, 1, 0, -1};

/* ======================================================================
 * Appendix A: hyperelastic closures W(F), P(F) = dW/dF (Eqs. A.1-A.9)
 * ====================================================================== */

int orc_piola(int law, const double *p, const double F[4], double P[4])
{
    /* Eq. (A.1): J = det F, H = F^{-T} */
    const double J = F[0] * F[3] - F[1] * F[2];
    const double H[4] = {F[3] / J, -F[2] / J, -F[1] / J, F[0] / J};
    const double trC = F[0] * F[0] + F[1] * F[1] + F[2] * F[2] + F[3] * F[3];
    int m;
    switch (law) {
    case ORC_SVK: { /* Eq. (A.4): P = F [lambda tr(E) I + 2 mu E] */
        const double lam = p[0], mu = p[1];
        const double C11 = F[0] * F[0] + F[2] * F[2];
        const double C12 = F[0] * F[1] + F[2] * F[3];
        const double C22 = F[1] * F[1] + F[3] * F[3];
        const double E11 = 0.5 * (C11 - 1.0), E12 = 0.5 * C12, E22 = 0.5 * (C22 - 1.0);
        const double trE = E11 + E22;
        const double S11 = lam * trE + 2.0 * mu * E11;
        const double S12 = 2.0 * mu * E12;
        const double S22 = lam * trE + 2.0 * mu * E22;
        P[0] = F[0] * S11 + F[1] * S12;
        P[1] = F[0] * S12 + F[1] * S22;
        P[2] = F[2] * S11 + F[3] * S12;
        P[3] = F[2] * S12 + F[3] * S22;
        break;
    }
    case ORC_NH: { /* Eq. (A.5): P = mu (F - H) + (lambda/2)(J^2 - 1) H */
        const double lam = p[0], mu = p[1];
        const double a = 0.5 * lam * (J * J - 1.0);
        for (m = 0; m < 4; ++m) P[m] = mu * (F[m] - H[m]) + a * H[m];
        break;
    }
    case ORC_LOGNH: { /* Eq. (A.6): P = mu (F - H) + lambda log J H */
        const double lam = p[0], mu = p[1];
        const double a = lam * log(J);
        for (m = 0; m < 4; ++m) P[m] = mu * (F[m] - H[m]) + a * H[m];
        break;
    }
    case ORC_MR:
    case ORC_YEOH:
    case ORC_GENT: {
        /* Eqs. (A.2)-(A.3): modified invariants and their gradients */
        const double lam = p[0];
        const double I1 = trC + 1.0, I2 = J * J + trC;
        const double Jm23 = pow(J, -2.0 / 3.0), Jm43 = pow(J, -4.0 / 3.0);
        const double A = Jm23 * I1 - 3.0;
        double G1[4], G2[4], s1, s2 = 0.0;
        for (m = 0; m < 4; ++m) {
            G1[m] = Jm23 * (2.0 * F[m] - (2.0 / 3.0) * I1 * H[m]);
            G2[m] = Jm43 * (2.0 * F[m] + (2.0 * J * J - (4.0 / 3.0) * I2) * H[m]);
        }
        if (law == ORC_MR) {          /* Eq. (A.7) */
            s1 = p[1];
            s2 = p[2];
        } else if (law == ORC_YEOH) { /* Eq. (A.8) */
            s1 = p[1] + 2.0 * p[2] * A + 3.0 * p[3] * A * A;
        } else {                      /* Eq. (A.9) */
            s1 = p[1] / (2.0 * (1.0 - A / p[2]));
        }
        for (m = 0; m < 4; ++m) P[m] = s1 * G1[m] + s2 * G2[m] + lam * log(J) * H[m];
        break;
    }
    default:
        return -1;
    }
    return (J > 0.0) ? 0 : 1;
}

double orc_energy(int law, const double *p, const double F[4])
{
    const double J = F[0] * F[3] - F[1] * F[2];
    const double trC = F[0] * F[0] + F[1] * F[1] + F[2] * F[2] + F[3] * F[3];
    switch (law) {
    case ORC_SVK: {
        const double C11 = F[0] * F[0] + F[2] * F[2];
        const double C12 = F[0] * F[1] + F[2] * F[3];
        const double C22 = F[1] * F[1] + F[3] * F[3];
        const double E11 = 0.5 * (C11 - 1.0), E12 = 0.5 * C12, E22 = 0.5 * (C22 - 1.0);
        const double trE = E11 + E22;
        return 0.5 * p[0] * trE * trE + p[1] * (E11 * E11 + 2.0 * E12 * E12 + E22 * E22);
    }
    case ORC_NH:
        return 0.5 * p[1] * (trC - 2.0 - 2.0 * log(J)) + 0.25 * p[0] * (J * J - 1.0 - 2.0 * log(J));
    case ORC_LOGNH:
        return 0.5 * p[1] * (trC - 2.0 - 2.0 * log(J)) + 0.5 * p[0] * log(J) * log(J);
    case ORC_MR:
    case ORC_YEOH:
    case ORC_GENT: {
        const double I1 = trC + 1.0, I2 = J * J + trC;
        const double A = pow(J, -2.0 / 3.0) * I1 - 3.0;
        const double vol = 0.5 * p[0] * log(J) * log(J);
        if (law == ORC_MR) return p[1] * A + p[2] * (pow(J, -4.0 / 3.0) * I2 - 3.0) + vol;
        if (law == ORC_YEOH) return p[1] * A + p[2] * A * A + p[3] * A * A * A + vol;
        return -0.5 * p[1] * p[2] * log(1.0 - A / p[2]) + vol;
    }
    default:
        return NAN;
    }
}

/* Complex-argument copy of orc_piola (same formulas). Used only to obtain the
 * tangent C = dP/dF of Eq. (4) by the complex-step derivative
 * dP/dF_kB = Im P(F + i h e_kB) / h (Squire & Trapp 1998), exact to rounding. */
static int piola_c(int law, const double *p, const double complex F[4], double complex P[4])
{
    const double complex J = F[0] * F[3] - F[1] * F[2];
    const double complex H[4] = {F[3] / J, -F[2] / J, -F[1] / J, F[0] / J};
    const double complex trC = F[0] * F[0] + F[1] * F[1] + F[2] * F[2] + F[3] * F[3];
    int m;
    switch (law) {
    case ORC_SVK: {
        const double lam = p[0], mu = p[1];
        const double complex C11 = F[0] * F[0] + F[2] * F[2];
        const double complex C12 = F[0] * F[1] + F[2] * F[3];
        const double complex C22 = F[1] * F[1] + F[3] * F[3];
        const double complex E11 = 0.5 * (C11 - 1.0), E12 = 0.5 * C12, E22 = 0.5 * (C22 - 1.0);
        const double complex trE = E11 + E22;
        const double complex S11 = lam * trE + 2.0 * mu * E11;
        const double complex S12 = 2.0 * mu * E12;
        const double complex S22 = lam * trE + 2.0 * mu * E22;
        P[0] = F[0] * S11 + F[1] * S12;
        P[1] = F[0] * S12 + F[1] * S22;
        P[2] = F[2] * S11 + F[3] * S12;
        P[3] = F[2] * S12 + F[3] * S22;
        break;
    }
    case ORC_NH: {
        const double complex a = 0.5 * p[0] * (J * J - 1.0);
        for (m = 0; m < 4; ++m) P[m] = p[1] * (F[m] - H[m]) + a * H[m];
        break;
    }
    case ORC_LOGNH: {
        const double complex a = p[0] * clog(J);
        for (m = 0; m < 4; ++m) P[m] = p[1] * (F[m] - H[m]) + a * H[m];
        break;
    }
    case ORC_MR:
    case ORC_YEOH:
    case ORC_GENT: {
        const double complex I1 = trC + 1.0, I2 = J * J + trC;
        const double complex Jm23 = cexp((-2.0 / 3.0) * clog(J));
        const double complex Jm43 = cexp((-4.0 / 3.0) * clog(J));
        const double complex A = Jm23 * I1 - 3.0;
        double complex G1[4], G2[4], s1, s2 = 0.0;
        for (m = 0; m < 4; ++m) {
            G1[m] = Jm23 * (2.0 * F[m] - (2.0 / 3.0) * I1 * H[m]);
            G2[m] = Jm43 * (2.0 * F[m] + (2.0 * J * J - (4.0 / 3.0) * I2) * H[m]);
        }
        if (law == ORC_MR) {
            s1 = p[1];
            s2 = p[2];
        } else if (law == ORC_YEOH) {
            s1 = p[1] + 2.0 * p[2] * A + 3.0 * p[3] * A * A;
        } else {
            s1 = p[1] / (2.0 * (1.0 - A / p[2]));
        }
        for (m = 0; m < 4; ++m) P[m] = s1 * G1[m] + s2 * G2[m] + p[0] * clog(J) * H[m];
        break;
    }
    default:
        return -1;
    }
    return 0;
}

int orc_piola_cplx(int law, const double *prm, const double Fre[4], const double Fim[4],
                   double Pre[4], double Pim[4])
{
    double complex F[4], P[4];
    int m, rc;
    for (m = 0; m < 4; ++m) F[m] = Fre[m] + Fim[m] * I;
    rc = piola_c(law, prm, F, P);
    for (m = 0; m < 4; ++m) {
        Pre[m] = creal(P[m]);
        Pim[m] = cimag(P[m]);
    }
    return rc;
}

/* Eq. (4): C_iAkB = dP_iA / dF_kB, stored at [(i*2+A)*4 + (k*2+B)] */
int orc_tangent(int law, const double *prm, const double F[4], double C[16])
{
    const double h = 1e-30;
    int col, m;
    for (col = 0; col < 4; ++col) {
        double complex Fc[4], Pc[4];
        for (m = 0; m < 4; ++m) Fc[m] = F[m];
        Fc[col] += h * I;
        if (piola_c(law, prm, Fc, Pc) != 0) return -1;
        for (m = 0; m < 4; ++m) C[m * 4 + col] = cimag(Pc[m]) / h;
    }
    return 0;
}

/* ======================================================================
 * Sec. 2.4 and 3.2: fluxes and moment-matched equilibrium
 * ====================================================================== */

/* Eq. (7): Phi_X = (-P11, -P21, -v1, 0, -v2, 0), Phi_Y = (-P12, -P22, 0, -v1, 0, -v2) */
void orc_flux(const double U[6], const double P[4], double PhiX[6], double PhiY[6])
{
    PhiX[0] = -P[0]; PhiX[1] = -P[2]; PhiX[2] = -U[0]; PhiX[3] = 0.0; PhiX[4] = -U[1]; PhiX[5] = 0.0;
    PhiY[0] = -P[1]; PhiY[1] = -P[3]; PhiY[2] = 0.0; PhiY[3] = -U[0]; PhiY[4] = 0.0; PhiY[5] = -U[1];
}

/* Eq. (12): f^eq_ij = (1/4) [ U + (2/c) (i Phi_X + j Phi_Y) ], stored feq[q*6 + k] */
void orc_feq(const double U[6], const double P[4], double c, double feq[24])
{
    double PhiX[6], PhiY[6];
    int q, k;
    orc_flux(U, P, PhiX, PhiY);
    for (q = 0; q < 4; ++q)
        for (k = 0; k < 6; ++k)
            feq[q * 6 + k] = 0.25 * (U[k] + (2.0 / c) * (CI[q] * PhiX[k] + CJ[q] * PhiY[k]));
}

/* boundary-data time functions g(t) (shapes of Eqs. 33, 35 and Sec. 5.4) */
double orc_timefn(int kind, const double *tp, double t)
{
    const double pi = 3.14159265358979323846;
    switch (kind) {
    case ORC_T_CONST:
        return 1.0;
    case ORC_T_LINEAR_RAMP:
        return (t < tp[0]) ? t / tp[0] : 1.0;
    case ORC_T_SIN2_RAMP: {
        const double s = sin(pi * t / (2.0 * tp[0]));
        return (t < tp[0]) ? s * s : 1.0;
    }
    case ORC_T_SIN_PULSE:
        return (t < tp[0]) ? sin(pi * t / tp[0]) : 0.0;
    case ORC_T_RICKER: { /* tp = {s, t0, t_end}; Ricker pulse of Sec. 5.4 per unit p0 */
        const double z = (t - tp[1]) / tp[0];
        if (t > tp[2]) return 0.0;
        return 2.0 / (sqrt(3.0 * tp[0]) * pow(pi, 0.25)) * (1.0 - z * z) * exp(-0.5 * z * z);
    }
    default:
        return NAN;
    }
}

/* ======================================================================
 * The lattice
 * ====================================================================== */

typedef struct {
    int kind, timefn;
    double value[2], tp[4];
    double *profile; /* edge length, or NULL */
    double *data;    /* 2 x edge length, or NULL */
} orc_edge;

struct orc {
    int nx, ny;
    long N;
    double dx, c, omega, dt;
    int law;
    double prm[8];
    double *mufield; /* per-node mu (N) with lambda = lam_ratio * mu, or NULL */
    double lam_ratio;
    double b[2];
    double *bfield; /* 2N or NULL */
    orc_edge e[4];
    double *f;      /* pre-collision populations f^n, [q*6+k][n] */
    double *fs;     /* post-collision populations f*^n           */
    double *U;      /* recovered state U^n of the current step    */
    double *ustar;  /* displacement accumulator u*^n, [2][n]      */
    long step;
    int status, ready, fb_mode;
};

static long nid(const orc *o, int ix, int iy) { return (long)iy * o->nx + ix; }
static int edge_len(const orc *o, int e) { return (e == ORC_LEFT || e == ORC_RIGHT) ? o->ny : o->nx; }
static int xper(const orc *o) { return o->e[ORC_LEFT].kind == ORC_PERIODIC; }
static int yper(const orc *o) { return o->e[ORC_BOTTOM].kind == ORC_PERIODIC; }
static double bforce(const orc *o, int comp, long n) { return o->bfield ? o->bfield[comp * o->N + n] : o->b[comp]; }

/* material parameters of node n: the uniform set, or {lam_ratio mu_n, mu_n}
 * when a shear-modulus field is set */
static const double *node_prm(const orc *o, long n, double buf[8])
{
    int i;
    if (!o->mufield) return o->prm;
    for (i = 0; i < 8; ++i) buf[i] = 0.0;
    buf[0] = o->lam_ratio * o->mufield[n];
    buf[1] = o->mufield[n];
    return buf;
}

orc *orc_new(int nx, int ny, double dx, double c, double omega)
{
    orc *o;
    int e;
    if (nx < 1 || ny < 1 || !(dx > 0.0) || !(c > 0.0) || !(omega > 0.0) || !(omega <= 2.0)) return NULL;
    o = (orc *)calloc(1, sizeof(orc));
    if (!o) return NULL;
    o->nx = nx;
    o->ny = ny;
    o->N = (long)nx * ny;
    o->dx = dx;
    o->c = c;
    o->omega = omega;
    o->dt = dx / c; /* Sec. 3.1: c = dx / dt */
    o->law = -1;
    for (e = 0; e < 4; ++e) o->e[e].kind = ORC_PERIODIC;
    o->f = (double *)calloc((size_t)24 * o->N, sizeof(double));
    o->fs = (double *)calloc((size_t)24 * o->N, sizeof(double));
    o->U = (double *)calloc((size_t)6 * o->N, sizeof(double));
    o->ustar = (double *)calloc((size_t)2 * o->N, sizeof(double));
    if (!o->f || !o->fs || !o->U || !o->ustar) {
        orc_free(o);
        return NULL;
    }
    return o;
}

void orc_free(orc *o)
{
    int e;
    if (!o) return;
    for (e = 0; e < 4; ++e) {
        free(o->e[e].profile);
        free(o->e[e].data);
    }
    free(o->bfield);
    free(o->mufield);
    free(o->f);
    free(o->fs);
    free(o->U);
    free(o->ustar);
    free(o);
}

int orc_set_law(orc *o, int law, const double *prm, int nprm)
{
    int i;
    if (law < ORC_SVK || law > ORC_GENT || nprm < 2 || nprm > 8) return -1;
    o->law = law;
    for (i = 0; i < 8; ++i) o->prm[i] = (i < nprm) ? prm[i] : 0.0;
    free(o->mufield); /* a new law drops a shear-modulus field */
    o->mufield = NULL;
    return 0;
}

int orc_set_material_field(orc *o, const double *mu_N, double lam_ratio)
{
    long n;
    free(o->mufield);
    o->mufield = NULL;
    if (!mu_N) return 0;
    if (o->law != ORC_SVK && o->law != ORC_NH && o->law != ORC_LOGNH) return -1;
    for (n = 0; n < o->N; ++n)
        if (!(mu_N[n] > 0.0)) return -2;
    o->mufield = (double *)malloc((size_t)o->N * sizeof(double));
    memcpy(o->mufield, mu_N, (size_t)o->N * sizeof(double));
    o->lam_ratio = lam_ratio;
    return 0;
}

int orc_set_fb_mode(orc *o, int mode)
{
    if (mode != ORC_FB_NODE && mode != ORC_FB_EXTRAP2) return -1;
    o->fb_mode = mode;
    return 0;
}

void orc_set_body_force(orc *o, double b1, double b2)
{
    o->b[0] = b1;
    o->b[1] = b2;
}

void orc_set_body_force_field(orc *o, const double *b2N)
{
    free(o->bfield);
    o->bfield = NULL;
    if (b2N) {
        o->bfield = (double *)malloc((size_t)2 * o->N * sizeof(double));
        memcpy(o->bfield, b2N, (size_t)2 * o->N * sizeof(double));
    }
}

int orc_set_edge(orc *o, int e, int kind, const double value[2], int timefn, const double tp[4],
                 const double *profile)
{
    orc_edge *E;
    int len, i;
    if (e < 0 || e > 3 || kind < ORC_PERIODIC || kind > ORC_TRACTION) return -1;
    E = &o->e[e];
    len = edge_len(o, e);
    E->kind = kind;
    E->timefn = timefn;
    E->value[0] = value ? value[0] : 0.0;
    E->value[1] = value ? value[1] : 0.0;
    for (i = 0; i < 4; ++i) E->tp[i] = tp ? tp[i] : 0.0;
    free(E->profile);
    E->profile = NULL;
    if (profile) {
        E->profile = (double *)malloc((size_t)len * sizeof(double));
        memcpy(E->profile, profile, (size_t)len * sizeof(double));
    }
    return 0;
}

int orc_set_edge_data(orc *o, int e, const double *vals)
{
    orc_edge *E;
    int len;
    if (e < 0 || e > 3) return -1;
    E = &o->e[e];
    len = edge_len(o, e);
    free(E->data);
    E->data = NULL;
    if (vals) {
        E->data = (double *)malloc((size_t)2 * len * sizeof(double));
        memcpy(E->data, vals, (size_t)2 * len * sizeof(double));
    }
    return 0;
}

/* second-order difference of field a (one component, N values) along x or y
 * at node (ix, iy): central inside, wrap-around when that direction is
 * periodic, one-sided three-point stencil at a non-periodic end (Sec. 3.4) */
static double fd(const orc *o, const double *a, int ix, int iy, int dir)
{
    const int n = dir == 0 ? o->nx : o->ny;
    const int i = dir == 0 ? ix : iy;
    const int per = dir == 0 ? xper(o) : yper(o);
#define AT(j) (dir == 0 ? a[nid(o, (j), iy)] : a[nid(o, ix, (j))])
    if (per) return (AT((i + 1) % n) - AT((i - 1 + n) % n)) / (2.0 * o->dx);
    if (i == 0) return (-3.0 * AT(0) + 4.0 * AT(1) - AT(2)) / (2.0 * o->dx);
    if (i == n - 1) return (3.0 * AT(n - 1) - 4.0 * AT(n - 2) + AT(n - 3)) / (2.0 * o->dx);
    return (AT(i + 1) - AT(i - 1)) / (2.0 * o->dx);
#undef AT
}

static int check_edges(const orc *o)
{
    if ((o->e[ORC_LEFT].kind == ORC_PERIODIC) != (o->e[ORC_RIGHT].kind == ORC_PERIODIC)) return -2;
    if ((o->e[ORC_BOTTOM].kind == ORC_PERIODIC) != (o->e[ORC_TOP].kind == ORC_PERIODIC)) return -2;
    if (!xper(o) && o->nx < 3) return -3;
    if (!yper(o) && o->ny < 3) return -3;
    return 0;
}

/* Sec. 3.4, Eqs. (16)-(21): f_q(X,0) = f^eq(U0) - (dt/2) D_q f^eq(U0) at node
 * (ix, iy), with the node's material; f[q*6+k]. Returns ORC_BAD_J or 0. */
static int init_at(const orc *o, const double *U0, int order, const double *dUdX, const double *dUdY, int ix,
                   int iy, double f[24])
{
    const long N = o->N, n = nid(o, ix, iy);
    const double c = o->c, dt = o->dt;
    double U[6], F[4], P[4], pb[8];
    const double *prm = node_prm(o, n, pb);
    int q, k, m, mm, st = 0;
    for (k = 0; k < 6; ++k) U[k] = U0[k * N + n];
    for (m = 0; m < 4; ++m) F[m] = U[2 + m];
    if (orc_piola(o->law, prm, F, P) != 0) st = ORC_BAD_J;
    orc_feq(U, P, c, f);
    if (order == 2) {
        double gX[6], gY[6], Ct[16], dPX[4], dPY[4];
        const double b1 = bforce(o, 0, n), b2 = bforce(o, 1, n);
        for (k = 0; k < 6; ++k) {
            gX[k] = dUdX ? dUdX[k * N + n] : fd(o, U0 + k * N, ix, iy, 0);
            gY[k] = dUdY ? dUdY[k * N + n] : fd(o, U0 + k * N, ix, iy, 1);
        }
        orc_tangent(o->law, prm, F, Ct);
        /* d_alpha P_iA = C_iAkB d_alpha F_kB (text after Eq. 18) */
        for (m = 0; m < 4; ++m) {
            dPX[m] = 0.0;
            dPY[m] = 0.0;
            for (mm = 0; mm < 4; ++mm) {
                dPX[m] += Ct[m * 4 + mm] * gX[2 + mm];
                dPY[m] += Ct[m * 4 + mm] * gY[2 + mm];
            }
        }
        for (q = 0; q < 4; ++q) {
            const double i = CI[q], j = CJ[q];
            double Z[6], dP[4], D[6];
            /* Eq. (18) */
            Z[0] = b1 + dPX[0] + dPY[1] + c * i * gX[0] + c * j * gY[0];
            Z[1] = b2 + dPX[2] + dPY[3] + c * i * gX[1] + c * j * gY[1];
            Z[2] = gX[0] + c * i * gX[2] + c * j * gY[2];
            Z[3] = gY[0] + c * i * gX[3] + c * j * gY[3];
            Z[4] = gX[1] + c * i * gX[4] + c * j * gY[4];
            Z[5] = gY[1] + c * i * gX[5] + c * j * gY[5];
            /* Eqs. (19)-(20): delta P^q = C : Z_F */
            for (m = 0; m < 4; ++m) {
                dP[m] = 0.0;
                for (mm = 0; mm < 4; ++mm) dP[m] += Ct[m * 4 + mm] * Z[2 + mm];
            }
            /* Eq. (21) */
            D[0] = 0.25 * (Z[0] - (2.0 / c) * (i * dP[0] + j * dP[1]));
            D[1] = 0.25 * (Z[1] - (2.0 / c) * (i * dP[2] + j * dP[3]));
            D[2] = 0.25 * (Z[2] - (2.0 * i / c) * Z[0]);
            D[3] = 0.25 * (Z[3] - (2.0 * j / c) * Z[0]);
            D[4] = 0.25 * (Z[4] - (2.0 * i / c) * Z[1]);
            D[5] = 0.25 * (Z[5] - (2.0 * j / c) * Z[1]);
            for (k = 0; k < 6; ++k) f[q * 6 + k] -= 0.5 * dt * D[k];
        }
    }
    return st;
}

int orc_init(orc *o, const double *U0, const double *u0, int order, const double *dUdX,
             const double *dUdY)
{
    const long N = o->N;
    const double dt = o->dt;
    int iy, st = 0;
    int rc = check_edges(o);
    if (rc) return rc;
    if (o->law < 0) return -4;
    if (order != 0 && order != 2) return -5;
#pragma omp parallel for schedule(static) reduction(| : st)
    for (iy = 0; iy < o->ny; ++iy)
        for (int ix = 0; ix < o->nx; ++ix) {
            const long n = nid(o, ix, iy);
            double f[24];
            st |= init_at(o, U0, order, dUdX, dUdY, ix, iy, f);
            for (int q = 0; q < 4; ++q)
                for (int k = 0; k < 6; ++k) o->f[(long)(q * 6 + k) * N + n] = f[q * 6 + k];
            /* Sec. 3.5: u*^0 = u0 - (dt/2) v0 */
            for (int k = 0; k < 2; ++k)
                o->ustar[k * N + n] = (u0 ? u0[k * N + n] : 0.0) - 0.5 * dt * U0[k * N + n];
        }
    o->status = st;
    o->step = 0;
    o->ready = 1;
    return 0;
}

/* node index of the node in layer L (0 = on the edge) at position s along edge e */
static long edge_node(const orc *o, int e, int L, int s)
{
    switch (e) {
    case ORC_LEFT: return nid(o, L, s);
    case ORC_RIGHT: return nid(o, o->nx - 1 - L, s);
    case ORC_BOTTOM: return nid(o, s, L);
    default: return nid(o, s, o->ny - 1 - L);
    }
}

/* derivative of state component comp of U^n along edge e (the tangential
 * material direction), in layer L at position s */
static double dT(const orc *o, int e, int L, int s, int comp)
{
    const int len = edge_len(o, e);
    const int per = (e == ORC_LEFT || e == ORC_RIGHT) ? yper(o) : xper(o);
    const double *a = o->U + (long)comp * o->N;
#define AV(p) a[edge_node(o, e, L, (p))]
    if (per) return (AV((s + 1) % len) - AV((s - 1 + len) % len)) / (2.0 * o->dx);
    if (s == 0) return (-3.0 * AV(0) + 4.0 * AV(1) - AV(2)) / (2.0 * o->dx);
    if (s == len - 1) return (3.0 * AV(len - 1) - 4.0 * AV(len - 2) + AV(len - 3)) / (2.0 * o->dx);
    return (AV(s + 1) - AV(s - 1)) / (2.0 * o->dx);
#undef AV
}

/* r_i = P_iA(F) N_A - T_i on an edge whose normal is material direction a
 * with sign Na */
static void traction_residual(const orc *o, const double *prm, const double F[4], int a, double Na,
                              const double T[2], double r[2])
{
    double P[4];
    orc_piola(o->law, prm, F, P);
    r[0] = Na * P[0 * 2 + a] - T[0];
    r[1] = Na * P[1 * 2 + a] - T[1];
}

/* Sec. 3.6.2: boundary deformation gradient F^b for a traction edge */
static int boundary_F(orc *o, int e, int s, const double T[2], double Fb[4])
{
    const int a = (e == ORC_LEFT || e == ORC_RIGHT) ? 0 : 1; /* normal material index   */
    const int tc = 1 - a;                                    /* tangential column index */
    const double Na = (e == ORC_LEFT || e == ORC_BOTTOM) ? -1.0 : 1.0;
    const long n0 = edge_node(o, e, 0, s), n1 = (o->fb_mode == ORC_FB_EXTRAP2) ? edge_node(o, e, 1, s) : n0;
    double pb[8];
    const double *prm = node_prm(o, n0, pb);
    const double tmax = fmax(fabs(T[0]), fabs(T[1]));
    const double tol = 1e-13 * (tmax > 1.0 ? tmax : 1.0);
    double r[2];
    int i, it, ls;
    for (i = 0; i < 2; ++i) {
        const double F0t = o->U[(2 + i * 2 + tc) * o->N + n0];
        if (o->fb_mode == ORC_FB_EXTRAP2) {
            const double F1t = o->U[(2 + i * 2 + tc) * o->N + n1];
            const double dv0 = dT(o, e, 0, s, i), dv1 = dT(o, e, 1, s, i);
            Fb[i * 2 + tc] = 1.5 * F0t - 0.5 * F1t + 0.5 * o->dt * (1.5 * dv0 - 0.5 * dv1);
        } else {
            Fb[i * 2 + tc] = F0t;
        }
        Fb[i * 2 + a] = o->U[(2 + i * 2 + a) * o->N + n0]; /* Newton starting point */
    }
    traction_residual(o, prm, Fb, a, Na, T, r);
    for (it = 0; it < 20; ++it) {
        double Ct[16], Jac[4], det, d0, d1, rn, alpha = 1.0;
        int accepted = 0;
        if (fmax(fabs(r[0]), fabs(r[1])) <= tol) return 0;
        orc_tangent(o->law, prm, Fb, Ct);
        /* d r_i / d F_ka = Na C_iaka */
        for (i = 0; i < 2; ++i) {
            Jac[i * 2 + 0] = Na * Ct[(i * 2 + a) * 4 + (0 * 2 + a)];
            Jac[i * 2 + 1] = Na * Ct[(i * 2 + a) * 4 + (1 * 2 + a)];
        }
        det = Jac[0] * Jac[3] - Jac[1] * Jac[2];
        d0 = -(Jac[3] * r[0] - Jac[1] * r[1]) / det;
        d1 = -(-Jac[2] * r[0] + Jac[0] * r[1]) / det;
        rn = hypot(r[0], r[1]);
        for (ls = 0; ls <= 10; ++ls) {
            double Ft[4], rt[2];
            memcpy(Ft, Fb, sizeof Ft);
            Ft[0 * 2 + a] += alpha * d0;
            Ft[1 * 2 + a] += alpha * d1;
            if (Ft[0] * Ft[3] - Ft[1] * Ft[2] > 0.0) {
                traction_residual(o, prm, Ft, a, Na, T, rt);
                if (hypot(rt[0], rt[1]) < rn) {
                    memcpy(Fb, Ft, sizeof Ft);
                    r[0] = rt[0];
                    r[1] = rt[1];
                    accepted = 1;
                    break;
                }
            }
            alpha *= 0.5;
        }
        if (!accepted) break;
    }
    return (fmax(fabs(r[0]), fabs(r[1])) <= tol) ? 0 : -1;
}

/* edge data at t^n + dt/2 for position s */
static void edge_value(const orc *o, int e, int s, double t_half, double val[2])
{
    const orc_edge *E = &o->e[e];
    const int len = edge_len(o, e);
    if (E->data) {
        val[0] = E->data[s];
        val[1] = E->data[len + s];
    } else {
        const double g = orc_timefn(E->timefn, E->tp, t_half) * (E->profile ? E->profile[s] : 1.0);
        val[0] = E->value[0] * g;
        val[1] = E->value[1] * g;
    }
}

int orc_step(orc *o, int nsteps)
{
    const long N = o->N;
    const double c = o->c, dt = o->dt, w = o->omega;
    int s, k, iy, e;
    if (!o->ready) return -1;
    for (s = 0; s < nsteps; ++s) {
        const double t = o->step * dt;
        long n;
        int st = 0;
        /* 1. state recovery, Eq. (10): U^n = sum_q f_q + (dt/2) B */
#pragma omp parallel for schedule(static)
        for (n = 0; n < N; ++n)
            for (int k = 0; k < 6; ++k) {
                double sum = 0.0;
                for (int q = 0; q < 4; ++q) sum += o->f[(long)(q * 6 + k) * N + n];
                if (k < 2) sum += 0.5 * dt * bforce(o, k, n);
                o->U[k * N + n] = sum;
            }
        /* 2-3. P(F^n), fluxes, equilibrium and BGK collision with the
         * trapezoidal source, Eq. (14) with w_ij = 1/8 */
#pragma omp parallel for schedule(static) reduction(| : st)
        for (n = 0; n < N; ++n) {
            double U[6], F[4], P[4], feq[24], pb[8];
            for (int k = 0; k < 6; ++k) U[k] = o->U[k * N + n];
            for (int k = 0; k < 4; ++k) F[k] = U[2 + k];
            if (orc_piola(o->law, node_prm(o, n, pb), F, P) != 0) st |= ORC_BAD_J;
            for (int k = 0; k < 6; ++k)
                if (!isfinite(U[k])) st |= ORC_NONFINITE;
            orc_feq(U, P, c, feq);
            for (int q = 0; q < 4; ++q)
                for (int k = 0; k < 6; ++k) {
                    const long idx = (long)(q * 6 + k) * N + n;
                    const double Bk = (k < 2) ? bforce(o, k, n) : 0.0;
                    o->fs[idx] = o->f[idx] + w * (feq[q * 6 + k] - o->f[idx]) + dt * (2.0 - w) * 0.125 * Bk;
                }
        }
        o->status |= st;
        /* 4. streaming, Eq. (15): f_q(X + c_q dt) = f*_q(X); links that leave a
         * non-periodic domain are dropped and rebuilt in phase 5 */
#pragma omp parallel for schedule(static)
        for (n = 0; n < 24 * N; ++n) o->f[n] = NAN;
#pragma omp parallel for schedule(static)
        for (iy = 0; iy < o->ny; ++iy)
            for (int ix = 0; ix < o->nx; ++ix)
                for (int q = 0; q < 4; ++q) {
                    int tx = ix + CI[q], ty = iy + CJ[q];
                    if (tx < 0 || tx >= o->nx) {
                        if (!xper(o)) continue;
                        tx = (tx + o->nx) % o->nx;
                    }
                    if (ty < 0 || ty >= o->ny) {
                        if (!yper(o)) continue;
                        ty = (ty + o->ny) % o->ny;
                    }
                    for (int k = 0; k < 6; ++k)
                        o->f[(long)(q * 6 + k) * N + nid(o, tx, ty)] = o->fs[(long)(q * 6 + k) * N + nid(o, ix, iy)];
                }
        /* 5. half-way reconstruction of the missing incoming populations,
         * Eq. (23): f_d(t+dt) = D f*_{-d}(t) + S_d(t + dt/2), d = -N */
        for (e = 0; e < 4; ++e) {
            const orc_edge *E = &o->e[e];
            const int len = edge_len(o, e);
            /* missing direction d and its opposite -d = N, and the normal N */
            static const int dmiss[4] = {0, 2, 1, 3}, dout[4] = {2, 0, 3, 1};
            static const double NX[4] = {-1, 1, 0, 0}, NY[4] = {0, 0, -1, 1};
            int p;
            if (E->kind == ORC_PERIODIC) continue;
            for (p = 0; p < len; ++p) {
                const long nb = edge_node(o, e, 0, p);
                double val[2], D[6], S[6];
                edge_value(o, e, p, t + 0.5 * dt, val);
                if (E->kind == ORC_VELOCITY) {
                    /* Eq. (24) */
                    D[0] = -1; D[1] = -1; D[2] = 1; D[3] = 1; D[4] = 1; D[5] = 1;
                    S[0] = 0.5 * val[0];
                    S[1] = 0.5 * val[1];
                    S[2] = NX[e] * val[0] / c;
                    S[3] = NY[e] * val[0] / c;
                    S[4] = NX[e] * val[1] / c;
                    S[5] = NY[e] * val[1] / c;
                } else {
                    /* Eq. (25) with the boundary deformation gradient F^b */
                    double Fb[4];
                    if (boundary_F(o, e, p, val, Fb) != 0) o->status |= ORC_NEWTON_FAIL;
                    D[0] = 1; D[1] = 1; D[2] = -1; D[3] = -1; D[4] = -1; D[5] = -1;
                    S[0] = val[0] / c;
                    S[1] = val[1] / c;
                    for (k = 0; k < 4; ++k) S[2 + k] = 0.5 * Fb[k];
                }
                for (k = 0; k < 6; ++k)
                    o->f[(long)(dmiss[e] * 6 + k) * N + nb] = D[k] * o->fs[(long)(dout[e] * 6 + k) * N + nb] + S[k];
            }
        }
        /* 6. displacement quadrature, Eq. (22):
         * u^n = u*^n + (dt/2) v^n, u*^{n+1} = u^n + (dt/2) v^n */
#pragma omp parallel for schedule(static)
        for (n = 0; n < N; ++n)
            for (int k = 0; k < 2; ++k) {
                const double un = o->ustar[k * N + n] + 0.5 * dt * o->U[k * N + n];
                o->ustar[k * N + n] = un + 0.5 * dt * o->U[k * N + n];
            }
        o->step += 1;
    }
    return 0;
}

/* U^n = sum_q f_q^n + (dt/2) B(t^n), P(F^n) and sigma = J^{-1} P F^T (Sec. 3.5) */
void orc_state(const orc *o, double *U, double *P, double *sigma)
{
    const long N = o->N;
    long n;
#pragma omp parallel for schedule(static)
    for (n = 0; n < N; ++n) {
        double u6[6], F[4], Pn[4], J, pb[8];
        int k;
        for (k = 0; k < 6; ++k) {
            double sum = 0.0;
            for (int q = 0; q < 4; ++q) sum += o->f[(long)(q * 6 + k) * N + n];
            if (k < 2) sum += 0.5 * o->dt * bforce(o, k, n);
            u6[k] = sum;
            if (U) U[k * N + n] = sum;
        }
        for (k = 0; k < 4; ++k) F[k] = u6[2 + k];
        orc_piola(o->law, node_prm(o, n, pb), F, Pn);
        if (P)
            for (k = 0; k < 4; ++k) P[k * N + n] = Pn[k];
        if (sigma) {
            J = F[0] * F[3] - F[1] * F[2];
            /* sigma_ij = J^{-1} P_iA F_jA */
            sigma[0 * N + n] = (Pn[0] * F[0] + Pn[1] * F[1]) / J;
            sigma[1 * N + n] = (Pn[0] * F[2] + Pn[1] * F[3]) / J;
            sigma[2 * N + n] = (Pn[2] * F[0] + Pn[3] * F[1]) / J;
            sigma[3 * N + n] = (Pn[2] * F[2] + Pn[3] * F[3]) / J;
        }
    }
}

/* u^n = u*^n + (dt/2) v^n, Eq. (22) */
void orc_displacement(const orc *o, double *u)
{
    const long N = o->N;
    long n;
#pragma omp parallel for schedule(static)
    for (n = 0; n < N; ++n)
        for (int k = 0; k < 2; ++k) {
            double v = 0.0;
            for (int q = 0; q < 4; ++q) v += o->f[(long)(q * 6 + k) * N + n];
            v += 0.5 * o->dt * bforce(o, k, n);
            u[k * N + n] = o->ustar[k * N + n] + 0.5 * o->dt * v;
        }
}

void orc_populations(const orc *o, double *f) { memcpy(f, o->f, (size_t)24 * o->N * sizeof(double)); }
void orc_set_populations(orc *o, const double *f) { memcpy(o->f, f, (size_t)24 * o->N * sizeof(double)); }
int orc_status(const orc *o) { return o->status; }
long orc_step_count(const orc *o) { return o->step; }
double orc_time(const orc *o) { return o->step * o->dt; }
double orc_dt(const orc *o) { return o->dt; }

/* ======================================================================
 * Reference adjoint (the paper has none): the exact discrete adjoint of the
 * steps above, for the loss
 *   L = 1/2 sum_k sum_s |u(X_s, t^{n_k}) - d_{k,s}|^2
 * of displacements u^n = u*^n + (dt/2) v^n (Eq. 22) at sensor nodes X_s and
 * recorded steps n_k, with respect to the per-node shear modulus mu (lambda =
 * lam_ratio mu) and the initial velocity v0. Plain reverse sweep over stored
 * forward states, one phase of the step at a time in reverse order, each
 * phase transposed from its own definition:
 *   collision  local 24 x 24 Jacobian of Eq. (14) by the complex step, and
 *              the exact mu-derivative of an affine map (central difference);
 *   streaming  the transposed permutation of Eq. (15);
 *   edges      Eq. (23) with D and S; for a traction edge the implicit
 *              function theorem on N_a P_ia(F^b) = T_i (Sec. 3.6.2) gives
 *              how the normal column of F^b moves with the node's tangential
 *              column and with mu;
 *   quadrature Eq. (22);
 *   init       Eqs. (16)-(21) are linear in v0 and affine in each node's mu
 *              (P and C are linear in (lambda, mu) for SVK, NH and log-NH), so
 *              their Jacobian columns are exact central differences.
 * Node form of F^b only. Memory: every f^n is kept (small lattices only).
 * ====================================================================== */

/* Eq. (14) at one node in complex arithmetic (for the complex-step Jacobian) */
static void collide_c(const orc *o, const double *prm, double b1, double b2, const double complex f[24],
                      double complex fs[24])
{
    const double c = o->c, dt = o->dt, w = o->omega;
    double complex U[6], F[4], P[4], PhiX[6], PhiY[6];
    int q, k;
    for (k = 0; k < 6; ++k) {
        U[k] = 0.0;
        for (q = 0; q < 4; ++q) U[k] += f[q * 6 + k];
    }
    U[0] += 0.5 * dt * b1;
    U[1] += 0.5 * dt * b2;
    for (k = 0; k < 4; ++k) F[k] = U[2 + k];
    piola_c(o->law, prm, F, P);
    PhiX[0] = -P[0]; PhiX[1] = -P[2]; PhiX[2] = -U[0]; PhiX[3] = 0.0; PhiX[4] = -U[1]; PhiX[5] = 0.0;
    PhiY[0] = -P[1]; PhiY[1] = -P[3]; PhiY[2] = 0.0; PhiY[3] = -U[0]; PhiY[4] = 0.0; PhiY[5] = -U[1];
    for (q = 0; q < 4; ++q)
        for (k = 0; k < 6; ++k) {
            const double complex feq = 0.25 * (U[k] + (2.0 / c) * (CI[q] * PhiX[k] + CJ[q] * PhiY[k]));
            const double Bk = (k == 0) ? b1 : (k == 1) ? b2 : 0.0;
            fs[q * 6 + k] = f[q * 6 + k] + w * (feq - f[q * 6 + k]) + dt * (2.0 - w) * 0.125 * Bk;
        }
}

/* U^n of every node from o->f into o->U (Eq. 10) */
static void recover_all(orc *o)
{
    const long N = o->N;
    long n;
    int q, k;
    for (n = 0; n < N; ++n)
        for (k = 0; k < 6; ++k) {
            double sum = 0.0;
            for (q = 0; q < 4; ++q) sum += o->f[(long)(q * 6 + k) * N + n];
            if (k < 2) sum += 0.5 * o->dt * bforce(o, k, n);
            o->U[k * N + n] = sum;
        }
}

/* 2 x 2 solve A^T z = b */
static void solve2t(const double A[4], const double b[2], double z[2])
{
    const double det = A[0] * A[3] - A[1] * A[2];
    /* A^T = [[A0, A2], [A1, A3]] */
    z[0] = (A[3] * b[0] - A[2] * b[1]) / det;
    z[1] = (-A[1] * b[0] + A[0] * b[1]) / det;
}

int orc_adjoint(orc *o, const double *U0, int order, int nsteps, int nsens, const long *sens, int nrec,
                const int *rec_steps, const double *target, double *loss, double *g_mu, double *g_v0)
{
    const long N = o->N;
    const double dt = o->dt;
    static const int dmiss[4] = {0, 2, 1, 3}, dout[4] = {2, 0, 3, 1};
    double *fh = NULL, *uh = NULL, *fb = NULL, *fbn = NULL, *fsb = NULL, *Ub = NULL, *ub = NULL, *U0p = NULL,
           *mu_save = NULL;
    long m;
    int step, k, q, e, rc = 0;
    if (!o->mufield || o->fb_mode != ORC_FB_NODE || nsteps < 0) return -1;
    for (k = 0; k < nrec; ++k)
        if (rec_steps[k] < 0 || rec_steps[k] > nsteps) return -1;
    for (k = 0; k < nsens; ++k)
        if (sens[k] < 0 || sens[k] >= N) return -1;
    fh = (double *)malloc((size_t)(nsteps + 1) * 24 * N * sizeof(double));
    uh = (double *)malloc((size_t)(nsteps + 1) * 2 * N * sizeof(double));
    fb = (double *)calloc((size_t)24 * N, sizeof(double));
    fbn = (double *)calloc((size_t)24 * N, sizeof(double));
    fsb = (double *)calloc((size_t)24 * N, sizeof(double));
    Ub = (double *)calloc((size_t)6 * N, sizeof(double));
    ub = (double *)calloc((size_t)2 * N, sizeof(double));
    U0p = (double *)malloc((size_t)6 * N * sizeof(double));
    mu_save = (double *)malloc((size_t)N * sizeof(double));
    if (!fh || !uh || !fb || !fbn || !fsb || !Ub || !ub || !U0p || !mu_save) {
        rc = -2;
        goto done;
    }
    /* forward, keeping every f^n and u*^n */
    if (orc_init(o, U0, NULL, order, NULL, NULL) != 0) {
        rc = -3;
        goto done;
    }
    for (step = 0; step <= nsteps; ++step) {
        if (step > 0) orc_step(o, 1);
        memcpy(fh + (size_t)step * 24 * N, o->f, (size_t)24 * N * sizeof(double));
        memcpy(uh + (size_t)step * 2 * N, o->ustar, (size_t)2 * N * sizeof(double));
    }
    if (o->status) {
        rc = -4;
        goto done;
    }
    /* loss */
    *loss = 0.0;
    for (k = 0; k < nrec; ++k) {
        const double *f = fh + (size_t)rec_steps[k] * 24 * N, *us = uh + (size_t)rec_steps[k] * 2 * N;
        int s2, cc;
        for (s2 = 0; s2 < nsens; ++s2)
            for (cc = 0; cc < 2; ++cc) {
                const long nn = sens[s2];
                double v = 0.5 * dt * bforce(o, cc, nn), r;
                for (q = 0; q < 4; ++q) v += f[(long)(q * 6 + cc) * N + nn];
                r = us[cc * N + nn] + 0.5 * dt * v - target[((size_t)k * nsens + s2) * 2 + cc];
                *loss += 0.5 * r * r;
            }
    }
    for (m = 0; m < N; ++m) g_mu[m] = 0.0;
    /* reverse sweep */
    for (step = nsteps; step >= 0; --step) {
        /* loss terms of u^step = u*^step + (dt/2) v^step */
        for (k = 0; k < nrec; ++k) {
            const double *f = fh + (size_t)step * 24 * N, *us = uh + (size_t)step * 2 * N;
            int s2, cc;
            if (rec_steps[k] != step) continue;
            for (s2 = 0; s2 < nsens; ++s2)
                for (cc = 0; cc < 2; ++cc) {
                    const long nn = sens[s2];
                    double v = 0.5 * dt * bforce(o, cc, nn), r;
                    for (q = 0; q < 4; ++q) v += f[(long)(q * 6 + cc) * N + nn];
                    r = us[cc * N + nn] + 0.5 * dt * v - target[((size_t)k * nsens + s2) * 2 + cc];
                    ub[cc * N + nn] += r;
                    for (q = 0; q < 4; ++q) fb[(long)(q * 6 + cc) * N + nn] += 0.5 * dt * r;
                }
        }
        if (step == 0) break;
        /* the forward step (step - 1) -> step, transposed */
        memcpy(o->f, fh + (size_t)(step - 1) * 24 * N, (size_t)24 * N * sizeof(double));
        recover_all(o);
        memset(Ub, 0, (size_t)6 * N * sizeof(double));
        memset(fsb, 0, (size_t)24 * N * sizeof(double));
        /* quadrature u*^step = u*^(step-1) + dt v^(step-1): ub passes through */
        for (m = 0; m < N; ++m)
            for (k = 0; k < 2; ++k) Ub[k * N + m] += dt * ub[k * N + m];
        /* streaming: f^step_q(x + e_q) = f*_q(x) */
        {
            int ix, iy;
            for (iy = 0; iy < o->ny; ++iy)
                for (ix = 0; ix < o->nx; ++ix)
                    for (q = 0; q < 4; ++q) {
                        int tx = ix + CI[q], ty = iy + CJ[q];
                        if (tx < 0 || tx >= o->nx) {
                            if (!xper(o)) continue;
                            tx = (tx + o->nx) % o->nx;
                        }
                        if (ty < 0 || ty >= o->ny) {
                            if (!yper(o)) continue;
                            ty = (ty + o->ny) % o->ny;
                        }
                        for (k = 0; k < 6; ++k)
                            fsb[(long)(q * 6 + k) * N + nid(o, ix, iy)] += fb[(long)(q * 6 + k) * N + nid(o, tx, ty)];
                    }
        }
        /* edges: f_d(x_b) = D f*_{-d}(x_b) + S_d */
        for (e = 0; e < 4; ++e) {
            const orc_edge *E = &o->e[e];
            const int len = edge_len(o, e);
            int p;
            if (E->kind == ORC_PERIODIC) continue;
            for (p = 0; p < len; ++p) {
                const long nb = edge_node(o, e, 0, p);
                double D[6];
                int kk;
                if (E->kind == ORC_VELOCITY) {
                    D[0] = -1; D[1] = -1; D[2] = 1; D[3] = 1; D[4] = 1; D[5] = 1;
                } else {
                    D[0] = 1; D[1] = 1; D[2] = -1; D[3] = -1; D[4] = -1; D[5] = -1;
                }
                for (kk = 0; kk < 6; ++kk)
                    fsb[(long)(dout[e] * 6 + kk) * N + nb] += D[kk] * fb[(long)(dmiss[e] * 6 + kk) * N + nb];
                if (E->kind == ORC_TRACTION) {
                    /* S_F = F^b / 2 with F^b(U^(step-1) at x_b, mu(x_b)) */
                    const int a = (e == ORC_LEFT || e == ORC_RIGHT) ? 0 : 1, tc = 1 - a;
                    const double Na = (e == ORC_LEFT || e == ORC_BOTTOM) ? -1.0 : 1.0;
                    double val[2], Fb[4], Ct[16], Jn[4], Jt[4], Fbb[4], rhs[2], z[2], Pr[4];
                    double pb[8], unit[8] = {0};
                    int i, j;
                    const double *prm = node_prm(o, nb, pb);
                    edge_value(o, e, p, (step - 1) * dt + 0.5 * dt, val);
                    if (boundary_F(o, e, p, val, Fb) != 0) {
                        rc = -5;
                        goto done;
                    }
                    for (kk = 0; kk < 4; ++kk) Fbb[kk] = 0.5 * fb[(long)(dmiss[e] * 6 + 2 + kk) * N + nb];
                    orc_tangent(o->law, prm, Fb, Ct);
                    for (i = 0; i < 2; ++i)
                        for (j = 0; j < 2; ++j) {
                            Jn[i * 2 + j] = Na * Ct[(i * 2 + a) * 4 + (j * 2 + a)];
                            Jt[i * 2 + j] = Na * Ct[(i * 2 + a) * 4 + (j * 2 + tc)];
                        }
                    /* z = -Jn^{-T} Fbb_normal */
                    rhs[0] = -Fbb[0 * 2 + a];
                    rhs[1] = -Fbb[1 * 2 + a];
                    solve2t(Jn, rhs, z);
                    for (j = 0; j < 2; ++j)
                        Ub[(2 + j * 2 + tc) * N + nb] += Fbb[j * 2 + tc] + z[0] * Jt[0 * 2 + j] + z[1] * Jt[1 * 2 + j];
                    /* dr/dmu = Na P_ia(F^b; lam_ratio, 1) */
                    unit[0] = o->lam_ratio;
                    unit[1] = 1.0;
                    orc_piola(o->law, unit, Fb, Pr);
                    g_mu[nb] += z[0] * Na * Pr[0 * 2 + a] + z[1] * Na * Pr[1 * 2 + a];
                }
            }
        }
        /* collision, node by node */
        for (m = 0; m < N; ++m) {
            double pb[8], pp[8] = {0}, pm[8] = {0};
            const double *prm = node_prm(o, m, pb);
            const double b1 = bforce(o, 0, m), b2 = bforce(o, 1, m);
            double complex fc[24], fsc[24];
            double f[24], sb[24], dmu = 0.0;
            int i, j;
            for (j = 0; j < 24; ++j) {
                f[j] = o->f[(long)j * N + m];
                sb[j] = fsb[(long)j * N + m];
            }
            for (j = 0; j < 24; ++j) {
                double acc = 0.0;
                for (i = 0; i < 24; ++i) fc[i] = f[i];
                fc[j] += 1e-30 * I;
                collide_c(o, prm, b1, b2, fc, fsc);
                for (i = 0; i < 24; ++i) acc += (cimag(fsc[i]) / 1e-30) * sb[i];
                fbn[(long)j * N + m] = acc + Ub[(j % 6) * N + m];
            }
            /* d fs / d mu: affine in mu, central difference over +-mu/2 */
            pp[0] = o->lam_ratio * 1.5 * o->mufield[m];
            pp[1] = 1.5 * o->mufield[m];
            pm[0] = o->lam_ratio * 0.5 * o->mufield[m];
            pm[1] = 0.5 * o->mufield[m];
            {
                double complex fp[24], fm[24];
                for (i = 0; i < 24; ++i) fc[i] = f[i];
                collide_c(o, pp, b1, b2, fc, fp);
                collide_c(o, pm, b1, b2, fc, fm);
                for (i = 0; i < 24; ++i) dmu += (creal(fp[i]) - creal(fm[i])) / o->mufield[m] * sb[i];
            }
            g_mu[m] += dmu;
        }
        {
            double *t = fb;
            fb = fbn;
            fbn = t;
        }
    }
    /* init: f^0 = init(U0; mu), u*^0 = u0 - (dt/2) v0. f^0 at node j depends
     * on U0 at j and at the nodes of its finite-difference stencils (same row
     * or column, at most two away) and on mu at j only */
    memcpy(mu_save, o->mufield, (size_t)N * sizeof(double));
    memcpy(U0p, U0, (size_t)6 * N * sizeof(double));
    for (m = 0; m < N; ++m) {
        const int mx = (int)(m % o->nx), my = (int)(m / o->nx);
        long nb[10];
        int nn = 0, d, t, cc;
        for (d = -2; d <= 2; ++d) {
            int jx = mx + d, jy = my + d;
            if (xper(o)) jx = ((jx % o->nx) + o->nx) % o->nx;
            if (yper(o)) jy = ((jy % o->ny) + o->ny) % o->ny;
            if (jx >= 0 && jx < o->nx) nb[nn++] = nid(o, jx, my);
            if (d != 0 && jy >= 0 && jy < o->ny) nb[nn++] = nid(o, mx, jy);
        }
        for (cc = 0; cc < 2; ++cc) {
            double acc = 0.0;
            for (t = 0; t < nn; ++t) {
                const long j = nb[t];
                int dup = 0, u;
                double fp[24], fm[24];
                for (u = 0; u < t; ++u) dup |= (nb[u] == j);
                if (dup) continue;
                U0p[cc * N + m] = U0[cc * N + m] + 1.0;
                init_at(o, U0p, order, NULL, NULL, (int)(j % o->nx), (int)(j / o->nx), fp);
                U0p[cc * N + m] = U0[cc * N + m] - 1.0;
                init_at(o, U0p, order, NULL, NULL, (int)(j % o->nx), (int)(j / o->nx), fm);
                U0p[cc * N + m] = U0[cc * N + m];
                for (u = 0; u < 24; ++u) acc += 0.5 * (fp[u] - fm[u]) * fb[(long)u * N + j];
            }
            g_v0[cc * N + m] = acc - 0.5 * dt * ub[cc * N + m];
        }
        {
            double fp[24], fm[24], acc = 0.0;
            int u;
            o->mufield[m] = 1.5 * mu_save[m];
            init_at(o, U0, order, NULL, NULL, mx, my, fp);
            o->mufield[m] = 0.5 * mu_save[m];
            init_at(o, U0, order, NULL, NULL, mx, my, fm);
            o->mufield[m] = mu_save[m];
            for (u = 0; u < 24; ++u) acc += (fp[u] - fm[u]) / mu_save[m] * fb[(long)u * N + m];
            g_mu[m] += acc;
        }
    }
    /* leave the lattice in its final forward state */
    memcpy(o->f, fh + (size_t)nsteps * 24 * N, (size_t)24 * N * sizeof(double));
    memcpy(o->ustar, uh + (size_t)nsteps * 2 * N, (size_t)2 * N * sizeof(double));
    o->step = nsteps;
done:
    free(fh);
    free(uh);
    free(fb);
    free(fbn);
    free(fsb);
    free(Ub);
    free(ub);
    free(U0p);
    free(mu_save);
    return rc;
}
