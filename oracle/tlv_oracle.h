/*
 * tlv_oracle.h -- FP64 CPU oracle for the total-Lagrangian vectorial lattice
 * Boltzmann method (D2Q4 lattice, six-component populations) of Feng & Chu,
 * "A total-Lagrangian vectorial lattice Boltzmann method for finite-strain
 * hyperelastic dynamics".
 *
 * TEST INFRASTRUCTURE. This is the parity reference for the CUDA library. Only
 * the tests, the package smoke check and the benchmark's CPU-baseline leg load
 * it. It shares no code, header or constant with the CUDA sources.
 *
 * Conventions (all arrays are caller-owned, row-major, x fastest):
 *   node (ix, iy) sits at X = ((ix + 1/2) dx, (iy + 1/2) dx); index n = iy*nx + ix.
 *   state U = (v1, v2, F11, F12, F21, F22)                    (Sec. 2.4, Eq. 5)
 *   directions q = 0:(1,0) 1:(0,1) 2:(-1,0) 3:(0,-1)           (Sec. 3.1)
 *   F is passed as F[0]=F11, F[1]=F12, F[2]=F21, F[3]=F22 (F[i][A], i spatial,
 *   A material); the tangent C[iAkB] is stored at index ((i*2+A)*2+k)*2+B.
 *   fields of m components are stored component-major: a[m_index*N + n].
 */
#ifndef TLV_ORACLE_H
#define TLV_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* hyperelastic closures of Appendix A */
enum { ORC_SVK = 0, ORC_NH = 1, ORC_LOGNH = 2, ORC_MR = 3, ORC_YEOH = 4, ORC_GENT = 5 };
/* edges: normal N = (-1,0), (1,0), (0,-1), (0,1) */
enum { ORC_LEFT = 0, ORC_RIGHT = 1, ORC_BOTTOM = 2, ORC_TOP = 3 };
enum { ORC_PERIODIC = 0, ORC_VELOCITY = 1, ORC_TRACTION = 2 };
enum { ORC_T_CONST = 0, ORC_T_LINEAR_RAMP = 1, ORC_T_SIN2_RAMP = 2, ORC_T_SIN_PULSE = 3,
       ORC_T_RICKER = 4 };
/* tangential column of the traction-edge deformation gradient F^b:
 * NODE copies F at the boundary node (the form behind the paper's Table 2),
 * EXTRAP2 extrapolates to the wall and half a step ahead (Eq. B.20) */
enum { ORC_FB_NODE = 0, ORC_FB_EXTRAP2 = 1 };
/* status bits latched by orc_step */
enum { ORC_BAD_J = 1, ORC_NEWTON_FAIL = 2, ORC_NONFINITE = 4 };

typedef struct orc orc;

/* ---- pointwise building blocks (exported for the pin tests) ---- */
/* Parameters per law: SVK, NH, LOGNH: {lambda, mu}; MR: {lambda, c10, c01};
 * YEOH: {lambda, c1, c2, c3}; GENT: {lambda, mu, Jm}. */
int    orc_piola(int law, const double *prm, const double F[4], double P[4]);
double orc_energy(int law, const double *prm, const double F[4]);
int    orc_tangent(int law, const double *prm, const double F[4], double C[16]);
/* complex-argument Piola stress, used for the complex-step tangent; exported so
 * a test can check that its real restriction equals orc_piola */
int    orc_piola_cplx(int law, const double *prm, const double Fre[4], const double Fim[4],
                      double Pre[4], double Pim[4]);
void   orc_flux(const double U[6], const double P[4], double PhiX[6], double PhiY[6]);
void   orc_feq(const double U[6], const double P[4], double c, double feq[24]);
double orc_timefn(int kind, const double *tp, double t);

/* ---- threads: OpenMP threads of the per-node loops (results are
 * bit-identical for every count); n <= 0 leaves the count unchanged ---- */
void   orc_set_threads(int n);
int    orc_threads(void);

/* ---- the lattice ---- */
orc   *orc_new(int nx, int ny, double dx, double c, double omega);
void   orc_free(orc *o);
int    orc_set_law(orc *o, int law, const double *prm, int nprm);
int    orc_set_fb_mode(orc *o, int mode);
/* per-node shear modulus mu_N (N values, > 0) with lambda = lam_ratio * mu for
 * SVK, NH and LOGNH (set the law first; orc_set_law drops the field); NULL
 * reverts to the uniform parameters. Copied. */
int    orc_set_material_field(orc *o, const double *mu_N, double lam_ratio);
void   orc_set_body_force(orc *o, double b1, double b2);
/* per-node body acceleration b(X, t^n) for the current time level; NULL
 * reverts to the uniform value. Copied. */
void   orc_set_body_force_field(orc *o, const double *b2N);
/* edge kind and data: value[2] * profile[s] * g(t), profile NULL means 1 */
int    orc_set_edge(orc *o, int edge, int kind, const double value[2], int timefn,
                    const double tp[4], const double *profile);
/* explicit per-node edge data (2 x edge length, component-major) that replaces
 * value*profile*g for the next steps; NULL clears it. For a velocity edge it is
 * v_D, for a traction edge the nominal traction, both at t^n + dt/2. */
int    orc_set_edge_data(orc *o, int edge, const double *vals);
/* order 0: equilibrium; order 2: second-order initialization. dUdX/dUdY give
 * analytic gradients of U0 (6 x N each); NULL means finite differences. */
int    orc_init(orc *o, const double *U0, const double *u0, int order,
                const double *dUdX, const double *dUdY);
int    orc_step(orc *o, int nsteps);
/* U^n (6N), P(F^n) (4N), Cauchy stress (4N), any may be NULL */
void   orc_state(const orc *o, double *U, double *P, double *sigma);
void   orc_displacement(const orc *o, double *u);
void   orc_populations(const orc *o, double *f);     /* pre-collision f^n, 24N */
void   orc_set_populations(orc *o, const double *f);  /* inverse of the above   */
int    orc_status(const orc *o);
/* Reference adjoint. Runs orc_init(U0, u0 = 0, order) and nsteps steps and
 * returns L = 1/2 sum_k sum_s |u(X_s, t^{n_k}) - d_{k,s}|^2 (sensor node
 * indices sens[nsens], recorded steps rec_steps[nrec] in [0, nsteps], targets
 * d as target[(k * nsens + s) * 2 + c]) with dL/dmu (N, the shear-modulus
 * field; lambda = lam_ratio mu) and dL/dv0 (2N, the initial velocity).
 * Needs a material field and the node form of F^b. Returns 0, or < 0 on bad
 * arguments (-1), allocation (-2), init (-3), a latched status (-4) or a
 * Newton failure (-5). Keeps every forward state: small lattices only. */
int    orc_adjoint(orc *o, const double *U0, int order, int nsteps, int nsens, const long *sens,
                   int nrec, const int *rec_steps, const double *target, double *loss, double *g_mu,
                   double *g_v0);
long   orc_step_count(const orc *o);
double orc_time(const orc *o);
double orc_dt(const orc *o);

#ifdef __cplusplus
}
#endif
#endif
