/*
 * lbm.h -- C ABI of the GB300 (sm_103a) library for the total-Lagrangian
 * vectorial lattice Boltzmann method for finite-strain hyperelastic dynamics
 * (Feng & Chu): a D2Q4 lattice whose four populations per node are
 * six-component vectors carrying the material velocity v and the deformation
 * gradient F.
 *
 * Model (paper sections and equations):
 *   state     U = (v1, v2, F11, F12, F21, F22)                 Sec. 2.4, Eq. (5)
 *   system    dU/dt + dPhi_X/dX + dPhi_Y/dY = B                 Eqs. (6)-(7)
 *   lattice   q = (1,0), (0,1), (-1,0), (0,-1), c = dx/dt        Sec. 3.1
 *   one step  recover U, P(F), equilibrium, BGK collision with
 *             trapezoidal source, streaming, half-way edges,
 *             displacement quadrature                          Sec. 3.7
 *
 * Conventions shared by every call:
 *   - Every function returns lbm_status; nothing is thrown and nothing aborts.
 *     On an error the context is left as it was before the call unless the
 *     description says otherwise, and lbm_last_error() explains it.
 *   - Node (ix, iy), 0 <= ix < nx, 0 <= iy < ny, sits at material point
 *     X = ((ix + 1/2) dx, (iy + 1/2) dx); half-way walls lie dx/2 outside the
 *     first and last node of a non-periodic direction (Sec. 3.6).
 *   - Field arrays are float64, component-major, x fastest:
 *     a[(m * ny + iy) * nx + ix] for component m. N = nx * ny.
 *     U fields have 6 components in the order above, displacement 2 (u1, u2),
 *     stress 4 (P11, P12, P21, P22) or (s11, s12, s21, s22).
 *   - "host" pointers are ordinary (preferably pinned) host memory owned by
 *     the caller and only read or written during the call. "device" pointers
 *     are device memory of the context's GPU owned by the caller; the call
 *     enqueues work that uses them on the context's stream and returns
 *     without waiting.
 *   - All device work of a context runs on lbm_config.stream (NULL = the
 *     legacy default stream). A context must not be used from two host
 *     threads at once.
 *   - Device-side conditions (J <= 0, a traction Newton solve that did not
 *     converge, a non-finite state) are latched in a device status word; the
 *     next call that synchronises (lbm_step, lbm_sync, lbm_read_*) returns the
 *     matching LBM_ERR_* code. The state stays readable after such an error.
 *     lbm_init clears the latch. The staged 16-bit step kernel (chosen by
 *     the first lbm_step, see there) bounds each wait for its
 *     asynchronous copies to one second; one that runs out is latched the
 *     same way and returned as LBM_ERR_CUDA, and the steps that followed it
 *     are not valid.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_API_VERSION 1

typedef struct lbm_ctx lbm_ctx; /* opaque, owned by the library */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,            /* an argument is out of range or inconsistent        */
    LBM_ERR_STATE = 2,          /* call out of order (e.g. step before init)          */
    LBM_ERR_OOM = 3,            /* device or host allocation failed                   */
    LBM_ERR_CUDA = 4,           /* a CUDA runtime call failed, or a bounded device    *
                                 * wait for asynchronous copies ran out               */
    LBM_ERR_NONPOSITIVE_J = 5,  /* some node reached J = det F <= 0 (Sec. 2.2)        */
    LBM_ERR_NEWTON = 6,         /* a traction-edge Newton solve failed (Sec. 3.6.2)   */
    LBM_ERR_NONFINITE = 7,      /* the state became NaN or infinite                   */
    LBM_ERR_UNSUPPORTED = 8     /* valid request the library does not implement       */
} lbm_status;

/* Storage of the populations. Compute is in the storage precision (F64, F32).
 * Populations are stored as offsets from the rest-state equilibrium
 * f_rest = (0, 0, 1/4, 0, 0, 1/4) (Eq. 12 at U = (0,0,1,0,0,1), P(I) = 0). */
typedef enum { LBM_STORE_F64 = 0, LBM_STORE_F32 = 1, LBM_STORE_BF16 = 2, LBM_STORE_F16 = 3 } lbm_storage;

/* Edges and their outward normals N: left (-1,0), right (1,0), bottom (0,-1), top (0,1). */
typedef enum { LBM_EDGE_LEFT = 0, LBM_EDGE_RIGHT = 1, LBM_EDGE_BOTTOM = 2, LBM_EDGE_TOP = 3 } lbm_edge;

/* Edge rules: wrap-around, velocity Dirichlet (Eq. 24), nominal-traction
 * Neumann (Eq. 25). Periodic must be set on both opposite edges. */
typedef enum { LBM_BC_PERIODIC = 0, LBM_BC_VELOCITY = 1, LBM_BC_TRACTION = 2 } lbm_bc;

/* Hyperelastic closures of Appendix A. Parameters:
 *   SVK, NH, LOGNH: {lambda, mu}        (Eqs. A.4, A.5, A.6)
 *   MR: {lambda, c10, c01}; YEOH: {lambda, c1, c2, c3}; GENT: {lambda, mu, Jm} */
typedef enum { LBM_LAW_SVK = 0, LBM_LAW_NH = 1, LBM_LAW_LOGNH = 2, LBM_LAW_MR = 3,
               LBM_LAW_YEOH = 4, LBM_LAW_GENT = 5 } lbm_law;

/* Edge-data time functions g(t); the edge value is value * profile[s] * g(t),
 * evaluated at t^n + dt/2 (Eq. 23). tparams:
 *   CONST: -;  LINEAR_RAMP: {T}: min(t/T, 1);
 *   SIN2_RAMP: {T}: sin^2(pi t / (2T)) for t < T, else 1      (shape of Eq. 33)
 *   SIN_PULSE: {T}: sin(pi t / T) for t < T, else 0            (shape of Eq. 35)
 *   RICKER: {s, t0, t_end}: 2/(sqrt(3s) pi^(1/4)) (1 - z^2) exp(-z^2/2),
 *           z = (t - t0)/s, for t <= t_end, else 0              (Sec. 5.4)
 *   TABLE: -: the edge's table of lbm_set_boundary_table (a measured or
 *          otherwise given load history) */
typedef enum { LBM_T_CONST = 0, LBM_T_LINEAR_RAMP = 1, LBM_T_SIN2_RAMP = 2, LBM_T_SIN_PULSE = 3,
               LBM_T_RICKER = 4, LBM_T_TABLE = 5 } lbm_timefn;

/* Tangential column of the traction-edge boundary deformation gradient F^b
 * (Sec. 3.6.2; the normal column always solves P(F^b) N = T by Newton):
 *   NODE:    F at the boundary node at t^n -- the form that reproduces the
 *            paper's mixed-boundary results (Table 2);
 *   EXTRAP2: linear extrapolation to the wall plus the half-step kinematic
 *            shift (dt/2) dv/dT, so F^b = F(X_b, t + dt/2) + O(dt^2) (Eq. B.20). */
typedef enum { LBM_FB_NODE = 0, LBM_FB_EXTRAP2 = 1 } lbm_fb_mode;

typedef struct {
    int32_t nx, ny;    /* nodes; >= 1 (>= 3 along a non-periodic direction)       */
    double dx;         /* lattice spacing, > 0                                    */
    double c;          /* lattice speed c = dx/dt, > 0 (Sec. 3.1)                 */
    double omega;      /* BGK relaxation rate, 0 < omega <= 2 (Eq. 14)            */
    int32_t storage;   /* lbm_storage                                             */
    int32_t fb_mode;   /* lbm_fb_mode                                             */
    int32_t device;    /* CUDA device ordinal                                     */
    void *stream;      /* cudaStream_t used for all device work; NULL = default    */
} lbm_config;

/* Create a context and allocate its device state (two population buffers of
 * 24 planes each, the FP64 displacement accumulator u*, a status word). Sizes
 * are checked: LBM_ERR_ARG for invalid or oversize grids, LBM_ERR_OOM when the
 * device cannot hold the state. On success *out owns the allocation. */
lbm_status lbm_create(const lbm_config *cfg, lbm_ctx **out);

/* Free everything the context owns. NULL is accepted. Waits for the
 * context's stream. */
void lbm_destroy(lbm_ctx *ctx);

/* Text of the last error on ctx (or, when ctx is NULL, of the last failed
 * call on this host thread that takes no context: lbm_create or
 * lbm_diagnostics_state_noalloc). Valid until the next call on ctx. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Hyperelastic closure and its parameters (Sec. 2.3, Appendix A):
 *   SVK, NH, LOGNH: {lambda, mu}          (mu > 0)
 *   MR:   {lambda, c10, c01}              (c10, c01 >= 0, c10 + c01 > 0)
 *   YEOH: {lambda, c1, c2, c3}            (c1 > 0)
 *   GENT: {lambda, mu, Jm}                (mu > 0, Jm > 0)
 * with lambda + 2 mu_0 > 0 for the small-strain shear modulus mu_0 (2 (c10 +
 * c01) for MR, 2 c1 for Yeoh); LBM_ERR_ARG otherwise. The MR, Yeoh and Gent
 * closures use the isochoric invariants of the plane-strain C (C33 = 1).
 * Needed before lbm_init; set later, it applies from the next step on (the
 * lattice speed is not checked again). Waits for the context's queued work.
 * Replaces a material field. */
lbm_status lbm_set_material(lbm_ctx *ctx, int32_t law, const double *params, int32_t nparams);

/* Per-node material (the paper's closures are pointwise, so Eq. (14) takes
 * them node by node): shear modulus mu (host, N values, finite and > 0) and
 * lambda = lam_ratio * mu, for the SVK, NH or LOGNH closure. Replaces any
 * uniform material (lbm_set_material replaces the field). Every storage
 * type (BF16 and FP16 step with the register kernel). Set before lbm_init (the
 * lattice-speed check of lbm_init uses the stiffest node); set later, it
 * applies from the next step on. Copied; waits for the upload. Contexts with
 * a field cannot join a batch. */
lbm_status lbm_set_material_field(lbm_ctx *ctx, int32_t law, const double *mu, double lam_ratio);
/* The same from a device array mu_dev (N doubles on the context's GPU, read
 * on the context's stream; checked on the device). Synchronises. */
lbm_status lbm_set_material_field_device(lbm_ctx *ctx, int32_t law, const double *mu_dev, double lam_ratio);

/* Uniform body acceleration b = (b1, b2) of Eq. (1); B = (b1, b2, 0, 0, 0, 0)
 * enters the state recovery (Eq. 10) and the collision source (Eq. 14).
 * Must be called before lbm_init (default 0). */
lbm_status lbm_set_body_force(lbm_ctx *ctx, double b1, double b2);

/* Rule and data of one edge. value[2] is v_D for LBM_BC_VELOCITY and the
 * nominal traction T (per reference length) for LBM_BC_TRACTION; both are
 * ignored for LBM_BC_PERIODIC. tparams[4] per lbm_timefn (NULL = zeros).
 * profile (host, NULL = 1) holds one factor per edge node (ny for left and
 * right, nx for bottom and top) and is copied. May be called again between
 * steps; the new data applies from the next step. Default: periodic. */
lbm_status lbm_set_boundary(lbm_ctx *ctx, int32_t edge, int32_t bc, const double value[2],
                            int32_t timefn, const double tparams[4], const double *profile);

/* Tabulated time function of an edge (used when its timefn is LBM_T_TABLE):
 * g(t) piecewise linear through the n points (t[i], g[i]) (host arrays,
 * copied; t strictly increasing), constant before the first and after the
 * last. Stepping an edge with LBM_T_TABLE and no table is LBM_ERR_STATE. May
 * be changed between steps; waits for the context's queued work. */
lbm_status lbm_set_boundary_table(lbm_ctx *ctx, int32_t edge, int32_t n, const double *t, const double *g);

/* Initial state (Sec. 3.4 and 3.5). U0 (host, 6N) holds v0 and F0 = I + Grad u0;
 * u0 (host, 2N, NULL = 0) the initial displacement. order 0 starts from the
 * equilibrium f^eq(U0); order 2 uses f_q = f^eq(U0) - (dt/2) D_q f^eq(U0)
 * (Eqs. 16-21) with second-order central differences (one-sided three-point
 * stencils next to non-periodic edges) for the gradients. Sets t = 0, clears
 * the status latch and starts u* = u0 - (dt/2) v0. Requires lbm_set_material;
 * checks edge pairing and c > sqrt(lambda + 2 mu) (the rest-state P-wave
 * speed). Synchronises. */
lbm_status lbm_init(lbm_ctx *ctx, const double *U0, const double *u0, int32_t order);

/* As lbm_init with device pointers (6N and 2N float64, NULL u0 = 0); enqueued
 * on the stream, does not synchronise. */
lbm_status lbm_init_device(lbm_ctx *ctx, const double *U0_dev, const double *u0_dev, int32_t order);

/* Advance nsteps >= 0 time steps (Sec. 3.7), then wait and return the
 * latched device status. In the node form of F^b, the context's first call
 * with nsteps > 0 after its first lbm_init or lbm_init_device (or its first
 * lbm_adjoint_forward) first times the step-launch variants, which give
 * identical results: the task order (static, or claimed dynamically from
 * device counters) and, with BF16 or FP16 storage and uniform material, the
 * register or the shared-memory staged kernel; a few trial steps leave the
 * state untouched, and the fastest is kept for the context's life (the
 * trials take a u*-sized scratch allocation while they run). Until then, and
 * for lbm_step_async, the register kernel runs in static order.
 * LBM_STEP16=regs or staged, LBM_DYN=0 or 1 and LBM_DYN_STRIPES=1 or 4 in the
 * environment restrict the choice. */
lbm_status lbm_step(lbm_ctx *ctx, int64_t nsteps);

/* As lbm_step without waiting; check later with lbm_sync. */
lbm_status lbm_step_async(lbm_ctx *ctx, int64_t nsteps);

/* The step-launch variant the context runs now (host outputs, either may be
 * NULL): *staged = 1 for the shared-memory staged 16-bit kernel, 0 for the
 * register kernel; *dynamic = 0 for static task order, else the number of
 * device counters the dynamic claims are spread over (1 or 4; 1 only for the
 * 16-bit register kernel). No device work. */
lbm_status lbm_step_variant(const lbm_ctx *ctx, int32_t *staged, int32_t *dynamic);

/* Wait for the context's stream and return the latched device status. */
lbm_status lbm_sync(lbm_ctx *ctx);

/* Current time level n: U^n (6N), P(F^n) (4N, NULL to skip) into host arrays,
 * and t^n = n dt into *t (NULL to skip). Synchronises. */
lbm_status lbm_read_state(lbm_ctx *ctx, double *U, double *P, double *t);
lbm_status lbm_read_state_device(lbm_ctx *ctx, double *U_dev, double *P_dev);

/* Displacement u^n = u*^n + (dt/2) v^n (Eq. 22), 2N float64. */
lbm_status lbm_read_displacement(lbm_ctx *ctx, double *u);
lbm_status lbm_read_displacement_device(lbm_ctx *ctx, double *u_dev);

/* Cauchy stress sigma = J^{-1} P F^T (Sec. 3.5), 4N float64 host. */
lbm_status lbm_read_cauchy(lbm_ctx *ctx, double *sigma);

/* Global diagnostics of the current state, reduced in FP64:
 * out[0..1] sum over nodes of v1, v2; out[2..5] mean F11, F12, F21, F22;
 * out[6] energy dx^2 sum (|v|^2 / 2 + W(F)); out[7] min J; out[8] max J;
 * out[9] max over nodes of the Frobenius norm |F - I|. Synchronises. */
lbm_status lbm_diagnostics(lbm_ctx *ctx, double out[10]);

/* Checkpoint: populations, u*, step count. With buf == NULL, *bytes receives
 * the size needed. lbm_load restores a checkpoint of the same nx, ny and
 * storage (LBM_ERR_ARG otherwise) into an initialised context. */
lbm_status lbm_save(lbm_ctx *ctx, void *buf, size_t *bytes);
lbm_status lbm_load(lbm_ctx *ctx, const void *buf, size_t bytes);

/* Step count n, time t^n and time step dt (any may be NULL). No device work. */
lbm_status lbm_info(lbm_ctx *ctx, int64_t *step, double *t, double *dt);

/* Per-kernel timing with CUDA events on the context's stream. enable != 0
 * starts recording (and clears earlier records), 0 stops. lbm_profile_read
 * synchronises and returns, for each of the kernels below, the number of
 * timed launches and their total device time in milliseconds:
 *   out[0], out[1]: fused collide-stream kernel (launches, ms)
 *   out[2], out[3]: edge reconstruction kernel  (launches, ms) */
lbm_status lbm_profile(lbm_ctx *ctx, int32_t enable);
lbm_status lbm_profile_read(lbm_ctx *ctx, double out[4]);

/* Algorithmic bytes one node-update of the fused step moves in and out of
 * HBM for this context's storage (populations read and written, u* read and
 * written). */
double lbm_bytes_per_node_update(const lbm_ctx *ctx);

/* Diagnostics of a state field without allocating device memory. The paper
 * has no counterpart; this entry point exists for callers that cannot let a
 * library call cudaMalloc -- applications that give out all device memory
 * from their own pool, or loops that must not pay for or be serialised by an
 * allocation. It reduces the caller's FP64 state U_dev (device, 6N,
 * component-major v1, v2, F11, F12, F21, F22; e.g. from
 * lbm_read_state_device) into the caller's out_dev (device, 10 doubles, the
 * layout of lbm_diagnostics) for closure `law` with its params (as
 * lbm_set_material lists them) and spacing dx, on `stream` of `device`,
 * without waiting. The material is uniform: for a context with a per-node
 * shear-modulus field (lbm_set_material_field) the energy out[6] is that of
 * the uniform params passed here, not of the field (the other nine entries
 * do not depend on the material). The call makes `device` current while it
 * runs and restores the calling thread's current device before it returns.
 * Its block partials live in one fixed 1.25 MiB array in the library's device
 * memory (held on every GPU that loads the library until the process exits),
 * so a call takes at most 67,108,864 nodes (8192^2) and returns LBM_ERR_ARG
 * beyond that. The first call on a device looks the array's address up; make
 * that first call before any stream capture. Calls share the array, so calls
 * whose kernels overlap on the GPU race with each other. Errors are reported
 * by lbm_last_error(NULL). */
lbm_status lbm_diagnostics_state_noalloc(const double *U_dev, int32_t nx, int32_t ny, int32_t law,
                                         const double *params, int32_t nparams, double dx, double *out_dev,
                                         int32_t device, void *stream);

/* ------------------------------------------------------------ batches
 * Many lattices ("members": specimens of uneven size, material and edges)
 * advanced together by shared persistent launches. The paper has no
 * counterpart; every member still follows Sec. 3.7 exactly: after
 * lbm_batch_step(b, n, ...) each member holds, bit for bit, the state that
 * lbm_step(member, n) would have produced from the same start.
 *
 * Members are grouped by closure and size class; each group is one launch
 * per step over a work list of (member, row, segment) tasks, and the groups of
 * a step run concurrently. A segment is 32 x vec consecutive nodes of a row
 * ("tile": vec nodes per lane); vec is chosen per size class of nx:
 *   class 0: nx <= 48, 1: nx <= 96, 2: nx <= 192, 3: nx <= 384, 4: larger.
 * Tiles that exist: F64 {1, 2}, F32 {1, 2, 4}, BF16 / F16 {2, 4}. The default
 * tile of a class is the widest whose segment is no wider than the class's
 * largest nx (48, 96, 192, 384; the narrowest if none is); lbm_batch_tune
 * measures them all. The tasks of a group are taken in static order (warp w
 * of W takes tasks w, w + W, ...) or, per size class, in dynamic order
 * (warps claim the next task from a device counter, so that warps slowed by
 * short or edge tasks take fewer); the order changes no result.
 *
 * The batch owns a stream of its own. Every call orders its device work after
 * the work already enqueued on the members' streams, and the members' streams
 * after it. */
typedef struct lbm_batch lbm_batch; /* opaque, owned by the library */

#define LBM_BATCH_MAX_MEMBERS 4096
#define LBM_BATCH_CLASSES 5

/* members: host array of n distinct contexts (1 <= n <= LBM_BATCH_MAX_MEMBERS)
 * created on one device with one storage type and fb_mode LBM_FB_NODE
 * (LBM_ERR_ARG otherwise). The contexts stay owned by the caller, must outlive
 * the batch and can still be used on their own between batch calls. Errors
 * of create are reported by lbm_batch_last_error(NULL). */
lbm_status lbm_batch_create(lbm_ctx *const *members, int32_t n, lbm_batch **out);
void lbm_batch_destroy(lbm_batch *b);
const char *lbm_batch_last_error(const lbm_batch *b);

/* size class of a lattice of width nx (0 .. LBM_BATCH_CLASSES - 1) */
int32_t lbm_batch_size_class(int32_t nx);

/* Tiles (nodes per lane) of the size classes: vec[LBM_BATCH_CLASSES] (host).
 * lbm_batch_set_tile returns LBM_ERR_ARG for a tile that does not exist for
 * the members' storage. */
lbm_status lbm_batch_get_tiles(const lbm_batch *b, int32_t *vec);
lbm_status lbm_batch_set_tile(lbm_batch *b, int32_t size_class, int32_t vec);

/* Task order of the size classes: dynamic[LBM_BATCH_CLASSES] (host), 0 static
 * (the default), 1 dynamic. lbm_batch_set_task_order returns LBM_ERR_ARG for
 * a class out of range or a value other than 0 or 1. */
lbm_status lbm_batch_get_task_orders(const lbm_batch *b, int32_t *dynamic);
lbm_status lbm_batch_set_task_order(lbm_batch *b, int32_t size_class, int32_t dynamic);

/* Autotuner: for every size class that has members, times `reps` (>= 1)
 * launches of that class alone for each tile that exists, in each task order,
 * and keeps the fastest (tile, order); where a class other than the one with
 * the most nodes chose dynamic order, it then times the whole batch with
 * those orders and with static order for those classes, and keeps the
 * faster. The trial launches write only the
 * members' second population buffer and scratch copies of the displacement
 * accumulator and status, so the members' states do not change. us (host,
 * optional) receives LBM_BATCH_CLASSES x 3 doubles: mean microseconds per
 * launch for the tiles in the order listed above, the faster of the two task
 * orders (0 where not tried). Synchronises. */
lbm_status lbm_batch_tune(lbm_batch *b, int32_t reps, double *us);

/* Advance every member by nsteps >= 0 steps. graph_steps = 0 enqueues the
 * launches one by one; an even graph_steps >= 2 captures the launches of
 * graph_steps steps once into a CUDA graph (captured again when the tiles or
 * the members' closures change) and replays it, enqueueing the remainder
 * directly. Every member must be initialised (LBM_ERR_STATE). member_status
 * (host, optional, n) receives each member's status. Synchronises; returns
 * LBM_OK or the status of the first member that failed (whose own
 * lbm_last_error explains it). */
lbm_status lbm_batch_step(lbm_batch *b, int64_t nsteps, int32_t graph_steps, int32_t *member_status);

/* Total nodes of the members, kernel launches per step and graphs captured
 * so far (any may be NULL). No device work. */
lbm_status lbm_batch_info(const lbm_batch *b, int64_t *nodes, int32_t *launches_per_step, int32_t *graphs);

/* ------------------------------------------------------------ adjoint
 * Gradients of the sensor-displacement misfit
 *     L = 1/2 sum_k sum_s | u(X_s, t^{n_k}) - d_{k,s} |^2
 * (u from Eq. (22), sensors X_s at nodes, recorded steps n_k) with respect to
 * the shear-modulus field mu(X) of lbm_set_material_field (lambda = lam_ratio
 * mu throughout) and the initial velocity v0, by the discrete adjoint of the
 * whole run: init (Eqs. 16-21), nsteps steps (collision, streaming, the
 * half-way edges of Eqs. 23-25 with the traction Newton solve differentiated
 * by the implicit function theorem, the quadrature of Eq. 22). The paper has
 * no adjoint; the gradient is that of the discrete scheme as implemented.
 * F0 is held fixed (only v0 of the initial state is differentiated).
 *
 * The forward pass stores the state every checkpoint_every steps (0 = the
 * ceiling of sqrt(nsteps)); the backward pass recomputes each segment from
 * its checkpoint. Device memory: (number of checkpoints + checkpoint_every
 * - 1 + 2) population buffers, and when the device has room another
 * checkpoint_every - 1, with which the recomputation of the next segment
 * runs on a second stream while the adjoint steps of the current one run
 * (the gradient is the same bit for bit). Needs FP64 or FP32 storage and the node form
 * of F^b (LBM_ERR_UNSUPPORTED otherwise) and a material field
 * (LBM_ERR_STATE). The object drives the context it was created on; the
 * context must outlive it. */
typedef struct lbm_adjoint lbm_adjoint; /* opaque, owned by the library */

/* Errors of create are reported by lbm_adjoint_last_error(NULL). Allocates
 * the checkpoint storage. */
lbm_status lbm_adjoint_create(lbm_ctx *ctx, int64_t nsteps, int32_t checkpoint_every, lbm_adjoint **out);
void lbm_adjoint_destroy(lbm_adjoint *adj);
const char *lbm_adjoint_last_error(const lbm_adjoint *adj);

/* sens_xy: host, nsens (x, y) node pairs, distinct; rec_steps: host, nrec
 * distinct steps in [0, nsteps]; target: host, nrec * nsens * 2 values d,
 * index (k * nsens + s) * 2 + component. Copied. */
lbm_status lbm_adjoint_set_loss(lbm_adjoint *adj, int32_t nsens, const int32_t *sens_xy, int32_t nrec,
                                const int32_t *rec_steps, const double *target);

/* Initialises the context from U0_dev (device, 6N, as lbm_init_device, u0 =
 * 0) with the given init order, runs nsteps steps storing checkpoints and
 * sensor readings, and returns L in *loss (host). Synchronises. The context
 * then holds the state after nsteps steps. */
lbm_status lbm_adjoint_forward(lbm_adjoint *adj, const double *U0_dev, int32_t order, double *loss);

/* dL/dmu into g_mu_dev (device, N) and dL/dv0 into g_v0_dev (device, 2N,
 * component-major v1 then v2), for the last lbm_adjoint_forward; the context
 * must not have been stepped since (LBM_ERR_STATE). Synchronises. */
lbm_status lbm_adjoint_backward(lbm_adjoint *adj, double *g_mu_dev, double *g_v0_dev);

/* Checkpoint interval, number of stored population buffers, and the device
 * time of the last forward and backward passes in milliseconds (CUDA events
 * on the context's stream; 0 if not run). Any pointer may be NULL. */
lbm_status lbm_adjoint_info(const lbm_adjoint *adj, int32_t *checkpoint_every, int64_t *stored_states,
                            double *forward_ms, double *backward_ms);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
