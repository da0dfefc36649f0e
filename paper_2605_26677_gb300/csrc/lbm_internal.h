// lbm_internal.h -- host-side declarations shared by the library's
// translation units (kernel launchers); not part of the public C ABI.
#pragma once
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "lbm.h"
#include "lbm_device.cuh"

namespace tlv {
// 16-bit step kernel forced by the environment: LBM_STEP16=regs (register
// kernel, 0) or LBM_STEP16=staged (shared-memory staged kernel, 1); -1 when
// unset, and each context then uses the one its first lbm_step timed faster.
// Task order forced by the environment: LBM_DYN=0 (static grid-stride, 0)
// or LBM_DYN=1 (dynamic claims, 1); -1 when unset, and the first lbm_step
// of each context then times both. LBM_DYN_STRIPES=1 or 4 restricts the
// dynamic claims to that many counters (returned; -1 when unset).
inline int dyn_env_choice()
{
    const char *v = std::getenv("LBM_DYN");
    if (v && !std::strcmp(v, "0")) return 0;
    if (v && !std::strcmp(v, "1")) return 1;
    return -1;
}

inline int stripes_env_choice()
{
    const char *v = std::getenv("LBM_DYN_STRIPES");
    if (v && !std::strcmp(v, "1")) return 1;
    if (v && !std::strcmp(v, "4")) return 4;
    return -1;
}

inline int step16_env_choice()
{
    static const int k = [] {
        const char *v = std::getenv("LBM_STEP16");
        if (v && !std::strcmp(v, "regs")) return 0;
        if (v && !std::strcmp(v, "staged")) return 1;
        return -1;
    }();
    return k;
}
} // namespace tlv

// One lattice: the object behind the opaque lbm_ctx handle of the C ABI.
struct lbm_ctx {
    lbm_config cfg{};
    cudaStream_t st = nullptr;
    int eb = 4;            // bytes per stored population value
    tlv::Layout L{};
    void *f[2] = {nullptr, nullptr};
    double *ustar = nullptr;
    int *d_status = nullptr;
    double *d_diag = nullptr; // diag_blocks * 10 partials + 10 results
    unsigned *d_ctr = nullptr; // two counter sets of the dynamic step kernels (2 x DYN_SET_WORDS)
    int ctr_par = 0;           // which of the pair the next dynamic launch takes
    int dyn = 0;               // task order: 0 static, else dynamic claims over that many
                               // counter stripes (chosen by the first lbm_step, or LBM_DYN)
    double *d_profile[4] = {nullptr, nullptr, nullptr, nullptr};
    int cur = 0;
    long long step = 0;
    double dt = 0.0;
    tlv::Material m{};
    bool have_material = false;
    double b[2] = {0.0, 0.0};
    tlv::EdgeDesc edge[4]{};
    bool initialized = false;
    bool ghosts_dirty = true;  // ghost cells of f[cur] must be rebuilt before the next step
    int grid_step = 1;
    int edge_blk_end[4] = {0, 0, 0, 0};
    std::string err;
    bool prof = false;
    std::vector<cudaEvent_t> ev_step, ev_edge; // start/stop pairs
    std::vector<double> tab_t[4], tab_g[4];  // per-edge tabulated g(t) (LBM_T_TABLE)
    double *d_mufield = nullptr;  // per-node mu, compact FP64 (N), or nullptr
    void *d_muplane = nullptr;    // the same in the compute type, u* plane layout
    int k16 = 0;                  // 16-bit storage: step kernel (0 register, 1 staged)
    bool tune_pending = true;     // the first lbm_step times the step-launch variants (tune_step)
    cudaStream_t st_copy = nullptr;     // lbm_init's banded host copies (created on first use)
    std::vector<cudaEvent_t> ev_band;   // their per-band events (+ one for the fork)
};


namespace tlv {

// NVTX range around a library call, shown by Nsight tools on their timeline
// (header-only NVTX 3: without an attached tool the calls return at once)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// lbm_step.cu
// fuse: the step kernel also writes the next step's ghost cells (node form)
// storage: STORE_F64 / F32 / BF16 / F16
cudaError_t launch_step(int storage, int law, bool fuse, const void *step_args, int grid, cudaStream_t st);
// ghost cells of the current buffer: k_edges (either F^b form, FP64 Newton)
// and k_ghosts (node form, the fused kernel's arithmetic)
cudaError_t launch_edges(int storage, const EdgeArgs &a, int grid, cudaStream_t st);
cudaError_t launch_ghosts(int storage, const EdgeArgs &a, int grid, cudaStream_t st);
int step_blocks_per_sm(int storage, int law);
int step_vec(int storage);

// lbm_aux.cu
struct InitArgs {
    const double *U0;   // 6 x N compact, device
    const double *u0;   // 2 x N compact, device, or nullptr
    void *fout;         // population buffer that receives f*^0
    double *ustar;
    int *status;
    Layout L;
    Material m;
    double c, dt, dx, omega, b1, b2;
    int order, xper, yper;
    int y0, y1;         // rows [y0, y1) written by this launch (its stencils read
                        // U0 one or two rows beyond them)
};
cudaError_t launch_init(int storage, const InitArgs &a, cudaStream_t st);
// per-node mu (compact FP64) -> compute-type plane in the u* layout (zero padding)
cudaError_t launch_mu_plane(int storage, const double *mu, void *plane, const Layout &L, cudaStream_t st);
// min, max and the number of non-finite values of a device array (host out[3]; synchronises)
cudaError_t launch_field_stats(const double *v, long long n, double out[3], cudaStream_t st);

struct ReadArgs {
    const void *f;      // current post-collision populations
    const double *ustar;
    Layout L;
    Material m;
    double dt, b1, b2;
    double *U;          // 6 x N or nullptr
    double *P;          // 4 x N or nullptr
    double *sigma;      // 4 x N or nullptr
    double *u;          // 2 x N or nullptr
};
cudaError_t launch_read(int storage, const ReadArgs &a, cudaStream_t st);

struct DiagArgs {
    const void *f;
    Layout L;
    Material m;
    double dt, dx, b1, b2;
    double *partial;    // [blocks][10]
    double *out;        // [10]
};
int diag_blocks(const Layout &L);
cudaError_t launch_diag(int storage, const DiagArgs &a, cudaStream_t st);

// lbm_adjoint_kernels.cu (see there for the equations)
template <typename T>
struct AdjArgs {
    const void *fin;    // f*^n, ghosts filled
    const void *ain;    // a^{n+1}
    void *aout;         // a^n (interior and ghost cells; k_adj_fold completes it)
    const T *mufield;   // u* plane layout
    const T *ubar;      // dL/du*, two planes, u* plane layout
    double *gmu;        // dL/dmu accumulator, u* plane layout
    const T *tug_in;    // cotangent of G at traction-edge nodes for every q of a^{n+1} (4 planes)
    T *tug_out;         // the same for a^n
    Layout L;
    int kind[4];        // edge kinds
    T one_m_omega, wq, wi2c, dtT;  // 1 - w, w/4, w/(2c), dt
    T hdtb1, hdtb2, lam_ratio;
    double wi2c_d;
    // dynamic task claims (claim_tasks, as the step kernels): this launch's
    // counter set and the one it zeroes for the next, or nullptr (static)
    unsigned *ctr, *ctr_next;
    int dyn_ns;         // stripes of the claims (1 or DYN_STRIPES) when ctr is set
};
struct RecordArgs {
    const void *f;
    const double *ustar;
    const int *sens;  // (x, y) pairs
    double *out;      // 2 per sensor
    int nsens;
    Layout L;
    double dt, b1, b2;
};
template <typename T>
struct InjectArgs {
    void *aout;
    T *ubar;
    const int *sens;
    const double *rec, *tgt;  // 2 per sensor, this record
    int nsens;
    Layout L;
    double dt;
};
struct AdjInitArgs {
    InitArgs ia;        // the forward's init arguments (U0, material, edges' periodicity)
    const void *a0;     // a^0
    const void *ubar;   // compute-type planes
    double *gmu;        // plane
    double *gv0;        // 2N compact (output)
    double *ghat;       // 4N compact scratch
    const void *tug;    // traction-edge cotangent of G for every q of a^0 (compute type, 4 planes)
    int kind[4];
};
cudaError_t launch_adj(int storage, int law, const void *args, int grid, cudaStream_t st);
int adj_blocks_per_sm(int storage, int law);
int adj_vec_for(int storage);  // nodes per lane of the adjoint kernel
cudaError_t launch_adj_record(int storage, const RecordArgs &a, cudaStream_t st);
cudaError_t launch_adj_inject(int storage, const void *args, cudaStream_t st);
cudaError_t launch_adj_init(int storage, const AdjInitArgs &a, cudaStream_t st);
cudaError_t launch_plane_to_compact(const double *plane, double *out, const Layout &L, cudaStream_t st);

// lbm_api.cu: message returned by lbm_last_error(NULL) on this host thread
void set_thread_error(const std::string &msg);

// lbm_api.cu: context operations shared with the batch entry points
lbm_status ctx_fail(lbm_ctx *c, lbm_status s, const std::string &msg);
lbm_status ctx_map_flags(lbm_ctx *c, int flags);  // device status bits -> status (and message)
lbm_status ctx_ready(lbm_ctx *c);                 // initialized, edges consistent, device current
lbm_status ctx_refresh_ghosts(lbm_ctx *c);        // rebuild stale ghost cells (stream-ordered)
template <typename T>
StepArgs<T> ctx_step_args(const lbm_ctx *c, int cur);  // arguments of the step that reads f[cur]
// the first synchronising step of an initialized context times the
// step-launch variants on its lattice and keeps the fastest (no-op later)
lbm_status ctx_tune_steps(lbm_ctx *c);
double ctx_time_factor(const lbm_ctx *c, int e, long long step);  // g of edge e for the step from f*^step

// lbm_batch_k32.cu / lbm_batch_k16.cu: batched step kernel for (law, nodes
// per lane), or nullptr if that form is not built
const void *batch_kernel_f64(int law, int vec);
const void *batch_kernel_f32(int law, int vec);
const void *batch_kernel_bf16(int law, int vec);
const void *batch_kernel_f16(int law, int vec);

} // namespace tlv
