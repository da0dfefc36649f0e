// lbm_api.cu -- implementation of the C ABI declared in include/lbm.h.
//
// The context owns two population buffers (each 24 planes, layout in
// lbm_device.cuh), the FP64 displacement accumulator u*, a device status word,
// a device step counter and a small diagnostics scratch area. Every device
// operation is enqueued on the stream given at creation.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace tlv;


static thread_local std::string g_create_err;

void tlv::set_thread_error(const std::string &msg) { g_create_err = msg; }

namespace {

lbm_status fail(lbm_ctx *c, lbm_status s, const std::string &msg)
{
    if (c)
        c->err = msg;
    else
        g_create_err = msg;
    return s;
}

lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *what)
{
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError(); // clear a non-sticky error
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, msg);
}

#define CK(ctx, call)                                                       \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);          \
    } while (0)

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

bool is_finite(double v) { return std::isfinite(v); }

int edge_len(const lbm_ctx *c, int e) { return (e <= EDGE_RIGHT) ? c->L.ny : c->L.nx; }

bool xper(const lbm_ctx *c) { return c->edge[EDGE_LEFT].kind == BC_PERIODIC; }
bool yper(const lbm_ctx *c) { return c->edge[EDGE_BOTTOM].kind == BC_PERIODIC; }

// Edge pairing and minimum sizes (one-sided three-point stencils need 3 nodes).
lbm_status check_edges(lbm_ctx *c)
{
    for (int e = 0; e < 4; ++e)
        if (c->edge[e].kind != BC_PERIODIC && c->edge[e].timefn == TF_TABLE && c->tab_t[e].empty())
            return fail(c, LBM_ERR_STATE, "an edge with LBM_T_TABLE has no table (lbm_set_boundary_table)");
    if ((c->edge[EDGE_LEFT].kind == BC_PERIODIC) != (c->edge[EDGE_RIGHT].kind == BC_PERIODIC))
        return fail(c, LBM_ERR_ARG, "left and right edges must both be periodic or both non-periodic");
    if ((c->edge[EDGE_BOTTOM].kind == BC_PERIODIC) != (c->edge[EDGE_TOP].kind == BC_PERIODIC))
        return fail(c, LBM_ERR_ARG, "bottom and top edges must both be periodic or both non-periodic");
    if (!xper(c) && c->L.nx < 3) return fail(c, LBM_ERR_ARG, "nx >= 3 is needed with non-periodic left/right edges");
    if (!yper(c) && c->L.ny < 3) return fail(c, LBM_ERR_ARG, "ny >= 3 is needed with non-periodic bottom/top edges");
    return LBM_OK;
}

lbm_status map_flags(lbm_ctx *c, int flags)
{
    if (flags & ST_NONFINITE) return fail(c, LBM_ERR_NONFINITE, "the state became non-finite");
    if (flags & ST_BAD_J) return fail(c, LBM_ERR_NONPOSITIVE_J, "a node reached J = det F <= 0");
    if (flags & ST_NEWTON) return fail(c, LBM_ERR_NEWTON, "a traction-edge Newton solve did not converge");
    if (flags & ST_STALL) return fail(c, LBM_ERR_CUDA, "a step kernel's wait for its bulk copies exceeded its time bound");
    return LBM_OK;
}

lbm_status sync_status(lbm_ctx *c)
{
    int flags = 0;
    CK(c, cudaMemcpyAsync(&flags, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    return map_flags(c, flags);
}

} // namespace

// The step that starts from f*^n (n = step) computes f*^{n+1} and writes the
// ghosts the next step pulls, whose edge data belong to t^{n+1} + dt/2
// (Eq. 23). One out-of-line function serves the single and batched paths so
// that both see the same rounding.
static double edge_time(const lbm_ctx *c, int e, double t)
{
    if (c->edge[e].timefn != TF_TABLE) return timefn(c->edge[e].timefn, c->edge[e].tp, t);
    // piecewise linear through (t_i, g_i), constant beyond the first and last point
    const std::vector<double> &ts = c->tab_t[e], &gs = c->tab_g[e];
    if (ts.empty()) return 0.0;
    if (t <= ts.front()) return gs.front();
    if (t >= ts.back()) return gs.back();
    const size_t i = (size_t)(std::upper_bound(ts.begin(), ts.end(), t) - ts.begin());  // ts[i-1] <= t < ts[i]
    const double w = (t - ts[i - 1]) / (ts[i] - ts[i - 1]);
    return gs[i - 1] + w * (gs[i] - gs[i - 1]);
}

__attribute__((noinline)) double tlv::ctx_time_factor(const lbm_ctx *c, int e, long long step)
{
    const double th = ((double)step + 1.5) * c->dt;
    return edge_time(c, e, th);
}

namespace {

template <typename T>
StepArgs<T> step_args(const lbm_ctx *c, int cur)
{
    StepArgs<T> a;
    a.fin = static_cast<const T *>(c->f[cur]);
    a.fout = static_cast<T *>(c->f[cur ^ 1]);
    a.ustar = c->ustar;
    a.status = c->d_status;
    a.L = c->L;
    const double w = c->cfg.omega;
    relax_pair<T>(w, a.omega, a.one_m_omega);
    a.wq = a.omega * T(0.25);  // exact: a power-of-two scaling of the rounded omega
    a.wc = (T)(w * 0.5 / c->cfg.c);
    a.hdtb1 = (T)(0.5 * c->dt * c->b[0]);
    a.hdtb2 = (T)(0.5 * c->dt * c->b[1]);
    a.src1 = (T)(c->dt * (2.0 - w) * 0.125 * c->b[0]);
    a.src2 = (T)(c->dt * (2.0 - w) * 0.125 * c->b[1]);
    a.lam = (T)c->m.lam;
    a.mu = (T)c->m.mu;
    a.p2 = (T)c->m.p2;
    a.p3 = (T)c->m.p3;
    a.mufield = static_cast<const T *>(c->d_muplane);
    a.lam_ratio = (T)c->m.lam_ratio;
    a.c = (T)c->cfg.c;
    a.dt = c->dt;
    for (int e = 0; e < 4; ++e) {
        a.kind[e] = c->edge[e].kind;
        a.value[e][0] = c->edge[e].value[0];
        a.value[e][1] = c->edge[e].value[1];
        a.g[e] = ctx_time_factor(c, e, c->step);
        a.profile[e] = c->edge[e].profile;
    }
    a.gdev = nullptr;
    a.k16 = c->k16;
    a.ctr2 = c->dyn ? c->d_ctr : nullptr;
    a.dyn_ns = c->dyn ? c->dyn : DYN_STRIPES;
    a.ctr_par = const_cast<int *>(&c->ctr_par);  // advanced by the launcher of each dynamic launch
    a.ctr = nullptr;
    a.ctr_next = nullptr;
    return a;
}

EdgeArgs edge_args(const lbm_ctx *c, int cur)
{
    EdgeArgs a;
    a.f = c->f[cur];
    a.L = c->L;
    for (int e = 0; e < 4; ++e) {
        a.e[e] = c->edge[e];
        a.blk_end[e] = c->edge_blk_end[e];
    }
    a.m = c->m;
    a.c = c->cfg.c;
    a.dt = c->dt;
    a.dx = c->cfg.dx;
    a.hdtb1 = 0.5 * c->dt * c->b[0];
    a.hdtb2 = 0.5 * c->dt * c->b[1];
    a.fb_mode = c->cfg.fb_mode;
    a.xper = xper(c);
    a.yper = yper(c);
    // the ghosts of the stored f*^n serve the pull of step n + 1: t^n + dt/2
    const double th = ((double)c->step + 0.5) * c->dt;
    for (int e = 0; e < 4; ++e) a.g[e] = edge_time(c, e, th);
    a.status = c->d_status;
    return a;
}

void clear_profile(lbm_ctx *c)
{
    for (cudaEvent_t e : c->ev_step) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_edge) cudaEventDestroy(e);
    c->ev_step.clear();
    c->ev_edge.clear();
}

lbm_status record(lbm_ctx *c, std::vector<cudaEvent_t> &v)
{
    cudaEvent_t e;
    CK(c, cudaEventCreate(&e));
    v.push_back(e);
    CK(c, cudaEventRecord(e, c->st));
    return LBM_OK;
}

// In the node form of F^b every ghost value depends only on its own boundary
// node, so the step kernel writes the next step's ghosts itself (fused) and
// the separate ghost kernel runs only when they are stale. The extrapolated
// form needs neighbouring nodes and keeps the edge kernel before every step.
template <typename T>
lbm_status do_step(lbm_ctx *c, int64_t nsteps)
{
    const bool prof = c->prof && (c->ev_step.size() < 200000);
    const bool fuse = c->cfg.fb_mode == LBM_FB_NODE;
    for (int64_t i = 0; i < nsteps; ++i) {
        if (!fuse || c->ghosts_dirty) {
            const EdgeArgs ea = edge_args(c, c->cur);
            if (prof && record(c, c->ev_edge) != LBM_OK) return LBM_ERR_CUDA;
            if (fuse)
                CK(c, launch_ghosts(c->cfg.storage, ea, c->edge_blk_end[3], c->st));
            else
                CK(c, launch_edges(c->cfg.storage, ea, c->edge_blk_end[3], c->st));
            if (prof && record(c, c->ev_edge) != LBM_OK) return LBM_ERR_CUDA;
            c->ghosts_dirty = false;
        }
        const StepArgs<T> sa = step_args<T>(c, c->cur);
        if (prof && record(c, c->ev_step) != LBM_OK) return LBM_ERR_CUDA;
        CK(c, launch_step(c->cfg.storage, c->m.law, fuse, &sa, c->grid_step, c->st));
        if (prof && record(c, c->ev_step) != LBM_OK) return LBM_ERR_CUDA;
        c->cur ^= 1;
        c->step += 1;
    }
    return LBM_OK;
}

lbm_status read_device(lbm_ctx *c, double *U, double *P, double *sigma, double *u)
{
    ReadArgs a;
    a.f = c->f[c->cur];
    a.ustar = c->ustar;
    a.L = c->L;
    a.m = c->m;
    a.dt = c->dt;
    a.b1 = c->b[0];
    a.b2 = c->b[1];
    a.U = U;
    a.P = P;
    a.sigma = sigma;
    a.u = u;
    CK(c, launch_read(c->cfg.storage, a, c->st));
    return LBM_OK;
}

// Device-visible address of a host array that the context's GPU can write
// in place, or nullptr: page-locked memory (cudaHostAlloc, cudaHostRegister)
// allocated for that device, which a GB300 reaches over NVLink-C2C at about
// the rate of a copy. The read-out kernels then write the caller's array
// directly: no device staging buffer and no separate copy (8192^2: the state
// read-out 30 -> 17 ms, the displacement 10.5 -> 5.6 ms). Pageable memory
// takes the copy path. The initialization keeps its copy: its stencil reads
// each input value several times, and read in place over NVLink-C2C it took
// 48 ms against 35 ms copied.
static void *host_alias(const lbm_ctx *c, const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type == cudaMemoryTypeHost && at.devicePointer && at.device == c->cfg.device) return at.devicePointer;
    return nullptr;
}

// run fn(device buffer) then copy `count` doubles to host `dst`; a
// page-locked dst is written by fn in place
template <typename Fn>
lbm_status read_to_host(lbm_ctx *c, double *dst, size_t count, Fn fn)
{
    if (double *alias = static_cast<double *>(host_alias(c, dst))) {
        lbm_status s = fn(alias);
        if (s != LBM_OK) return s;
        return sync_status(c);
    }
    double *tmp = nullptr;
    CK(c, cudaMallocAsync((void **)&tmp, count * sizeof(double), c->st));
    lbm_status s = fn(tmp);
    if (s == LBM_OK) {
        cudaError_t e = cudaMemcpyAsync(dst, tmp, count * sizeof(double), cudaMemcpyDeviceToHost, c->st);
        if (e != cudaSuccess) s = cuda_fail(c, e, "cudaMemcpyAsync");
    }
    cudaFreeAsync(tmp, c->st);
    if (s != LBM_OK) return s;
    return sync_status(c);
}

lbm_status check_ready(lbm_ctx *c)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (!c->initialized) return fail(c, LBM_ERR_STATE, "lbm_init has not been called");
    CK(c, cudaSetDevice(c->cfg.device));
    return LBM_OK;
}

struct SaveHeader {
    char magic[8];
    int32_t version, nx, ny, storage;
    int64_t step;
};

// Ghost cells of the current buffer (what the boundary nodes pull at the next
// step): left/right columns of planes q = 0 / 2 and bottom/top rows of planes
// q = 1 / 3, six components each. Checkpoints carry them so that a resumed
// run continues bit for bit.
size_t ghost_elems(const lbm_ctx *c) { return (size_t)12 * ((size_t)c->L.nx + c->L.ny); }

lbm_status copy_ghosts(lbm_ctx *c, char *host, bool to_host)
{
    char *base = static_cast<char *>(c->f[c->cur]);
    const size_t eb = c->eb, pitchb = (size_t)c->L.pitch * eb;
    const int nx = c->L.nx, ny = c->L.ny;
    for (int e = 0; e < 4; ++e) {
        const int q = (e == EDGE_LEFT) ? 0 : (e == EDGE_RIGHT) ? 2 : (e == EDGE_BOTTOM) ? 1 : 3;
        for (int k = 0; k < 6; ++k) {
            const size_t plane = (size_t)(q * 6 + k) * c->L.plane;
            size_t off, width, height, spitch;
            if (e <= EDGE_RIGHT) {  // one column, ny rows
                off = plane + c->L.pitch + c->L.xoff + (e == EDGE_LEFT ? -1 : nx);
                width = eb;
                height = ny;
                spitch = pitchb;
            } else {                // one row of nx nodes
                off = plane + (size_t)(e == EDGE_BOTTOM ? 0 : ny + 1) * c->L.pitch + c->L.xoff;
                width = (size_t)nx * eb;
                height = 1;
                spitch = width;
            }
            char *dev = base + off * eb;
            if (to_host)
                CK(c, cudaMemcpy2DAsync(host, width, dev, spitch, width, height, cudaMemcpyDeviceToHost, c->st));
            else
                CK(c, cudaMemcpy2DAsync(dev, spitch, host, width, width, height, cudaMemcpyHostToDevice, c->st));
            host += width * height;
        }
    }
    return LBM_OK;
}

template <typename T>
lbm_status refresh_ghosts(lbm_ctx *c)
{
    const EdgeArgs ea = edge_args(c, c->cur);
    if (c->cfg.fb_mode == LBM_FB_NODE)
        CK(c, launch_ghosts(c->cfg.storage, ea, c->edge_blk_end[3], c->st));
    else
        CK(c, launch_edges(c->cfg.storage, ea, c->edge_blk_end[3], c->st));
    c->ghosts_dirty = false;
    return LBM_OK;
}

} // namespace

// Parameters of Appendix A per law (SVK, NH, log-NH: lambda, mu; MR: lambda,
// c10, c01; Yeoh: lambda, c1, c2, c3; Gent: lambda, mu, Jm), copied to p[4];
// nullptr if valid, else the reason.
static const char *check_law_params(int law, const double *params, int nparams, double p[4])
{
    static const int need[6] = {2, 2, 2, 3, 4, 3};
    if (law < LBM_LAW_SVK || law > LBM_LAW_GENT) return "unknown law";
    if (!params || nparams < need[law])
        return law <= LBM_LAW_LOGNH ? "expected params {lambda, mu}"
               : law == LBM_LAW_MR  ? "expected params {lambda, c10, c01}"
               : law == LBM_LAW_YEOH ? "expected params {lambda, c1, c2, c3}"
                                     : "expected params {lambda, mu, Jm}";
    for (int i = 0; i < need[law]; ++i) {
        if (!is_finite(params[i])) return "parameters must be finite";
        p[i] = params[i];
    }
    double mus;  // small-strain shear modulus
    switch (law) {
    case LBM_LAW_MR:
        if (p[1] < 0.0 || p[2] < 0.0) return "c10 and c01 must be >= 0";
        mus = 2.0 * (p[1] + p[2]);
        break;
    case LBM_LAW_YEOH: mus = 2.0 * p[1]; break;
    case LBM_LAW_GENT:
        if (!(p[2] > 0.0)) return "Jm must be > 0";
        mus = p[1];
        break;
    default: mus = p[1]; break;
    }
    if (!(mus > 0.0)) return "the shear modulus must be > 0";
    if (!(p[0] + 2.0 * mus > 0.0)) return "lambda + 2 mu must be > 0";
    return nullptr;
}

// small-strain shear modulus of the context's material (for the lattice-speed check)
static double shear_modulus(const Material &m)
{
    return m.law == LBM_LAW_MR ? 2.0 * (m.mu + m.p2) : m.law == LBM_LAW_YEOH ? 2.0 * m.mu : m.mu;
}

static void drop_material_field(lbm_ctx *c)
{
    cudaFree(c->d_mufield);
    cudaFree(c->d_muplane);
    c->d_mufield = nullptr;
    c->d_muplane = nullptr;
    c->m.mufield = nullptr;
    c->m.lam_ratio = 0.0;
}

static lbm_status set_step_grid(lbm_ctx *c)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->cfg.device);
    const int per_sm = step_blocks_per_sm(c->cfg.storage, c->m.law);
    const int vec = step_vec(c->cfg.storage);
    const long long tasks = (long long)c->L.ny * ((c->L.nx + 32 * vec - 1) / (32 * vec));
    const long long needed = (tasks + 3) / 4; // 4 warps per block
    long long g = (long long)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    if (g > needed) g = needed;
    c->grid_step = (int)(g < 1 ? 1 : g);
    return LBM_OK;
}

namespace tlv {

lbm_status ctx_fail(lbm_ctx *c, lbm_status s, const std::string &msg) { return fail(c, s, msg); }

lbm_status ctx_map_flags(lbm_ctx *c, int flags) { return map_flags(c, flags); }

lbm_status ctx_ready(lbm_ctx *c)
{
    lbm_status s = check_ready(c);
    return s != LBM_OK ? s : check_edges(c);
}

lbm_status ctx_refresh_ghosts(lbm_ctx *c) { return refresh_ghosts<double>(c); }

template <typename T>
StepArgs<T> ctx_step_args(const lbm_ctx *c, int cur)
{
    return step_args<T>(c, cur);
}
template StepArgs<float> ctx_step_args<float>(const lbm_ctx *, int);
template StepArgs<double> ctx_step_args<double>(const lbm_ctx *, int);

} // namespace tlv

// ====================================================================== ABI

extern "C" {

lbm_status lbm_create(const lbm_config *cfg, lbm_ctx **out)
{
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, LBM_ERR_ARG, "cfg is NULL");
    if (cfg->nx < 1 || cfg->ny < 1) return fail(nullptr, LBM_ERR_ARG, "nx and ny must be >= 1 (empty lattice)");
    if (cfg->nx > (1 << 24) || cfg->ny > (1 << 24)) return fail(nullptr, LBM_ERR_ARG, "nx or ny above 2^24");
    // the step kernels index (row, 64-node segment) tasks with 32-bit integers
    if ((long long)cfg->ny * ((cfg->nx + 63) / 64) >= (1LL << 31)) return fail(nullptr, LBM_ERR_ARG, "grid too large");
    if (!(cfg->dx > 0.0) || !is_finite(cfg->dx)) return fail(nullptr, LBM_ERR_ARG, "dx must be finite and > 0");
    if (!(cfg->c > 0.0) || !is_finite(cfg->c)) return fail(nullptr, LBM_ERR_ARG, "c must be finite and > 0");
    if (!(cfg->omega > 0.0) || !(cfg->omega <= 2.0)) return fail(nullptr, LBM_ERR_ARG, "omega must be in (0, 2]");
    if (cfg->storage < LBM_STORE_F64 || cfg->storage > LBM_STORE_F16) return fail(nullptr, LBM_ERR_ARG, "unknown storage");
    if (cfg->fb_mode != LBM_FB_NODE && cfg->fb_mode != LBM_FB_EXTRAP2) return fail(nullptr, LBM_ERR_ARG, "unknown fb_mode");

    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
    c->cfg = *cfg;
    c->st = static_cast<cudaStream_t>(cfg->stream);
    c->eb = (cfg->storage == LBM_STORE_F64) ? 8 : (cfg->storage == LBM_STORE_F32) ? 4 : 2;
    c->dt = cfg->dx / cfg->c;
    const int line = 128 / c->eb, vec = 16 / c->eb;
    c->L.nx = cfg->nx;
    c->L.ny = cfg->ny;
    c->L.xoff = line;
    c->L.pitch = (int)round_up((long long)line + cfg->nx + vec, line);
    c->L.plane = (long long)(cfg->ny + 2) * c->L.pitch;
    c->L.upitch = (int)round_up((long long)cfg->nx + 4, 16);
    c->L.uplane = (long long)cfg->ny * c->L.upitch;
    for (int e = 0; e < 4; ++e) {
        c->edge[e] = EdgeDesc{};
        c->edge[e].kind = BC_PERIODIC;
    }
    int blk = 0;
    for (int e = 0; e < 4; ++e) {
        blk += (edge_len(c, e) + 127) / 128;
        c->edge_blk_end[e] = blk;
    }
    const size_t fbytes = (size_t)24 * (size_t)c->L.plane * c->eb;
    const size_t ubytes = (size_t)2 * (size_t)c->L.uplane * sizeof(double);

    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) {
        lbm_status s = cuda_fail(nullptr, e, "cudaSetDevice");
        delete c;
        return s;
    }
#define CKC(call)                                                   \
    do {                                                            \
        cudaError_t e2 = (call);                                    \
        if (e2 != cudaSuccess) {                                    \
            lbm_status s2 = cuda_fail(nullptr, e2, #call);          \
            lbm_destroy(c);                                         \
            return s2;                                              \
        }                                                           \
    } while (0)
    CKC(cudaMalloc(&c->f[0], fbytes));
    CKC(cudaMalloc(&c->f[1], fbytes));
    CKC(cudaMalloc((void **)&c->ustar, ubytes));
    CKC(cudaMalloc((void **)&c->d_status, sizeof(int)));
    CKC(cudaMalloc((void **)&c->d_diag, (size_t)(diag_blocks(c->L) * 10 + 10) * sizeof(double)));
    CKC(cudaMalloc((void **)&c->d_ctr, 2 * DYN_SET_WORDS * sizeof(unsigned)));
    CKC(cudaMemset(c->d_ctr, 0, 2 * DYN_SET_WORDS * sizeof(unsigned)));
    c->dyn = tlv::dyn_env_choice() == 1 ? DYN_STRIPES : 0;  // until the first lbm_step chooses
    CKC(cudaMemsetAsync(c->f[0], 0, fbytes, c->st));
    CKC(cudaMemsetAsync(c->f[1], 0, fbytes, c->st));
    CKC(cudaMemsetAsync(c->ustar, 0, ubytes, c->st));
    CKC(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->st));
    CKC(cudaStreamSynchronize(c->st));
#undef CKC
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cfg->device);
    c->grid_step = sms > 0 ? sms : 1; // refined in lbm_set_material (depends on the law)
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->cfg.device);
    cudaStreamSynchronize(c->st);
    clear_profile(c);
    cudaFree(c->f[0]);
    cudaFree(c->f[1]);
    cudaFree(c->ustar);
    cudaFree(c->d_status);
    cudaFree(c->d_diag);
    cudaFree(c->d_ctr);
    for (int e = 0; e < 4; ++e) cudaFree(c->d_profile[e]);
    cudaFree(c->d_mufield);
    cudaFree(c->d_muplane);
    if (c->st_copy) {
        cudaStreamSynchronize(c->st_copy);
        cudaStreamDestroy(c->st_copy);
    }
    for (cudaEvent_t e : c->ev_band) cudaEventDestroy(e);
    delete c;
}

const char *lbm_last_error(const lbm_ctx *c) { return c ? c->err.c_str() : g_create_err.c_str(); }

lbm_status lbm_set_material(lbm_ctx *c, int32_t law, const double *params, int32_t nparams)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    double p[4] = {0.0, 0.0, 0.0, 0.0};
    const char *msg = check_law_params(law, params, nparams, p);
    if (msg) return fail(c, LBM_ERR_ARG, msg);
    CK(c, cudaSetDevice(c->cfg.device));
    CK(c, cudaStreamSynchronize(c->st));  // queued steps may still read the old field
    c->m.law = law; // LBM_LAW_* and tlv::LAW_* share values
    c->m.lam = p[0];
    c->m.mu = p[1];
    c->m.p2 = p[2];
    c->m.p3 = p[3];
    c->have_material = true;
    c->ghosts_dirty = true;  // traction ghosts depend on the material
    drop_material_field(c);
    return set_step_grid(c);
}

static lbm_status field_checks(lbm_ctx *c, int32_t law, const void *mu, double lam_ratio)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (law != LBM_LAW_SVK && law != LBM_LAW_NH && law != LBM_LAW_LOGNH)
        return fail(c, LBM_ERR_ARG, "material fields take the SVK, NH or LOGNH closure");
    if (!mu) return fail(c, LBM_ERR_ARG, "mu is NULL");
    if (!is_finite(lam_ratio) || !(lam_ratio + 2.0 > 0.0)) return fail(c, LBM_ERR_ARG, "lam_ratio must be finite and > -2");
    return LBM_OK;
}

// Copy the field (host or device source) into new buffers, then replace the
// old field; on an error the context keeps its old material.
static lbm_status install_field(lbm_ctx *c, int32_t law, const double *mu, bool from_device, double lam_ratio,
                                double mumax)
{
    const size_t N = (size_t)c->L.nx * c->L.ny;
    const size_t pbytes = (size_t)c->L.uplane * (c->cfg.storage == LBM_STORE_F64 ? 8 : 4);
    double *field = nullptr;
    void *plane = nullptr;
    cudaError_t e = cudaMalloc((void **)&field, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&plane, pbytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(plane, 0, pbytes, c->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(field, mu, N * sizeof(double), from_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            c->st);
    if (e == cudaSuccess) e = launch_mu_plane(c->cfg.storage, field, plane, c->L, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);  // also: queued steps are done with the old field
    if (e != cudaSuccess) {
        cudaFree(field);
        cudaFree(plane);
        return cuda_fail(c, e, "material field upload");
    }
    drop_material_field(c);
    c->d_mufield = field;
    c->d_muplane = plane;
    c->m.law = law;
    c->m.p2 = c->m.p3 = 0.0;
    c->m.mufield = c->d_mufield;
    c->m.lam_ratio = lam_ratio;
    // the uniform pair holds the stiffest node, for the lattice-speed check
    c->m.mu = mumax;
    c->m.lam = lam_ratio * mumax;
    c->have_material = true;
    c->ghosts_dirty = true;
    return set_step_grid(c);
}

lbm_status lbm_set_material_field(lbm_ctx *c, int32_t law, const double *mu, double lam_ratio)
{
    lbm_status s = field_checks(c, law, mu, lam_ratio);
    if (s != LBM_OK) return s;
    const size_t N = (size_t)c->L.nx * c->L.ny;
    double mumax = 0.0;
    for (size_t n = 0; n < N; ++n) {
        if (!is_finite(mu[n]) || !(mu[n] > 0.0)) return fail(c, LBM_ERR_ARG, "mu must be finite and > 0 at every node");
        mumax = std::max(mumax, mu[n]);
    }
    CK(c, cudaSetDevice(c->cfg.device));
    return install_field(c, law, mu, false, lam_ratio, mumax);
}

lbm_status lbm_set_material_field_device(lbm_ctx *c, int32_t law, const double *mu_dev, double lam_ratio)
{
    lbm_status s = field_checks(c, law, mu_dev, lam_ratio);
    if (s != LBM_OK) return s;
    CK(c, cudaSetDevice(c->cfg.device));
    double stats[3];  // min, max, number of non-finite values
    CK(c, launch_field_stats(mu_dev, (long long)c->L.nx * c->L.ny, stats, c->st));
    if (stats[2] > 0.0 || !(stats[0] > 0.0)) return fail(c, LBM_ERR_ARG, "mu must be finite and > 0 at every node");
    return install_field(c, law, mu_dev, true, lam_ratio, stats[1]);
}


lbm_status lbm_set_body_force(lbm_ctx *c, double b1, double b2)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (c->initialized) return fail(c, LBM_ERR_STATE, "the body force must be set before lbm_init");
    if (!is_finite(b1) || !is_finite(b2)) return fail(c, LBM_ERR_ARG, "body force must be finite");
    c->b[0] = b1;
    c->b[1] = b2;
    return LBM_OK;
}

lbm_status lbm_set_boundary(lbm_ctx *c, int32_t edge, int32_t bc, const double value[2], int32_t timefn,
                            const double tparams[4], const double *profile)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (edge < 0 || edge > 3) return fail(c, LBM_ERR_ARG, "edge must be 0..3");
    if (bc < LBM_BC_PERIODIC || bc > LBM_BC_TRACTION) return fail(c, LBM_ERR_ARG, "unknown boundary kind");
    if (timefn < LBM_T_CONST || timefn > LBM_T_TABLE) return fail(c, LBM_ERR_ARG, "unknown time function");
    EdgeDesc d{};
    d.kind = bc;
    d.timefn = timefn;
    d.value[0] = value ? value[0] : 0.0;
    d.value[1] = value ? value[1] : 0.0;
    for (int i = 0; i < 4; ++i) d.tp[i] = tparams ? tparams[i] : 0.0;
    if (!is_finite(d.value[0]) || !is_finite(d.value[1])) return fail(c, LBM_ERR_ARG, "edge value must be finite");
    for (int i = 0; i < 4; ++i)
        if (!is_finite(d.tp[i])) return fail(c, LBM_ERR_ARG, "time-function parameters must be finite");
    if ((timefn == LBM_T_LINEAR_RAMP || timefn == LBM_T_SIN2_RAMP || timefn == LBM_T_SIN_PULSE) && !(d.tp[0] > 0.0))
        return fail(c, LBM_ERR_ARG, "ramp and pulse durations must be > 0");
    if (timefn == LBM_T_RICKER && !(d.tp[0] > 0.0)) return fail(c, LBM_ERR_ARG, "Ricker width must be > 0");
    const int len = edge_len(c, edge);
    if (profile)
        for (int i = 0; i < len; ++i)
            if (!is_finite(profile[i])) return fail(c, LBM_ERR_ARG, "profile must be finite");
    CK(c, cudaSetDevice(c->cfg.device));
    // an earlier edge kernel may still read the old profile
    CK(c, cudaStreamSynchronize(c->st));
    if (profile) {
        if (!c->d_profile[edge]) CK(c, cudaMalloc((void **)&c->d_profile[edge], (size_t)len * sizeof(double)));
        CK(c, cudaMemcpy(c->d_profile[edge], profile, (size_t)len * sizeof(double), cudaMemcpyHostToDevice));
        d.profile = c->d_profile[edge];
    } else {
        d.profile = nullptr;
    }
    c->edge[edge] = d;
    c->ghosts_dirty = true;
    return LBM_OK;
}

lbm_status lbm_set_boundary_table(lbm_ctx *c, int32_t edge, int32_t n, const double *t, const double *g)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (edge < 0 || edge > 3) return fail(c, LBM_ERR_ARG, "edge must be 0..3");
    if (n < 1 || !t || !g) return fail(c, LBM_ERR_ARG, "a table needs n >= 1 points");
    for (int i = 0; i < n; ++i) {
        if (!is_finite(t[i]) || !is_finite(g[i])) return fail(c, LBM_ERR_ARG, "table entries must be finite");
        if (i > 0 && !(t[i] > t[i - 1])) return fail(c, LBM_ERR_ARG, "table times must increase strictly");
    }
    CK(c, cudaSetDevice(c->cfg.device));
    CK(c, cudaStreamSynchronize(c->st));  // steps already queued used the old table on the host
    c->tab_t[edge].assign(t, t + n);
    c->tab_g[edge].assign(g, g + n);
    c->ghosts_dirty = true;
    return LBM_OK;
}

static InitArgs init_args(const lbm_ctx *c, const double *U0_dev, const double *u0_dev, int32_t order)
{
    InitArgs a;
    a.U0 = U0_dev;
    a.u0 = u0_dev;
    a.fout = c->f[0];
    a.ustar = c->ustar;
    a.status = c->d_status;
    a.L = c->L;
    a.m = c->m;
    a.c = c->cfg.c;
    a.dt = c->dt;
    a.dx = c->cfg.dx;
    a.omega = c->cfg.omega;
    a.b1 = c->b[0];
    a.b2 = c->b[1];
    a.order = order;
    a.xper = xper(c);
    a.yper = yper(c);
    a.y0 = 0;
    a.y1 = c->L.ny;
    return a;
}

static void init_done(lbm_ctx *c)
{
    c->cur = 0;
    c->step = 0;
    c->initialized = true;
    c->ghosts_dirty = true;
}

static lbm_status init_common(lbm_ctx *c, const double *U0_dev, const double *u0_dev, int32_t order)
{
    const InitArgs a = init_args(c, U0_dev, u0_dev, order);
    CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->st));
    CK(c, launch_init(c->cfg.storage, a, c->st));
    init_done(c);
    return LBM_OK;
}

// lbm_init from host arrays: the copy of U0 (and u0) in row bands on the
// context's copy stream, overlapped with the initialization of the bands
// already copied on the context's stream. Band b's stencils read up to two
// rows past it (one-sided at a non-periodic edge, one row when periodic), so
// it starts once band b + 1 has arrived; with periodic rows band 0 also needs
// the last row and goes last. Bands hold at least INIT_BAND_MIN_ROWS rows, so
// the rows a band's stencils reach lie in the next band.
constexpr int INIT_BANDS = 8;
constexpr int INIT_BAND_MIN_ROWS = 4;
constexpr size_t INIT_PIPELINE_MIN_BYTES = size_t(64) << 20;

static lbm_status init_from_host(lbm_ctx *c, const double *U0, const double *u0, int32_t order, double *dU,
                                 double *du)
{
    const int nx = c->L.nx, ny = c->L.ny;
    const size_t N = (size_t)nx * ny;
    int K = INIT_BANDS;
    if (6 * N * sizeof(double) < INIT_PIPELINE_MIN_BYTES) K = 1;
    if (ny / INIT_BAND_MIN_ROWS < K) K = ny / INIT_BAND_MIN_ROWS;
    if (K <= 1) {
        CK(c, cudaMemcpyAsync(dU, U0, 6 * N * sizeof(double), cudaMemcpyHostToDevice, c->st));
        if (u0) CK(c, cudaMemcpyAsync(du, u0, 2 * N * sizeof(double), cudaMemcpyHostToDevice, c->st));
        return init_common(c, dU, du, order);
    }
    if (!c->st_copy) CK(c, cudaStreamCreateWithFlags(&c->st_copy, cudaStreamNonBlocking));
    while ((int)c->ev_band.size() < K + 1) {
        cudaEvent_t e;
        CK(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->ev_band.push_back(e);
    }
    // the copies follow the allocations (and earlier work) of the context's stream
    CK(c, cudaEventRecord(c->ev_band[K], c->st));
    CK(c, cudaStreamWaitEvent(c->st_copy, c->ev_band[K], 0));
    std::vector<int> y(K + 1);
    for (int b = 0; b <= K; ++b) y[b] = (int)((long long)ny * b / K);
    for (int b = 0; b < K; ++b) {
        const size_t off = (size_t)y[b] * nx, len = (size_t)(y[b + 1] - y[b]) * nx * sizeof(double);
        for (int k = 0; k < 6; ++k)
            CK(c, cudaMemcpyAsync(dU + k * N + off, U0 + k * N + off, len, cudaMemcpyHostToDevice, c->st_copy));
        if (u0)
            for (int k = 0; k < 2; ++k)
                CK(c, cudaMemcpyAsync(du + k * N + off, u0 + k * N + off, len, cudaMemcpyHostToDevice, c->st_copy));
        CK(c, cudaEventRecord(c->ev_band[b], c->st_copy));
    }
    InitArgs a = init_args(c, dU, du, order);
    CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->st));
    for (int i = 0; i < K; ++i) {
        const int b = a.yper ? (i + 1) % K : i;  // periodic rows: band 0 last
        const int need = (a.yper && b == 0) ? K - 1 : std::min(b + 1, K - 1);
        CK(c, cudaStreamWaitEvent(c->st, c->ev_band[need], 0));
        a.y0 = y[b];
        a.y1 = y[b + 1];
        CK(c, launch_init(c->cfg.storage, a, c->st));
    }
    init_done(c);
    return LBM_OK;
}

// Step-launch variants: which 16-bit kernel (registers, or rows staged in
// shared memory) and which task order (static grid-stride, or dynamic claims
// over DYN_STRIPES counters, or for the 16-bit register kernel also over one
// counter). All give bit-identical states, and which is fastest depends on
// the lattice (fraction of the copy bandwidth, static / one counter / striped:
// BF16 4096 x 2048 clamped 0.909 / 0.923 / 0.856, BF16 8192^2 periodic
// 0.918 / 0.718 / 0.924, FP32 4096 x 2048 clamped 0.955 / 0.937 / 0.979,
// FP32 8192^2 periodic 0.960 / 0.958 / 1.009). The first lbm_step of a
// context times the candidates on its lattice and keeps the fastest for the
// context's life. The trials read the current buffer, whose ghost cells are
// refreshed first exactly as the first step would, and write only the other
// buffer, which the first real step overwrites; u* and the status word go to
// scratch, so the state is untouched. LBM_STEP16, LBM_DYN and
// LBM_DYN_STRIPES in the environment restrict the candidates; contexts in
// the extrapolated F^b form, or without room for the scratch, keep the
// register kernel in static order, and contexts with a material field have
// no staged kernel.
} // extern "C"

namespace {

struct StepVariant {
    int k16;  // 16-bit kernel: 0 register, 1 staged
    int dyn;  // 0 static order, else the stripes of the dynamic claims
};

template <typename T>
lbm_status tune_step(lbm_ctx *c)
{
    if (c->cfg.fb_mode != LBM_FB_NODE) return LBM_OK;
    std::vector<StepVariant> cand;
    const int env16 = tlv::step16_env_choice(), envdyn = tlv::dyn_env_choice(), envns = tlv::stripes_env_choice();
    // the staged kernel has no per-node-material form
    for (int k16 = 0; k16 < (c->eb == 2 && !c->d_muplane ? 2 : 1); ++k16)
        for (int d : {0, DYN_STRIPES, 1}) {
            if (d == 1 && (c->eb != 2 || DYN_STRIPES == 1)) continue;  // one counter: 16-bit kernels only
            if (k16 == 1 && d != 0) continue;                         // the staged kernel keeps static order
            if ((env16 >= 0 && k16 != env16) || (envdyn >= 0 && (d != 0) != (envdyn == 1))) continue;
            if (envns >= 0 && d != 0 && d != envns) continue;
            cand.push_back({k16, d});
        }
    if (cand.size() == 1) {
        c->k16 = cand[0].k16;
        c->dyn = cand[0].dyn;
    }
    if (cand.size() <= 1) return LBM_OK;
    if (c->ghosts_dirty) {
        // the refresh the first step would make, timed like it when profiling
        const bool prof = c->prof && (c->ev_step.size() < 200000);
        if (prof && record(c, c->ev_edge) != LBM_OK) return LBM_ERR_CUDA;
        lbm_status s = refresh_ghosts<T>(c);
        if (s != LBM_OK) return s;
        if (prof && record(c, c->ev_edge) != LBM_OK) return LBM_ERR_CUDA;
    }
    double *us = nullptr;
    int *st = nullptr;
    const size_t ubytes = (size_t)2 * c->L.uplane * sizeof(double);
    if (cudaMallocAsync((void **)&us, ubytes, c->st) != cudaSuccess) {
        cudaGetLastError();  // clear it: without scratch the default variant runs
        return LBM_OK;
    }
    if (cudaMallocAsync((void **)&st, sizeof(int), c->st) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(us, c->st);
        return LBM_OK;
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaMemsetAsync(us, 0, ubytes, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(int), c->st);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    StepArgs<T> a = step_args<T>(c, c->cur);
    a.ustar = us;
    a.status = st;
    auto set = [&](const StepVariant &v) {
        a.k16 = v.k16;
        a.ctr2 = v.dyn ? c->d_ctr : nullptr;
        a.dyn_ns = v.dyn ? v.dyn : DYN_STRIPES;
    };
    // a warm-up step of each, then three rounds of three steps of each
    // variant, interleaved so that clock changes weigh on all alike
    const int nk = (int)cand.size();
    std::vector<float> ms(nk, 0.f);
    for (int v = 0; v < nk && e == cudaSuccess; ++v) {
        set(cand[v]);
        e = launch_step(c->cfg.storage, c->m.law, true, &a, c->grid_step, c->st);
    }
    for (int round = 0; round < 3 && e == cudaSuccess; ++round)
        for (int v = 0; v < nk && e == cudaSuccess; ++v) {
            set(cand[v]);
            float t = 0.f;
            e = cudaEventRecord(ev[0], c->st);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r)
                e = launch_step(c->cfg.storage, c->m.law, true, &a, c->grid_step, c->st);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->st);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
            ms[v] += t;
        }
    if (e == cudaSuccess) {
        int best = 0;
        for (int v = 1; v < nk; ++v)
            if (ms[v] < ms[best]) best = v;
        c->k16 = cand[best].k16;
        c->dyn = cand[best].dyn;
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    cudaFreeAsync(us, c->st);
    cudaFreeAsync(st, c->st);
    CK(c, e);
    return LBM_OK;
}

} // namespace

lbm_status tlv::ctx_tune_steps(lbm_ctx *c)
{
    if (!c->initialized || !c->tune_pending) return LBM_OK;
    lbm_status s = check_edges(c);
    if (s == LBM_OK) s = (c->eb == 8) ? tune_step<double>(c) : tune_step<float>(c);
    if (s != LBM_OK) return s;
    c->tune_pending = false;
    return LBM_OK;
}


extern "C" {

static lbm_status init_checks(lbm_ctx *c, const void *U0, int32_t order)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (!c->have_material) return fail(c, LBM_ERR_STATE, "lbm_set_material must precede lbm_init");
    if (!U0) return fail(c, LBM_ERR_ARG, "U0 is NULL");
    if (order != 0 && order != 2) return fail(c, LBM_ERR_ARG, "order must be 0 or 2");
    lbm_status s = check_edges(c);
    if (s != LBM_OK) return s;
    const double cP = std::sqrt(c->m.lam + 2.0 * shear_modulus(c->m));
    if (!(c->cfg.c > cP)) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "lattice speed c = %g must exceed the P-wave speed sqrt(lambda + 2 mu) = %g",
                      c->cfg.c, cP);
        return fail(c, LBM_ERR_ARG, buf);
    }
    return LBM_OK;
}

lbm_status lbm_init(lbm_ctx *c, const double *U0, const double *u0, int32_t order)
{
    Range range_("lbm_init");
    lbm_status s = init_checks(c, U0, order);
    if (s != LBM_OK) return s;
    CK(c, cudaSetDevice(c->cfg.device));
    const size_t N = (size_t)c->L.nx * c->L.ny;
    // The copied state is staged in the second population buffer: the
    // initialization writes f[0] and the first step overwrites f[1], and its
    // 24 planes hold U0's 6 N doubles in every storage type (u0's 2 N too,
    // except with 16-bit storage, where u0 gets an allocation of its own).
    const size_t fbytes = (size_t)24 * c->L.plane * c->eb;
    double *dU = static_cast<double *>(c->f[1]), *du = nullptr;
    bool du_owned = false;
    cudaError_t e = cudaSuccess;
    if (u0) {
        if (8 * N * sizeof(double) <= fbytes) {
            du = dU + 6 * N;
        } else {
            e = cudaMallocAsync((void **)&du, 2 * N * sizeof(double), c->st);
            du_owned = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) s = init_from_host(c, U0, u0, order, dU, du);
    if (s != LBM_OK) cudaStreamSynchronize(c->st_copy ? c->st_copy : c->st);  // copies still in flight
    if (du_owned) cudaFreeAsync(du, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "allocating the initial displacement");
    if (s != LBM_OK) return s;
    return sync_status(c);
}

lbm_status lbm_init_device(lbm_ctx *c, const double *U0_dev, const double *u0_dev, int32_t order)
{
    Range range_("lbm_init_device");
    lbm_status s = init_checks(c, U0_dev, order);
    if (s != LBM_OK) return s;
    CK(c, cudaSetDevice(c->cfg.device));
    return init_common(c, U0_dev, u0_dev, order);
}

lbm_status lbm_step_async(lbm_ctx *c, int64_t nsteps)
{
    Range range_("lbm_step");
    lbm_status s = check_ready(c);
    if (s != LBM_OK) return s;
    if (nsteps < 0) return fail(c, LBM_ERR_ARG, "nsteps must be >= 0");
    s = check_edges(c);
    if (s != LBM_OK) return s;
    return (c->eb == 8) ? do_step<double>(c, nsteps) : do_step<float>(c, nsteps);
}

lbm_status lbm_step(lbm_ctx *c, int64_t nsteps)
{
    if (c && nsteps > 0) {
        // the context's first synchronising step picks the step-launch
        // variant for the lattice (tune_step)
        lbm_status s = tlv::ctx_tune_steps(c);
        if (s != LBM_OK) return s;
    }
    lbm_status s = lbm_step_async(c, nsteps);
    if (s != LBM_OK) return s;
    return sync_status(c);
}

lbm_status lbm_step_variant(const lbm_ctx *c, int32_t *staged, int32_t *dynamic)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (staged) *staged = c->k16;
    if (dynamic) *dynamic = c->dyn;
    return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx *c)
{
    lbm_status s = check_ready(c);
    if (s != LBM_OK) return s;
    return sync_status(c);
}

lbm_status lbm_read_state(lbm_ctx *c, double *U, double *P, double *t)
{
    Range range_("lbm_read_state");
    lbm_status s = check_ready(c);
    if (s != LBM_OK) return s;
    if (!U) return fail(c, LBM_ERR_ARG, "U is NULL");
    const size_t N = (size_t)c->L.nx * c->L.ny;
    if (t) *t = c->step * c->dt;
    s = read_to_host(c, U, 6 * N, [&](double *d) { return read_device(c, d, nullptr, nullptr, nullptr); });
    if (s != LBM_OK && s != LBM_ERR_NONFINITE && s != LBM_ERR_NONPOSITIVE_J && s != LBM_ERR_NEWTON) return s;
    if (!P) return s;
    lbm_status s2 = read_to_host(c, P, 4 * N, [&](double *d) { return read_device(c, nullptr, d, nullptr, nullptr); });
    return s != LBM_OK ? s : s2;
}

lbm_status lbm_read_state_device(lbm_ctx *c, double *U_dev, double *P_dev)
{
    lbm_status s = check_ready(c);
    if (s != LBM_OK) return s;
    if (!U_dev && !P_dev) return fail(c, LBM_ERR_ARG, "both outputs are NULL");
    return read_device(c, U_dev, P_dev, nullptr, nullptr);
}

lbm_status lbm_read_displacement(lbm_ctx *c, double *u)
{
    Range range_("lbm_read_displacement");
    lbm_status s = check_ready(c);
    if (s != LBM_OK) return s;
    if (!u) return fail(c, LBM_ERR_ARG, "u is NULL");
    const size_t N = (size_t)c->L.nx * c->L.ny;
    return read_to_host(c, u, 2 * N, [&](double *d) { return read_device(c, nullptr, nullptr, nullptr, d); });
}

lbm_status lbm_read_displacement_device(lbm_ctx *c, double *u_dev)
{
    lbm_status s = check_ready(c);
    if (s != LBM_OK) return s;
    if (!u_dev) return fail(c, LBM_ERR_ARG, "u is NULL");
    return read_device(c, nullptr, nullptr, nullptr, u_dev);
}

lbm_status lbm_read_cauchy(lbm_ctx *c, double *sigma)
{
    lbm_status s = check_ready(c);
    if (s != LBM_OK) return s;
    if (!sigma) return fail(c, LBM_ERR_ARG, "sigma is NULL");
    const size_t N = (size_t)c->L.nx * c->L.ny;
    return read_to_host(c, sigma, 4 * N, [&](double *d) { return read_device(c, nullptr, nullptr, d, nullptr); });
}

lbm_status lbm_diagnostics(lbm_ctx *c, double out[10])
{
    Range range_("lbm_diagnostics");
    lbm_status s = check_ready(c);
    if (s != LBM_OK) return s;
    if (!out) return fail(c, LBM_ERR_ARG, "out is NULL");
    DiagArgs a;
    a.f = c->f[c->cur];
    a.L = c->L;
    a.m = c->m;
    a.dt = c->dt;
    a.dx = c->cfg.dx;
    a.b1 = c->b[0];
    a.b2 = c->b[1];
    a.partial = c->d_diag;
    a.out = c->d_diag + (size_t)diag_blocks(c->L) * 10;
    CK(c, launch_diag(c->cfg.storage, a, c->st));
    CK(c, cudaMemcpyAsync(out, a.out, 10 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    return sync_status(c);
}

lbm_status lbm_save(lbm_ctx *c, void *buf, size_t *bytes)
{
    Range range_("lbm_save");
    lbm_status s = check_ready(c);
    if (s != LBM_OK) return s;
    if (!bytes) return fail(c, LBM_ERR_ARG, "bytes is NULL");
    const size_t N = (size_t)c->L.nx * c->L.ny;
    const size_t need = sizeof(SaveHeader) + 24 * N * c->eb + 2 * N * sizeof(double) + ghost_elems(c) * c->eb;
    if (!buf) {
        *bytes = need;
        return LBM_OK;
    }
    if (*bytes < need) return fail(c, LBM_ERR_ARG, "buffer too small");
    if (c->ghosts_dirty) {
        s = (c->eb == 8) ? refresh_ghosts<double>(c) : refresh_ghosts<float>(c);
        if (s != LBM_OK) return s;
    }
    SaveHeader h{};
    std::memcpy(h.magic, "TLVLBM02", 8);
    h.version = 2;
    h.nx = c->L.nx;
    h.ny = c->L.ny;
    h.storage = c->cfg.storage;
    h.step = c->step;
    std::memcpy(buf, &h, sizeof h);
    char *p = static_cast<char *>(buf) + sizeof h;
    const size_t rowb = (size_t)c->L.nx * c->eb;
    for (int pl = 0; pl < 24; ++pl) {
        const char *src = static_cast<const char *>(c->f[c->cur]) +
                          ((size_t)pl * c->L.plane + c->L.pitch + c->L.xoff) * c->eb;
        CK(c, cudaMemcpy2DAsync(p, rowb, src, (size_t)c->L.pitch * c->eb, rowb, c->L.ny, cudaMemcpyDeviceToHost, c->st));
        p += rowb * c->L.ny;
    }
    for (int k = 0; k < 2; ++k) {
        CK(c, cudaMemcpy2DAsync(p, (size_t)c->L.nx * sizeof(double), c->ustar + k * c->L.uplane,
                                (size_t)c->L.upitch * sizeof(double), (size_t)c->L.nx * sizeof(double), c->L.ny,
                                cudaMemcpyDeviceToHost, c->st));
        p += N * sizeof(double);
    }
    s = copy_ghosts(c, p, true);
    if (s != LBM_OK) return s;
    *bytes = need;
    return sync_status(c);
}

lbm_status lbm_load(lbm_ctx *c, const void *buf, size_t bytes)
{
    Range range_("lbm_load");
    lbm_status s = check_ready(c);
    if (s != LBM_OK) return s;
    if (!buf || bytes < sizeof(SaveHeader)) return fail(c, LBM_ERR_ARG, "buffer too small");
    SaveHeader h;
    std::memcpy(&h, buf, sizeof h);
    const size_t N = (size_t)c->L.nx * c->L.ny;
    if (std::memcmp(h.magic, "TLVLBM02", 8) != 0 || h.version != 2) return fail(c, LBM_ERR_ARG, "not a checkpoint");
    if (h.nx != c->L.nx || h.ny != c->L.ny || h.storage != c->cfg.storage)
        return fail(c, LBM_ERR_ARG, "checkpoint grid or storage differs from the context");
    if (bytes < sizeof h + 24 * N * c->eb + 2 * N * sizeof(double) + ghost_elems(c) * c->eb)
        return fail(c, LBM_ERR_ARG, "truncated checkpoint");
    CK(c, cudaStreamSynchronize(c->st));
    const char *p = static_cast<const char *>(buf) + sizeof h;
    const size_t rowb = (size_t)c->L.nx * c->eb;
    c->cur = 0;
    for (int pl = 0; pl < 24; ++pl) {
        char *dst = static_cast<char *>(c->f[0]) + ((size_t)pl * c->L.plane + c->L.pitch + c->L.xoff) * c->eb;
        CK(c, cudaMemcpy2DAsync(dst, (size_t)c->L.pitch * c->eb, p, rowb, rowb, c->L.ny, cudaMemcpyHostToDevice, c->st));
        p += rowb * c->L.ny;
    }
    for (int k = 0; k < 2; ++k) {
        CK(c, cudaMemcpy2DAsync(c->ustar + k * c->L.uplane, (size_t)c->L.upitch * sizeof(double), p,
                                (size_t)c->L.nx * sizeof(double), (size_t)c->L.nx * sizeof(double), c->L.ny,
                                cudaMemcpyHostToDevice, c->st));
        p += N * sizeof(double);
    }
    s = copy_ghosts(c, const_cast<char *>(p), false);
    if (s != LBM_OK) return s;
    c->step = h.step;
    c->ghosts_dirty = false;
    CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->st));
    return sync_status(c);
}

lbm_status lbm_info(lbm_ctx *c, int64_t *step, double *t, double *dt)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (step) *step = c->step;
    if (t) *t = c->step * c->dt;
    if (dt) *dt = c->dt;
    return LBM_OK;
}

lbm_status lbm_profile(lbm_ctx *c, int32_t enable)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    CK(c, cudaSetDevice(c->cfg.device));
    CK(c, cudaStreamSynchronize(c->st));
    if (enable) clear_profile(c);
    c->prof = enable != 0;
    return LBM_OK;
}

lbm_status lbm_profile_read(lbm_ctx *c, double out[4])
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (!out) return fail(c, LBM_ERR_ARG, "out is NULL");
    CK(c, cudaSetDevice(c->cfg.device));
    CK(c, cudaStreamSynchronize(c->st));
    const std::vector<cudaEvent_t> *v[2] = {&c->ev_step, &c->ev_edge};
    for (int i = 0; i < 2; ++i) {
        double tot = 0.0;
        for (size_t j = 0; j + 1 < v[i]->size(); j += 2) {
            float ms = 0.f;
            CK(c, cudaEventElapsedTime(&ms, (*v[i])[j], (*v[i])[j + 1]));
            tot += ms;
        }
        out[2 * i] = (double)(v[i]->size() / 2);
        out[2 * i + 1] = tot;
    }
    return LBM_OK;
}

double lbm_bytes_per_node_update(const lbm_ctx *c)
{
    if (!c) return 0.0;
    return 2.0 * 24.0 * c->eb + 4.0 * sizeof(double);
}

} // extern "C"
