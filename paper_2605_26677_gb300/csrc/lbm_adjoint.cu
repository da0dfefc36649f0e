// lbm_adjoint.cu -- the adjoint entry points of include/lbm.h: gradients of a
// sensor-displacement misfit with respect to the per-node shear modulus and
// the initial velocity, by the discrete adjoint of the step with checkpoints.
//
// Forward: init and nsteps steps on the context's own buffers; the state
// f*^n (with its ghost cells) is copied to checkpoint n / K whenever n is a
// multiple of K, and the sensors are read at the recorded steps.
// Backward, segment by segment from the last: the states of the segment are
// recomputed from its checkpoint into K - 1 slots (the step kernel, writing
// u* and status into scratch), then for n = s1 - 1 .. s0 the adjoint kernel
// maps a^{n+1} to a^n (edges included) and, at a recorded step, the loss
// terms are added. Finally the init is transposed.
// K = ceil(sqrt(nsteps)) by default: about 2 sqrt(nsteps) stored states and
// one recomputed forward step per backward step.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace tlv;

struct lbm_adjoint {
    lbm_ctx *c = nullptr;
    long long nsteps = 0;
    int K = 1;
    size_t fbytes = 0;
    std::vector<void *> ck;    // checkpoints f*^{kK}
    std::vector<void *> slot;  // recomputed states of one segment
    // A second slot set and a side stream let the recomputation of segment
    // k - 1 run while the adjoint steps of segment k do; empty when the
    // memory for it was not available (the backward then runs serially).
    std::vector<void *> slot2;
    cudaStream_t side = nullptr;
    cudaEvent_t ready[2] = {nullptr, nullptr};  // slot set s holds its segment
    cudaEvent_t freed[2] = {nullptr, nullptr};  // the adjoint steps reading set s are done
    void *A[2] = {nullptr, nullptr};
    void *tug[2] = {nullptr, nullptr};  // traction-edge cotangent of G, compute type, 4 planes (u* layout)
    void *ubar = nullptr;      // compute type, 2 planes (u* layout)
    double *gmu = nullptr;     // plane (u* layout)
    int *status_scr = nullptr;
    // task order of the FP32 adjoint kernel: 0 static, else dynamic claims
    // over that many counter stripes (two counter sets, alternating)
    int dyn = 0;
    unsigned *d_ctr = nullptr;
    int ctr_par = 0;
    double *U0 = nullptr;      // copy of the initial state (6N)
    double *ghat = nullptr;    // 4N
    int order = 2;
    // loss
    int nsens = 0;
    int *d_sens = nullptr;     // (x, y) pairs
    std::vector<int> rec_steps;
    std::vector<int> rec_at;   // record index of step n, or -1 (nsteps + 1)
    double *d_tgt = nullptr;   // [nrec][nsens][2]
    double *d_rec = nullptr;
    std::vector<double> h_tgt;
    bool forward_done = false;
    long long fwd_step = -1;   // the context's step count after the forward
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    std::string err;
};

static thread_local std::string g_adj_err;

namespace {

// task order of the FP32 adjoint kernel: LBM_ADJ_DYN=0 (static), 1 (dynamic
// claims on one counter, the default) or 4 (over DYN_STRIPES counters) in
// the environment, else dflt
int adj_dyn_choice(int dflt)
{
    const char *v = std::getenv("LBM_ADJ_DYN");
    if (v && !std::strcmp(v, "0")) return 0;
    if (v && !std::strcmp(v, "1")) return 1;
    if (v && !std::strcmp(v, "4")) return DYN_STRIPES;
    return dflt;
}

lbm_status afail(lbm_adjoint *a, lbm_status s, const std::string &msg)
{
    if (a)
        a->err = msg;
    else
        g_adj_err = msg;
    return s;
}

lbm_status acuda(lbm_adjoint *a, cudaError_t e, const char *what)
{
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return afail(a, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, msg);
}

#define AK(a, call)                                                         \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return acuda((a), e_, #call);                \
    } while (0)

bool fp64(const lbm_adjoint *a) { return a->c->cfg.storage == LBM_STORE_F64; }

// the step that maps a^{n+1} (buffers cur) to a^n (buffers cur ^ 1)
template <typename T>
AdjArgs<T> adj_args(const lbm_adjoint *a, const void *fin, int cur)
{
    const lbm_ctx *c = a->c;
    const double w = c->cfg.omega;
    AdjArgs<T> r;
    r.fin = fin;
    r.ain = a->A[cur];
    r.aout = a->A[cur ^ 1];
    r.tug_in = static_cast<const T *>(a->tug[cur]);
    r.tug_out = static_cast<T *>(a->tug[cur ^ 1]);
    for (int e = 0; e < 4; ++e) r.kind[e] = c->edge[e].kind;
    r.mufield = static_cast<const T *>(c->d_muplane);
    r.ubar = static_cast<const T *>(a->ubar);
    r.gmu = a->gmu;
    r.L = c->L;
    T wT;
    relax_pair<T>(w, wT, r.one_m_omega);  // the forward's pair (transposed collision)
    r.wq = T(0.25) * wT;
    r.wi2c = (T)(0.5 * (double)wT / c->cfg.c);
    r.wi2c_d = 0.5 * w / c->cfg.c;
    r.dtT = (T)c->dt;
    r.hdtb1 = (T)(0.5 * c->dt * c->b[0]);
    r.hdtb2 = (T)(0.5 * c->dt * c->b[1]);
    r.lam_ratio = (T)c->m.lam_ratio;
    r.ctr = r.ctr_next = nullptr;
    r.dyn_ns = DYN_STRIPES;
    return r;
}

// sensor displacements of the state in buffer f (u* of the context)
lbm_status record(lbm_adjoint *a, int k, const void *f)
{
    lbm_ctx *c = a->c;
    RecordArgs r;
    r.f = f;
    r.ustar = c->ustar;
    r.sens = a->d_sens;
    r.out = a->d_rec + (size_t)k * a->nsens * 2;
    r.nsens = a->nsens;
    r.L = c->L;
    r.dt = c->dt;
    r.b1 = c->b[0];
    r.b2 = c->b[1];
    AK(a, launch_adj_record(c->cfg.storage, r, c->st));
    return LBM_OK;
}

lbm_status inject(lbm_adjoint *a, void *aout, int k)
{
    lbm_ctx *c = a->c;
    if (fp64(a)) {
        InjectArgs<double> r{aout, static_cast<double *>(a->ubar), a->d_sens, a->d_rec + (size_t)k * a->nsens * 2,
                             a->d_tgt + (size_t)k * a->nsens * 2, a->nsens, c->L, c->dt};
        AK(a, launch_adj_inject(c->cfg.storage, &r, c->st));
    } else {
        InjectArgs<float> r{aout, static_cast<float *>(a->ubar), a->d_sens, a->d_rec + (size_t)k * a->nsens * 2,
                            a->d_tgt + (size_t)k * a->nsens * 2, a->nsens, c->L, c->dt};
        AK(a, launch_adj_inject(c->cfg.storage, &r, c->st));
    }
    return LBM_OK;
}

// one forward step from buffer fin (state n) into fout, without the
// displacement quadrature (the recomputed states need only their
// populations) and with the status word in scratch, on stream st
lbm_status recompute_step(lbm_adjoint *a, const void *fin, void *fout, long long n, cudaStream_t st)
{
    lbm_ctx *c = a->c;
    if (fp64(a)) {
        StepArgs<double> s = ctx_step_args<double>(c, c->cur);
        s.fin = fin;
        s.fout = fout;
        s.ustar = nullptr;
        s.status = a->status_scr;
        s.ctr2 = nullptr;  // static order (the reason is given in the FP32 branch)
        for (int e = 0; e < 4; ++e) s.g[e] = ctx_time_factor(c, e, n);
        AK(a, launch_step(c->cfg.storage, c->m.law, true, &s, c->grid_step, st));
    } else {
        StepArgs<float> s = ctx_step_args<float>(c, c->cur);
        s.fin = fin;
        s.fout = fout;
        s.ustar = nullptr;
        s.status = a->status_scr;
        // static order: beside the adjoint kernel on the other stream, the
        // recomputation in dynamic order slowed the backward pass by 2.5%
        s.ctr2 = nullptr;
        for (int e = 0; e < 4; ++e) s.g[e] = ctx_time_factor(c, e, n);
        AK(a, launch_step(c->cfg.storage, c->m.law, true, &s, c->grid_step, st));
    }
    return LBM_OK;
}

// forward step from buffer fin (state n) into fout with the context's u*
// and status word: the step lbm_step would take, with its output placed
// where the forward pass wants it
lbm_status forward_step(lbm_adjoint *a, const void *fin, void *fout, long long n)
{
    lbm_ctx *c = a->c;
    if (fp64(a)) {
        StepArgs<double> s = ctx_step_args<double>(c, c->cur);
        s.fin = fin;
        s.fout = fout;
        for (int e = 0; e < 4; ++e) s.g[e] = ctx_time_factor(c, e, n);
        AK(a, launch_step(c->cfg.storage, c->m.law, true, &s, c->grid_step, c->st));
    } else {
        StepArgs<float> s = ctx_step_args<float>(c, c->cur);
        s.fin = fin;
        s.fout = fout;
        for (int e = 0; e < 4; ++e) s.g[e] = ctx_time_factor(c, e, n);
        AK(a, launch_step(c->cfg.storage, c->m.law, true, &s, c->grid_step, c->st));
    }
    return LBM_OK;
}

lbm_status adjoint_step(lbm_adjoint *a, const void *fin, int cur, int grid)
{
    lbm_ctx *c = a->c;
    if (fp64(a)) {
        const AdjArgs<double> r = adj_args<double>(a, fin, cur);
        AK(a, launch_adj(c->cfg.storage, c->m.law, &r, grid, c->st));
    } else {
        AdjArgs<float> r = adj_args<float>(a, fin, cur);
        if (a->dyn) {
            // this launch takes the counter set the previous one zeroed
            r.ctr = a->d_ctr + a->ctr_par * DYN_SET_WORDS;
            r.ctr_next = a->d_ctr + (a->ctr_par ^ 1) * DYN_SET_WORDS;
            r.dyn_ns = a->dyn;
            a->ctr_par ^= 1;
        }
        AK(a, launch_adj(c->cfg.storage, c->m.law, &r, grid, c->st));
    }
    return LBM_OK;
}

void free_all(lbm_adjoint *a)
{
    for (void *p : a->ck) cudaFree(p);
    for (void *p : a->slot) cudaFree(p);
    for (void *p : a->slot2) cudaFree(p);
    a->ck.clear();
    a->slot.clear();
    a->slot2.clear();
    for (int i = 0; i < 2; ++i) {
        if (a->ready[i]) cudaEventDestroy(a->ready[i]);
        if (a->freed[i]) cudaEventDestroy(a->freed[i]);
        a->ready[i] = a->freed[i] = nullptr;
    }
    if (a->side) cudaStreamDestroy(a->side);
    a->side = nullptr;
    cudaFree(a->A[0]);
    cudaFree(a->A[1]);
    cudaFree(a->tug[0]);
    cudaFree(a->tug[1]);
    cudaFree(a->ubar);
    cudaFree(a->gmu);
    cudaFree(a->status_scr);
    cudaFree(a->d_ctr);
    cudaFree(a->U0);
    cudaFree(a->ghat);
    cudaFree(a->d_sens);
    cudaFree(a->d_tgt);
    cudaFree(a->d_rec);
    for (cudaEvent_t &e : a->ev)
        if (e) cudaEventDestroy(e);
}

} // namespace

extern "C" {

lbm_status lbm_adjoint_create(lbm_ctx *c, int64_t nsteps, int32_t checkpoint_every, lbm_adjoint **out)
{
    if (!out) return afail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!c) return afail(nullptr, LBM_ERR_ARG, "null context");
    if (nsteps < 0 || nsteps > (1LL << 30)) return afail(nullptr, LBM_ERR_ARG, "nsteps out of range");
    if (checkpoint_every < 0) return afail(nullptr, LBM_ERR_ARG, "checkpoint_every must be >= 0");
    if (!c->m.mufield) return afail(nullptr, LBM_ERR_STATE, "the context needs a material field (lbm_set_material_field)");
    if (c->cfg.storage != LBM_STORE_F64 && c->cfg.storage != LBM_STORE_F32)
        return afail(nullptr, LBM_ERR_UNSUPPORTED, "the adjoint needs FP64 or FP32 storage");
    if (c->cfg.fb_mode != LBM_FB_NODE) return afail(nullptr, LBM_ERR_UNSUPPORTED, "the adjoint needs the node form of F^b");
    lbm_adjoint *a = new (std::nothrow) lbm_adjoint();
    if (!a) return afail(nullptr, LBM_ERR_OOM, "host allocation failed");
    a->c = c;
    a->nsteps = nsteps;
    a->K = checkpoint_every > 0 ? checkpoint_every
                                : std::max(1, (int)std::ceil(std::sqrt((double)std::max<long long>(nsteps, 1))));
    a->fbytes = (size_t)24 * (size_t)c->L.plane * c->eb;
    // dynamic claims on one counter: backward / forward 1.656 at 1024^2
    // against 1.706 in static order and 1.696 over four stripes
    a->dyn = (c->cfg.storage == LBM_STORE_F32) ? adj_dyn_choice(1) : 0;
    a->rec_at.assign((size_t)nsteps + 1, -1);
    const int R = (c->cfg.storage == LBM_STORE_F64) ? 8 : 4;
    const size_t N = (size_t)c->L.nx * c->L.ny;
    const long long nck = nsteps > 0 ? (nsteps - 1) / a->K + 1 : 0;
    lbm_status s = LBM_OK;
    auto alloc = [&](void **p, size_t bytes) {
        if (s != LBM_OK) return;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) s = acuda(a, e, "cudaMalloc");
    };
    cudaError_t e = cudaSetDevice(c->cfg.device);
    if (e != cudaSuccess) s = acuda(a, e, "cudaSetDevice");
    a->ck.assign((size_t)nck, nullptr);
    for (auto &p : a->ck) alloc(&p, a->fbytes);
    a->slot.assign((size_t)std::max(0, a->K - 1), nullptr);
    for (auto &p : a->slot) alloc(&p, a->fbytes);
    alloc(&a->A[0], a->fbytes);
    alloc(&a->A[1], a->fbytes);
    alloc(&a->tug[0], (size_t)4 * c->L.uplane * R);
    alloc(&a->tug[1], (size_t)4 * c->L.uplane * R);
    alloc(&a->ubar, (size_t)2 * c->L.uplane * R);
    alloc((void **)&a->gmu, (size_t)c->L.uplane * sizeof(double));
    alloc((void **)&a->status_scr, sizeof(int));
    alloc((void **)&a->d_ctr, 2 * DYN_SET_WORDS * sizeof(unsigned));
    alloc((void **)&a->U0, 6 * N * sizeof(double));
    alloc((void **)&a->ghat, 4 * N * sizeof(double));
    for (cudaEvent_t &ev : a->ev)
        if (s == LBM_OK && cudaEventCreate(&ev) != cudaSuccess) s = afail(a, LBM_ERR_CUDA, "cudaEventCreate");
    if (s == LBM_OK) {
        e = cudaMemsetAsync(a->status_scr, 0, sizeof(int), c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(a->d_ctr, 0, 2 * DYN_SET_WORDS * sizeof(unsigned), c->st);
        // slots and adjoint buffers: ghosts and padding start defined
        for (void *p : a->slot)
            if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, a->fbytes, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) s = acuda(a, e, "cudaMemsetAsync");
    }
    if (s == LBM_OK && a->slot.size() > 0) {
        // optional: the second slot set, its stream and events; without them
        // the backward runs serially
        bool ok = cudaStreamCreateWithFlags(&a->side, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; i < 2 && ok; ++i)
            ok = cudaEventCreateWithFlags(&a->ready[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&a->freed[i], cudaEventDisableTiming) == cudaSuccess;
        a->slot2.assign(a->slot.size(), nullptr);
        for (auto &p : a->slot2)
            if (ok) ok = cudaMalloc(&p, a->fbytes) == cudaSuccess;
        for (void *p : a->slot2)
            if (ok && p) ok = cudaMemsetAsync(p, 0, a->fbytes, c->st) == cudaSuccess;
        if (ok) ok = cudaStreamSynchronize(c->st) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            for (void *p : a->slot2) cudaFree(p);
            a->slot2.clear();
            for (int i = 0; i < 2; ++i) {
                if (a->ready[i]) cudaEventDestroy(a->ready[i]);
                if (a->freed[i]) cudaEventDestroy(a->freed[i]);
                a->ready[i] = a->freed[i] = nullptr;
            }
            if (a->side) cudaStreamDestroy(a->side);
            a->side = nullptr;
        }
    }
    if (s != LBM_OK) {
        g_adj_err = a->err;
        free_all(a);
        delete a;
        return s;
    }
    *out = a;
    return LBM_OK;
}

void lbm_adjoint_destroy(lbm_adjoint *a)
{
    if (!a) return;
    cudaSetDevice(a->c->cfg.device);
    cudaStreamSynchronize(a->c->st);
    if (a->side) cudaStreamSynchronize(a->side);
    free_all(a);
    delete a;
}

const char *lbm_adjoint_last_error(const lbm_adjoint *a) { return a ? a->err.c_str() : g_adj_err.c_str(); }

lbm_status lbm_adjoint_set_loss(lbm_adjoint *a, int32_t nsens, const int32_t *sens_xy, int32_t nrec,
                                const int32_t *rec_steps, const double *target)
{
    if (!a) return afail(nullptr, LBM_ERR_ARG, "null adjoint");
    lbm_ctx *c = a->c;
    if (nsens < 1 || nrec < 1 || !sens_xy || !rec_steps || !target)
        return afail(a, LBM_ERR_ARG, "need at least one sensor and one record, and non-NULL arrays");
    std::vector<long long> seen;
    for (int s = 0; s < nsens; ++s) {
        const int x = sens_xy[2 * s], y = sens_xy[2 * s + 1];
        if (x < 0 || x >= c->L.nx || y < 0 || y >= c->L.ny) return afail(a, LBM_ERR_ARG, "sensor outside the lattice");
        seen.push_back((long long)y * c->L.nx + x);
    }
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return afail(a, LBM_ERR_ARG, "a sensor node appears twice");
    std::vector<int> at((size_t)a->nsteps + 1, -1);
    for (int k = 0; k < nrec; ++k) {
        if (rec_steps[k] < 0 || rec_steps[k] > a->nsteps) return afail(a, LBM_ERR_ARG, "recorded step outside [0, nsteps]");
        if (at[rec_steps[k]] >= 0) return afail(a, LBM_ERR_ARG, "a step is recorded twice");
        at[rec_steps[k]] = k;
    }
    for (size_t i = 0; i < (size_t)nrec * nsens * 2; ++i)
        if (!std::isfinite(target[i])) return afail(a, LBM_ERR_ARG, "targets must be finite");
    AK(a, cudaSetDevice(c->cfg.device));
    cudaFree(a->d_sens);
    cudaFree(a->d_tgt);
    cudaFree(a->d_rec);
    a->d_sens = nullptr;
    a->d_tgt = a->d_rec = nullptr;
    AK(a, cudaMalloc((void **)&a->d_sens, (size_t)2 * nsens * sizeof(int)));
    AK(a, cudaMalloc((void **)&a->d_tgt, (size_t)nrec * nsens * 2 * sizeof(double)));
    AK(a, cudaMalloc((void **)&a->d_rec, (size_t)nrec * nsens * 2 * sizeof(double)));
    AK(a, cudaMemcpy(a->d_sens, sens_xy, (size_t)2 * nsens * sizeof(int), cudaMemcpyHostToDevice));
    AK(a, cudaMemcpy(a->d_tgt, target, (size_t)nrec * nsens * 2 * sizeof(double), cudaMemcpyHostToDevice));
    a->nsens = nsens;
    a->rec_steps.assign(rec_steps, rec_steps + nrec);
    a->rec_at = at;
    a->h_tgt.assign(target, target + (size_t)nrec * nsens * 2);
    a->forward_done = false;
    return LBM_OK;
}

namespace {

lbm_status forward_body(lbm_adjoint *a, const double *U0_dev, int32_t order, double *loss)
{
    lbm_ctx *c = a->c;
    const size_t N = (size_t)c->L.nx * c->L.ny;
    AK(a, cudaEventRecord(a->ev[0], c->st));
    lbm_status s = lbm_init_device(c, U0_dev, nullptr, order);
    if (s != LBM_OK) return afail(a, s, "init: " + c->err);
    a->order = order;
    AK(a, cudaMemcpyAsync(a->U0, U0_dev, 6 * N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    s = ctx_refresh_ghosts(c);
    if (s != LBM_OK) return afail(a, s, c->err);
    // the forward and the recomputed segments step with the variant the
    // context keeps for its lattice (chosen here if no lbm_step has yet)
    s = ctx_tune_steps(c);
    if (s != LBM_OK) return afail(a, s, c->err);
    const long long n0 = c->step;  // 0 after init
    // Each step writes its state straight into its checkpoint buffer when it
    // is a checkpoint step, else into the context buffer it does not read,
    // so no state is copied except f*^0; the last state lands in a context
    // buffer, which the context then takes as current.
    const void *in = c->f[c->cur];
    if (a->nsteps > 0) AK(a, cudaMemcpyAsync(a->ck[0], in, a->fbytes, cudaMemcpyDeviceToDevice, c->st));
    if (a->rec_at[0] >= 0) {
        s = record(a, a->rec_at[0], in);
        if (s != LBM_OK) return s;
    }
    if (a->nsteps > 0) in = a->ck[0];
    for (long long n = 1; n <= a->nsteps; ++n) {
        void *out = (n < a->nsteps && n % a->K == 0) ? a->ck[(size_t)(n / a->K)]
                                                    : (in == c->f[0] ? c->f[1] : c->f[0]);
        s = forward_step(a, in, out, n0 + n - 1);
        if (s != LBM_OK) return s;
        in = out;
        if (a->rec_at[(size_t)n] >= 0) {
            s = record(a, a->rec_at[(size_t)n], in);
            if (s != LBM_OK) return s;
        }
    }
    if (a->nsteps > 0) {
        c->cur = (in == c->f[1]) ? 1 : 0;
        c->step = n0 + a->nsteps;
    }
    AK(a, cudaEventRecord(a->ev[1], c->st));
    s = lbm_sync(c);
    if (s != LBM_OK) return afail(a, s, c->err);
    const size_t nr = a->rec_steps.size() * a->nsens * 2;
    std::vector<double> rec(nr);
    AK(a, cudaMemcpy(rec.data(), a->d_rec, nr * sizeof(double), cudaMemcpyDeviceToHost));
    double L = 0.0;
    for (size_t i = 0; i < nr; ++i) {
        const double r = rec[i] - a->h_tgt[i];
        L += 0.5 * r * r;
    }
    *loss = L;
    a->forward_done = true;
    a->fwd_step = n0 + a->nsteps;
    return LBM_OK;
}

} // namespace

lbm_status lbm_adjoint_forward(lbm_adjoint *a, const double *U0_dev, int32_t order, double *loss)
{
    Range range_("lbm_adjoint_forward");
    if (!a) return afail(nullptr, LBM_ERR_ARG, "null adjoint");
    if (!loss) return afail(a, LBM_ERR_ARG, "loss is NULL");
    if (a->nsens < 1) return afail(a, LBM_ERR_STATE, "lbm_adjoint_set_loss must come first");
    lbm_ctx *c = a->c;
    if (!c->m.mufield) return afail(a, LBM_ERR_STATE, "the context lost its material field");
    AK(a, cudaSetDevice(c->cfg.device));
    a->forward_done = false;
    lbm_status s = forward_body(a, U0_dev, order, loss);
    // a failure part way leaves the context's buffers holding a partial run
    // that its time level no longer describes: it needs a new lbm_init
    if (s != LBM_OK) c->initialized = false;
    return s;
}

namespace {

lbm_status backward_body(lbm_adjoint *a, double *g_mu_dev, double *g_v0_dev)
{
    lbm_ctx *c = a->c;
    const int R = fp64(a) ? 8 : 4;
    AK(a, cudaEventRecord(a->ev[2], c->st));
    AK(a, cudaMemsetAsync(a->A[0], 0, a->fbytes, c->st));
    AK(a, cudaMemsetAsync(a->A[1], 0, a->fbytes, c->st));
    AK(a, cudaMemsetAsync(a->tug[0], 0, (size_t)4 * c->L.uplane * R, c->st));
    AK(a, cudaMemsetAsync(a->tug[1], 0, (size_t)4 * c->L.uplane * R, c->st));
    AK(a, cudaMemsetAsync(a->ubar, 0, (size_t)2 * c->L.uplane * R, c->st));
    AK(a, cudaMemsetAsync(a->gmu, 0, (size_t)c->L.uplane * sizeof(double), c->st));
    int cur = 0;
    lbm_status s = LBM_OK;
    if (a->rec_at[(size_t)a->nsteps] >= 0) s = inject(a, a->A[cur], a->rec_at[(size_t)a->nsteps]);
    if (s != LBM_OK) return s;
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->cfg.device);
    const int per_sm = std::max(1, adj_blocks_per_sm(c->cfg.storage, c->m.law));
    const int vec = adj_vec_for(c->cfg.storage);
    const long long tasks = (long long)c->L.ny * ((c->L.nx + 32 * vec - 1) / (32 * vec));
    const int grid = (int)std::max(1LL, std::min((tasks + 3) / 4, (long long)sms * per_sm));
    const long long nck = (long long)a->ck.size();
    const bool pipe = !a->slot2.empty();
    // slot set of segment k: with the second set, segments alternate between
    // them, so that segment k - 1 is recomputed on the side stream while the
    // adjoint steps of segment k run on the context's stream
    auto slots = [&](long long k) -> std::vector<void *> & { return (pipe && (k & 1)) ? a->slot2 : a->slot; };
    auto recompute = [&](long long k, cudaStream_t st) -> lbm_status {
        const long long s0 = k * a->K, s1 = std::min(s0 + a->K, a->nsteps);
        std::vector<void *> &sl = slots(k);
        for (long long n = s0 + 1; n < s1; ++n) {
            const void *fin = n - 1 == s0 ? a->ck[(size_t)k] : sl[(size_t)(n - 1 - s0 - 1)];
            lbm_status r = recompute_step(a, fin, sl[(size_t)(n - s0 - 1)], n - 1, st);
            if (r != LBM_OK) return r;
        }
        return LBM_OK;
    };
    if (pipe && nck > 0) {
        // the side stream starts after everything queued so far; both slot
        // sets start free
        AK(a, cudaEventRecord(a->freed[0], c->st));
        AK(a, cudaEventRecord(a->freed[1], c->st));
        AK(a, cudaStreamWaitEvent(a->side, a->freed[0], 0));
        s = recompute(nck - 1, a->side);
        if (s != LBM_OK) return s;
        AK(a, cudaEventRecord(a->ready[(nck - 1) & 1], a->side));
    }
    for (long long k = nck - 1; k >= 0; --k) {
        const long long s0 = k * a->K, s1 = std::min(s0 + a->K, a->nsteps);
        if (pipe) {
            AK(a, cudaStreamWaitEvent(c->st, a->ready[k & 1], 0));
            if (k > 0) {
                // segment k - 1 into the other set once the steps that read it are done
                AK(a, cudaStreamWaitEvent(a->side, a->freed[(k - 1) & 1], 0));
                s = recompute(k - 1, a->side);
                if (s != LBM_OK) return s;
                AK(a, cudaEventRecord(a->ready[(k - 1) & 1], a->side));
            }
        } else {
            s = recompute(k, c->st);
            if (s != LBM_OK) return s;
        }
        std::vector<void *> &sl = slots(k);
        auto state = [&](long long n) -> const void * { return n == s0 ? a->ck[(size_t)k] : sl[(size_t)(n - s0 - 1)]; };
        for (long long n = s1 - 1; n >= s0; --n) {
            s = adjoint_step(a, state(n), cur, grid);
            if (s != LBM_OK) return s;
            cur ^= 1;
            if (a->rec_at[(size_t)n] >= 0) {
                s = inject(a, a->A[cur], a->rec_at[(size_t)n]);
                if (s != LBM_OK) return s;
            }
        }
        if (pipe) AK(a, cudaEventRecord(a->freed[k & 1], c->st));
    }
    // the init (its u* and its collision included)
    AdjInitArgs ai;
    std::memset(&ai, 0, sizeof ai);
    ai.ia.U0 = a->U0;
    ai.ia.u0 = nullptr;
    ai.ia.fout = nullptr;
    ai.ia.ustar = nullptr;
    ai.ia.status = nullptr;
    ai.ia.L = c->L;
    ai.ia.m = c->m;
    ai.ia.c = c->cfg.c;
    ai.ia.dt = c->dt;
    ai.ia.dx = c->cfg.dx;
    ai.ia.omega = c->cfg.omega;
    ai.ia.b1 = c->b[0];
    ai.ia.b2 = c->b[1];
    ai.ia.order = a->order;
    ai.ia.xper = c->edge[LBM_EDGE_LEFT].kind == LBM_BC_PERIODIC;
    ai.ia.yper = c->edge[LBM_EDGE_BOTTOM].kind == LBM_BC_PERIODIC;
    ai.ia.y0 = 0;
    ai.ia.y1 = c->L.ny;
    ai.a0 = a->A[cur];
    ai.ubar = a->ubar;
    ai.gmu = a->gmu;
    ai.gv0 = g_v0_dev;
    ai.ghat = a->ghat;
    ai.tug = a->tug[cur];
    for (int e = 0; e < 4; ++e) ai.kind[e] = c->edge[e].kind;
    AK(a, launch_adj_init(c->cfg.storage, ai, c->st));
    AK(a, launch_plane_to_compact(a->gmu, g_mu_dev, c->L, c->st));
    AK(a, cudaEventRecord(a->ev[3], c->st));
    AK(a, cudaStreamSynchronize(c->st));
    return LBM_OK;
}

} // namespace

lbm_status lbm_adjoint_backward(lbm_adjoint *a, double *g_mu_dev, double *g_v0_dev)
{
    Range range_("lbm_adjoint_backward");
    if (!a) return afail(nullptr, LBM_ERR_ARG, "null adjoint");
    if (!g_mu_dev || !g_v0_dev) return afail(a, LBM_ERR_ARG, "output pointers must be non-NULL");
    lbm_ctx *c = a->c;
    if (!a->forward_done || c->step != a->fwd_step)
        return afail(a, LBM_ERR_STATE, "lbm_adjoint_forward must precede, with no other step of the context between");
    AK(a, cudaSetDevice(c->cfg.device));
    lbm_status s = backward_body(a, g_mu_dev, g_v0_dev);
    if (s != LBM_OK && !a->slot2.empty()) {
        // recomputation may still be queued on the side stream, reading the
        // checkpoints: order the context's stream after it, so that work
        // enqueued next on the context (a forward rewriting the checkpoints)
        // cannot overtake it
        if (cudaEventRecord(a->freed[0], a->side) == cudaSuccess) cudaStreamWaitEvent(c->st, a->freed[0], 0);
        cudaGetLastError();
    }
    return s;
}

lbm_status lbm_adjoint_info(const lbm_adjoint *a, int32_t *checkpoint_every, int64_t *stored_states,
                            double *forward_ms, double *backward_ms)
{
    if (!a) return afail(nullptr, LBM_ERR_ARG, "null adjoint");
    if (checkpoint_every) *checkpoint_every = a->K;
    if (stored_states) *stored_states = (int64_t)(a->ck.size() + a->slot.size());
    float f = 0.f, b = 0.f;
    if (forward_ms) {
        *forward_ms = 0.0;
        if (a->forward_done && cudaEventElapsedTime(&f, a->ev[0], a->ev[1]) == cudaSuccess) *forward_ms = f;
    }
    if (backward_ms) {
        *backward_ms = 0.0;
        if (cudaEventQuery(a->ev[3]) == cudaSuccess && cudaEventElapsedTime(&b, a->ev[2], a->ev[3]) == cudaSuccess)
            *backward_ms = b;
        cudaGetLastError();
    }
    return LBM_OK;
}

} // extern "C"
