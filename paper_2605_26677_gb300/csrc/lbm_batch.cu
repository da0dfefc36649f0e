// lbm_batch.cu -- the batch entry points of include/lbm.h: many lattices
// advanced by shared persistent launches, optionally replayed from a CUDA
// graph, with a per-size-class tile chosen by default or by measurement.
//
// Per step the batch enqueues (on its own stream, groups forked onto side
// streams so that they overlap):
//   [k_batch_time]            edge time factors of the step, if any member
//                             has a time-dependent edge
//   k_batch / k_batch16 x G   one launch per group (closure, tile, task order)
// Two StepArgs arrays live in device memory, one per step parity: parity 0
// reads each member's current buffer, parity 1 the other one, so a captured
// graph of an even number of steps is valid for every call, and each call
// only rewrites the arrays' contents (same addresses) before replaying it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace tlv;

namespace {

constexpr int NCLASS = LBM_BATCH_CLASSES;
constexpr int CLASS_MAX_NX[NCLASS - 1] = {48, 96, 192, 384};
constexpr int TIME_CHUNK = 1024;  // steps of edge time factors per upload
constexpr int MAX_GROUPS = 64;    // (closure, tile, order) groups; 6 x 3 x 2 exist
// per group: DYN_STRIPES claim counters and a finished-blocks counter
constexpr int GROUP_CTR_WORDS = (DYN_STRIPES + 1) * DYN_CTR_STRIDE;

int size_class(int nx)
{
    for (int k = 0; k < NCLASS - 1; ++k)
        if (nx <= CLASS_MAX_NX[k]) return k;
    return NCLASS - 1;
}

// tiles built per storage, narrowest first
std::vector<int> tiles_for(int storage)
{
    if (storage == STORE_F64) return {1, 2};
    if (storage == STORE_F32) return {1, 2, 4};
    return {2, 4};
}

int default_tile(int storage, int cls)
{
    const std::vector<int> t = tiles_for(storage);
    const int maxnx = cls < NCLASS - 1 ? CLASS_MAX_NX[cls] : 1 << 30;
    int best = t.front();
    for (int v : t)
        if (32 * v <= maxnx) best = v;
    return best;
}

const void *kernel_for(int storage, int law, int vec)
{
    switch (storage) {
    case STORE_F64: return batch_kernel_f64(law, vec);
    case STORE_F32: return batch_kernel_f32(law, vec);
    case STORE_BF16: return batch_kernel_bf16(law, vec);
    default: return batch_kernel_f16(law, vec);
    }
}

struct Group {
    int law = 0, vec = 0;
    bool dyn = false;          // dynamic task order
    int first = 0, count = 0;  // range of plan.order
    int ntask = 0, grid = 0;
    const void *fn = nullptr;
    bool operator==(const Group &o) const
    {
        return law == o.law && vec == o.vec && dyn == o.dyn && first == o.first && count == o.count && ntask == o.ntask &&
               grid == o.grid && fn == o.fn;
    }
};

struct Plan {
    std::vector<int> order;  // member indices grouped by (law, vec)
    std::vector<Group> groups;
    bool timed = false;      // some edge has a time-dependent factor
    bool operator==(const Plan &o) const { return order == o.order && groups == o.groups && timed == o.timed; }
};

__global__ void k_batch_time(BatchTime t)
{
    __shared__ int k;
    if (threadIdx.x == 0) k = min(max(*t.k, 0), t.rows - 1);  // the host keeps k < rows
    __syncthreads();
    const double *row = t.tab + (size_t)k * t.n4;
    for (int i = threadIdx.x; i < t.n4; i += blockDim.x) t.g[i] = row[i];
    if (threadIdx.x == 0) *t.k = k + 1;
}

template <typename T>
__global__ void k_batch_status(const StepArgs<T> *args, int n, int *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = *args[i].status;
}

} // namespace

struct lbm_batch {
    std::vector<lbm_ctx *> m;
    int n = 0, device = 0, storage = 0;
    size_t argsz = 0;  // sizeof(StepArgs<R>)
    int vec[NCLASS] = {};
    int dyn[NCLASS] = {};  // task order per size class (0 static, 1 dynamic)
    int sms = 1;
    cudaStream_t st = nullptr;
    std::vector<cudaStream_t> side;  // one per group beyond the first
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr, ev_upload = nullptr;
    std::vector<cudaEvent_t> ev_join;
    // device
    char *d_args = nullptr;  // [2][n] StepArgs, plan order
    int *d_off = nullptr;    // per group count + 1 prefix sums
    double *d_g = nullptr;   // [4n]
    int *d_k = nullptr;
    double *d_tab = nullptr; // [TIME_CHUNK][4n]
    int *d_stat = nullptr;   // [n]
    unsigned *d_ctr = nullptr; // [MAX_GROUPS][GROUP_CTR_WORDS] task counters of dynamic groups
    // pinned host staging
    char *h_args = nullptr;
    double *h_tab = nullptr;
    int *h_stat = nullptr;
    int *h_off = nullptr;
    Plan plan;
    bool have_plan = false;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    int graphs = 0;
    std::string err;
};

static thread_local std::string g_batch_err;

namespace {

lbm_status bfail(lbm_batch *b, lbm_status s, const std::string &msg)
{
    if (b)
        b->err = msg;
    else
        g_batch_err = msg;
    return s;
}

lbm_status bcuda(lbm_batch *b, cudaError_t e, const char *what)
{
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return bfail(b, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, msg);
}

#define BK(b, call)                                                         \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return bcuda((b), e_, #call);                \
    } while (0)

int ntask_of(const lbm_ctx *c, int vec) { return c->L.ny * ((c->L.nx + 32 * vec - 1) / (32 * vec)); }

bool any_timed(const lbm_batch *b)
{
    for (const lbm_ctx *c : b->m)
        for (int e = 0; e < 4; ++e)
            if (c->edge[e].kind != BC_PERIODIC && c->edge[e].timefn != TF_CONST) return true;
    return false;
}

// Groups of (law, tile, task order) in a fixed order; grid = enough 4-warp
// blocks for every task, at most the resident blocks of the whole GPU
// (persistent).
lbm_status make_plan(lbm_batch *b, Plan &p)
{
    p = Plan();
    p.timed = any_timed(b);
    std::vector<std::pair<long long, int>> key(b->n);
    for (int i = 0; i < b->n; ++i) {
        const lbm_ctx *c = b->m[i];
        const int k = size_class(c->L.nx);
        key[i] = {(long long)c->m.law * 32 + b->vec[k] * 2 + b->dyn[k], i};
    }
    std::stable_sort(key.begin(), key.end(),
                     [](const std::pair<long long, int> &x, const std::pair<long long, int> &y) { return x.first < y.first; });
    for (int i = 0; i < b->n; ++i) {
        const int mi = key[i].second;
        const lbm_ctx *c = b->m[mi];
        const int k = size_class(c->L.nx);
        const int law = c->m.law, v = b->vec[k];
        const bool dyn = b->dyn[k] != 0;
        if (p.groups.empty() || p.groups.back().law != law || p.groups.back().vec != v ||
            p.groups.back().dyn != dyn) {
            if ((int)p.groups.size() == MAX_GROUPS) return bfail(b, LBM_ERR_ARG, "too many groups");
            Group g;
            g.law = law;
            g.vec = v;
            g.dyn = dyn;
            g.first = i;
            g.fn = kernel_for(b->storage, law, v);
            if (!g.fn) return bfail(b, LBM_ERR_UNSUPPORTED, "no batched kernel for this closure and tile");
            p.groups.push_back(g);
        }
        Group &g = p.groups.back();
        const long long nt = (long long)g.ntask + ntask_of(c, v);
        if (nt >= (1LL << 31)) return bfail(b, LBM_ERR_ARG, "a group of the batch has 2^31 or more tasks");
        g.ntask = (int)nt;
        g.count += 1;
        p.order.push_back(mi);
    }
    for (Group &g : p.groups) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, g.fn, 128, (g.count + 1) * sizeof(int)) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        const long long want = (g.ntask + 3) / 4;
        g.grid = (int)std::max(1LL, std::min(want, (long long)per_sm * b->sms));
    }
    return LBM_OK;
}

// trial launches of the tuner write u* and status into scratch (ustar_scratch
// non-null); otherwise the members' own buffers are used
template <typename T>
void fill_args(lbm_batch *b, const Plan &p, double *ustar_scratch, int *status_scratch)
{
    StepArgs<T> *arr = reinterpret_cast<StepArgs<T> *>(b->h_args);
    size_t uoff = 0;
    for (int i = 0; i < b->n; ++i) {
        lbm_ctx *c = b->m[p.order[i]];
        for (int par = 0; par < 2; ++par) {
            StepArgs<T> a = ctx_step_args<T>(c, c->cur ^ par);
            a.gdev = p.timed ? b->d_g + 4 * i : nullptr;
            if (ustar_scratch) {
                a.ustar = ustar_scratch + uoff;
                a.status = status_scratch;
            }
            arr[par * b->n + i] = a;
        }
        if (ustar_scratch) uoff += (size_t)2 * c->L.uplane;
    }
}

lbm_status upload_plan(lbm_batch *b, const Plan &p, double *ustar_scratch, int *status_scratch)
{
    BK(b, cudaEventSynchronize(b->ev_upload));  // the staging buffers are free again
    if (b->storage == STORE_F64)
        fill_args<double>(b, p, ustar_scratch, status_scratch);
    else
        fill_args<float>(b, p, ustar_scratch, status_scratch);
    int w = 0;
    for (const Group &g : p.groups) {
        int acc = 0;
        b->h_off[w++] = 0;
        for (int i = 0; i < g.count; ++i) {
            acc += ntask_of(b->m[p.order[g.first + i]], g.vec);
            b->h_off[w++] = acc;
        }
    }
    BK(b, cudaMemcpyAsync(b->d_args, b->h_args, 2 * (size_t)b->n * b->argsz, cudaMemcpyHostToDevice, b->st));
    BK(b, cudaMemcpyAsync(b->d_off, b->h_off, (size_t)w * sizeof(int), cudaMemcpyHostToDevice, b->st));
    BK(b, cudaEventRecord(b->ev_upload, b->st));
    return LBM_OK;
}

lbm_status launch_group(lbm_batch *b, const Plan &p, int gi, int parity, cudaStream_t s)
{
    const Group &g = p.groups[gi];
    BatchList bl;
    bl.args = b->d_args + ((size_t)parity * b->n + g.first) * b->argsz;
    bl.off = b->d_off + g.first + gi;
    bl.ctr = g.dyn ? b->d_ctr + (size_t)gi * GROUP_CTR_WORDS : nullptr;
    bl.n = g.count;
    void *params[] = {&bl};
    BK(b, cudaLaunchKernel(g.fn, dim3(g.grid), dim3(128), params, (g.count + 1) * sizeof(int), s));
    return LBM_OK;
}

lbm_status enqueue_step(lbm_batch *b, const Plan &p, int parity)
{
    if (p.timed) {
        BatchTime t{b->d_tab, b->d_k, b->d_g, 4 * b->n, TIME_CHUNK};
        k_batch_time<<<1, 256, 0, b->st>>>(t);
        BK(b, cudaGetLastError());
    }
    const int G = (int)p.groups.size();
    if (G > 1) BK(b, cudaEventRecord(b->ev_fork, b->st));
    for (int gi = 1; gi < G; ++gi) {
        BK(b, cudaStreamWaitEvent(b->side[gi - 1], b->ev_fork, 0));
        lbm_status s = launch_group(b, p, gi, parity, b->side[gi - 1]);
        if (s != LBM_OK) return s;
        BK(b, cudaEventRecord(b->ev_join[gi - 1], b->side[gi - 1]));
    }
    if (G > 0) {
        lbm_status s = launch_group(b, p, 0, parity, b->st);
        if (s != LBM_OK) return s;
    }
    for (int gi = 1; gi < G; ++gi) BK(b, cudaStreamWaitEvent(b->st, b->ev_join[gi - 1], 0));
    return LBM_OK;
}

lbm_status ensure_side_streams(lbm_batch *b, int groups)
{
    while ((int)b->side.size() < groups - 1) {
        cudaStream_t s;
        cudaEvent_t e;
        BK(b, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        b->side.push_back(s);
        BK(b, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->ev_join.push_back(e);
    }
    return LBM_OK;
}

void drop_graph(lbm_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_steps = 0;
}

lbm_status capture(lbm_batch *b, const Plan &p, int steps)
{
    drop_graph(b);
    BK(b, cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    lbm_status s = LBM_OK;
    for (int i = 0; i < steps && s == LBM_OK; ++i) s = enqueue_step(b, p, i & 1);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->st, &g);
    if (s != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return bcuda(b, e, "cudaGraphInstantiate");
    }
    b->graph_steps = steps;
    b->graphs += 1;
    return LBM_OK;
}

// make the batch stream wait for every member stream (or the reverse)
lbm_status join_streams(lbm_batch *b, bool members_to_batch)
{
    std::vector<cudaStream_t> seen;
    for (lbm_ctx *c : b->m) {
        if (std::find(seen.begin(), seen.end(), c->st) != seen.end()) continue;
        seen.push_back(c->st);
        if (members_to_batch) {
            BK(b, cudaEventRecord(b->ev_in, c->st));
            BK(b, cudaStreamWaitEvent(b->st, b->ev_in, 0));
        } else {
            BK(b, cudaStreamWaitEvent(c->st, b->ev_out, 0));
        }
    }
    return LBM_OK;
}

lbm_status members_ready(lbm_batch *b)
{
    for (lbm_ctx *c : b->m) {
        lbm_status s = ctx_ready(c);
        if (s != LBM_OK) return bfail(b, s, "member not ready: " + c->err);
        if (c->m.mufield) return bfail(b, LBM_ERR_ARG, "batches take members with uniform material");
        if (c->ghosts_dirty) {
            s = ctx_refresh_ghosts(c);
            if (s != LBM_OK) return bfail(b, s, "member ghost refresh: " + c->err);
        }
    }
    return LBM_OK;
}

// the plan for the current tiles and members; a new plan drops the graph
lbm_status current_plan(lbm_batch *b)
{
    Plan p;
    lbm_status s = make_plan(b, p);
    if (s != LBM_OK) return s;
    if (!b->have_plan || !(p == b->plan)) {
        drop_graph(b);
        b->plan = p;
        b->have_plan = true;
        s = ensure_side_streams(b, (int)p.groups.size());
        if (s != LBM_OK) return s;
    }
    return LBM_OK;
}

// edge time factors of steps [s0, s0 + len) of this call into row 0.. of the table
lbm_status upload_times(lbm_batch *b, long long s0, int len)
{
    BK(b, cudaEventSynchronize(b->ev_upload));  // the staging buffer is free again
    const Plan &p = b->plan;
    for (int k = 0; k < len; ++k)
        for (int i = 0; i < b->n; ++i) {
            const lbm_ctx *c = b->m[p.order[i]];
            for (int e = 0; e < 4; ++e)
                b->h_tab[((size_t)k * b->n + i) * 4 + e] = ctx_time_factor(c, e, c->step + s0 + k);
        }
    BK(b, cudaMemcpyAsync(b->d_tab, b->h_tab, (size_t)len * 4 * b->n * sizeof(double), cudaMemcpyHostToDevice,
                          b->st));
    BK(b, cudaMemsetAsync(b->d_k, 0, sizeof(int), b->st));
    BK(b, cudaEventRecord(b->ev_upload, b->st));
    return LBM_OK;
}

lbm_status run_steps(lbm_batch *b, int64_t nsteps, int graph_steps)
{
    const Plan &p = b->plan;
    if (graph_steps > 0 && b->graph_steps != graph_steps) {
        lbm_status s = capture(b, p, graph_steps);
        if (s != LBM_OK) return s;
    }
    // chunks of whole graphs; each chunk refreshes the time table if needed
    const int64_t chunk = p.timed ? (graph_steps > 0 ? std::max<int64_t>(graph_steps, TIME_CHUNK / graph_steps * graph_steps)
                                                     : TIME_CHUNK)
                                  : nsteps;
    for (int64_t s0 = 0; s0 < nsteps; s0 += chunk) {
        const int64_t len = std::min<int64_t>(chunk, nsteps - s0);
        if (p.timed) {
            lbm_status s = upload_times(b, s0, (int)len);
            if (s != LBM_OK) return s;
        }
        int64_t done = 0;
        if (graph_steps > 0)
            for (; done + graph_steps <= len; done += graph_steps) BK(b, cudaGraphLaunch(b->graph, b->st));
        for (; done < len; ++done) {
            lbm_status s = enqueue_step(b, p, (int)((s0 + done) & 1));
            if (s != LBM_OK) return s;
        }
    }
    return LBM_OK;
}

lbm_status alloc_batch(lbm_batch *b)
{
    const size_t n = b->n;
    BK(b, cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking));
    BK(b, cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    BK(b, cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    BK(b, cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    BK(b, cudaEventCreateWithFlags(&b->ev_upload, cudaEventDisableTiming));
    BK(b, cudaEventRecord(b->ev_upload, b->st));
    BK(b, cudaMalloc((void **)&b->d_args, 2 * n * b->argsz));
    BK(b, cudaMalloc((void **)&b->d_off, (2 * n + 1) * sizeof(int)));
    BK(b, cudaMalloc((void **)&b->d_g, 4 * n * sizeof(double)));
    BK(b, cudaMalloc((void **)&b->d_k, sizeof(int)));
    BK(b, cudaMalloc((void **)&b->d_tab, (size_t)TIME_CHUNK * 4 * n * sizeof(double)));
    BK(b, cudaMalloc((void **)&b->d_stat, n * sizeof(int)));
    BK(b, cudaMalloc((void **)&b->d_ctr, (size_t)MAX_GROUPS * GROUP_CTR_WORDS * sizeof(unsigned)));
    BK(b, cudaMallocHost((void **)&b->h_args, 2 * n * b->argsz));
    BK(b, cudaMallocHost((void **)&b->h_tab, (size_t)TIME_CHUNK * 4 * n * sizeof(double)));
    BK(b, cudaMallocHost((void **)&b->h_stat, n * sizeof(int)));
    BK(b, cudaMallocHost((void **)&b->h_off, (2 * n + 1) * sizeof(int)));
    BK(b, cudaMemsetAsync(b->d_g, 0, 4 * n * sizeof(double), b->st));
    BK(b, cudaMemsetAsync(b->d_k, 0, sizeof(int), b->st));
    BK(b, cudaMemsetAsync(b->d_ctr, 0, (size_t)MAX_GROUPS * GROUP_CTR_WORDS * sizeof(unsigned), b->st));
    BK(b, cudaStreamSynchronize(b->st));
    return LBM_OK;
}

// per-member flags -> statuses; returns the first failure
lbm_status gather_status(lbm_batch *b, int32_t *member_status)
{
    const Plan &p = b->plan;
    const int n = b->n;
    if (b->storage == STORE_F64)
        k_batch_status<double><<<(n + 127) / 128, 128, 0, b->st>>>(reinterpret_cast<const StepArgs<double> *>(b->d_args), n, b->d_stat);
    else
        k_batch_status<float><<<(n + 127) / 128, 128, 0, b->st>>>(reinterpret_cast<const StepArgs<float> *>(b->d_args), n, b->d_stat);
    BK(b, cudaGetLastError());
    BK(b, cudaMemcpyAsync(b->h_stat, b->d_stat, n * sizeof(int), cudaMemcpyDeviceToHost, b->st));
    BK(b, cudaStreamSynchronize(b->st));
    lbm_status first = LBM_OK;
    for (int i = 0; i < n; ++i) {
        const int mi = p.order[i];
        const lbm_status s = ctx_map_flags(b->m[mi], b->h_stat[i]);
        if (member_status) member_status[mi] = s;
        if (s != LBM_OK && first == LBM_OK) {
            first = s;
            bfail(b, s, "member " + std::to_string(mi) + ": " + b->m[mi]->err);
        }
    }
    return first;
}

} // namespace

extern "C" {

lbm_status lbm_batch_create(lbm_ctx *const *members, int32_t n, lbm_batch **out)
{
    if (!out) return bfail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!members) return bfail(nullptr, LBM_ERR_ARG, "members is NULL");
    if (n < 1 || n > LBM_BATCH_MAX_MEMBERS) return bfail(nullptr, LBM_ERR_ARG, "n must be in [1, 4096]");
    for (int i = 0; i < n; ++i) {
        const lbm_ctx *c = members[i];
        if (!c) return bfail(nullptr, LBM_ERR_ARG, "a member is NULL");
        for (int j = 0; j < i; ++j)
            if (members[j] == c) return bfail(nullptr, LBM_ERR_ARG, "a context appears twice");
        if (c->cfg.device != members[0]->cfg.device) return bfail(nullptr, LBM_ERR_ARG, "members on different devices");
        if (c->cfg.storage != members[0]->cfg.storage)
            return bfail(nullptr, LBM_ERR_ARG, "members with different storage types");
        if (c->cfg.fb_mode != LBM_FB_NODE) return bfail(nullptr, LBM_ERR_ARG, "batches take members in the node form of F^b");
        if (c->m.mufield) return bfail(nullptr, LBM_ERR_ARG, "batches take members with uniform material");
    }
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(nullptr, LBM_ERR_OOM, "host allocation failed");
    b->m.assign(members, members + n);
    b->n = n;
    b->device = members[0]->cfg.device;
    b->storage = members[0]->cfg.storage;
    b->argsz = b->storage == STORE_F64 ? sizeof(StepArgs<double>) : sizeof(StepArgs<float>);
    for (int k = 0; k < NCLASS; ++k) b->vec[k] = default_tile(b->storage, k);
    cudaError_t e = cudaSetDevice(b->device);
    if (e == cudaSuccess) cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (b->sms < 1) b->sms = 1;
    lbm_status s = e != cudaSuccess ? bcuda(b, e, "cudaSetDevice") : alloc_batch(b);
    if (s != LBM_OK) {
        g_batch_err = b->err;
        lbm_batch_destroy(b);
        return s;
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->st) cudaStreamSynchronize(b->st);
    drop_graph(b);
    for (cudaStream_t s : b->side) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
    for (cudaEvent_t e : {b->ev_in, b->ev_out, b->ev_fork, b->ev_upload})
        if (e) cudaEventDestroy(e);
    cudaFree(b->d_args);
    cudaFree(b->d_off);
    cudaFree(b->d_g);
    cudaFree(b->d_k);
    cudaFree(b->d_tab);
    cudaFree(b->d_stat);
    cudaFree(b->d_ctr);
    cudaFreeHost(b->h_args);
    cudaFreeHost(b->h_tab);
    cudaFreeHost(b->h_stat);
    cudaFreeHost(b->h_off);
    if (b->st) cudaStreamDestroy(b->st);
    delete b;
}

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

int32_t lbm_batch_size_class(int32_t nx) { return size_class(nx); }

lbm_status lbm_batch_get_tiles(const lbm_batch *b, int32_t *vec)
{
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "null batch");
    if (!vec) return bfail(const_cast<lbm_batch *>(b), LBM_ERR_ARG, "vec is NULL");
    for (int k = 0; k < NCLASS; ++k) vec[k] = b->vec[k];
    return LBM_OK;
}

lbm_status lbm_batch_set_tile(lbm_batch *b, int32_t size_class, int32_t vec)
{
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "null batch");
    if (size_class < 0 || size_class >= NCLASS) return bfail(b, LBM_ERR_ARG, "size class out of range");
    const std::vector<int> t = tiles_for(b->storage);
    if (std::find(t.begin(), t.end(), vec) == t.end()) return bfail(b, LBM_ERR_ARG, "no such tile for this storage");
    b->vec[size_class] = vec;
    return LBM_OK;
}

lbm_status lbm_batch_get_task_orders(const lbm_batch *b, int32_t *dynamic)
{
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "null batch");
    if (!dynamic) return bfail(const_cast<lbm_batch *>(b), LBM_ERR_ARG, "dynamic is NULL");
    for (int k = 0; k < NCLASS; ++k) dynamic[k] = b->dyn[k];
    return LBM_OK;
}

lbm_status lbm_batch_set_task_order(lbm_batch *b, int32_t size_class, int32_t dynamic)
{
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "null batch");
    if (size_class < 0 || size_class >= NCLASS) return bfail(b, LBM_ERR_ARG, "size class out of range");
    if (dynamic != 0 && dynamic != 1) return bfail(b, LBM_ERR_ARG, "dynamic must be 0 or 1");
    b->dyn[size_class] = dynamic;
    return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch *b, int32_t reps, double *us)
{
    Range range_("lbm_batch_tune");
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "null batch");
    if (reps < 1) return bfail(b, LBM_ERR_ARG, "reps must be >= 1");
    BK(b, cudaSetDevice(b->device));
    lbm_status s = members_ready(b);
    if (s != LBM_OK) return s;
    s = join_streams(b, true);
    if (s != LBM_OK) return s;
    if (us)
        for (int i = 0; i < NCLASS * 3; ++i) us[i] = 0.0;
    const std::vector<int> tiles = tiles_for(b->storage);
    size_t ubytes = 256;  // trial status word first, then u* copies
    for (lbm_ctx *c : b->m) ubytes += (size_t)2 * c->L.uplane * sizeof(double);
    char *scratch = nullptr;
    BK(b, cudaMallocAsync((void **)&scratch, ubytes, b->st));
    int *stat_scratch = reinterpret_cast<int *>(scratch);
    double *u_scratch = reinterpret_cast<double *>(scratch + 256);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    int chosen[NCLASS], chosen_dyn[NCLASS];
    for (int k = 0; k < NCLASS; ++k) {
        chosen[k] = b->vec[k];
        chosen_dyn[k] = b->dyn[k];
    }
    const std::vector<lbm_ctx *> all = b->m;
    const int n_all = b->n;
    // mean microseconds per step of the current tiles and orders on the
    // members `ms` alone (trial launches: scratch u* and status)
    auto trial = [&](const std::vector<lbm_ctx *> &ms, double &t_us) -> lbm_status {
        b->m = ms;
        b->n = (int)ms.size();
        Plan p;
        lbm_status r = make_plan(b, p);
        p.timed = false;  // trials take the time factors of the current step from the host
        if (r == LBM_OK) r = upload_plan(b, p, u_scratch, stat_scratch);
        if (r == LBM_OK) r = ensure_side_streams(b, (int)p.groups.size());
        float ms_ = 0.f;
        if (r == LBM_OK) {
            for (int i = 0; i < 2 && r == LBM_OK; ++i) r = enqueue_step(b, p, 0);  // warm-up
            if (r == LBM_OK) cudaEventRecord(t0, b->st);
            for (int i = 0; i < reps && r == LBM_OK; ++i) r = enqueue_step(b, p, 0);
            if (r == LBM_OK) {
                cudaEventRecord(t1, b->st);
                cudaError_t e = cudaEventSynchronize(t1);
                if (e != cudaSuccess) r = bcuda(b, e, "cudaEventSynchronize");
            }
            if (r == LBM_OK) cudaEventElapsedTime(&ms_, t0, t1);
        }
        b->m = all;
        b->n = n_all;
        t_us = 1000.0 * ms_ / reps;
        return r;
    };
    long long cls_nodes[NCLASS] = {};
    for (lbm_ctx *c : all) cls_nodes[size_class(c->L.nx)] += (long long)c->L.nx * c->L.ny;
    for (int cls = 0; cls < NCLASS && s == LBM_OK; ++cls) {
        // the batch viewed as this class's members alone
        std::vector<lbm_ctx *> mine;
        for (lbm_ctx *c : all)
            if (size_class(c->L.nx) == cls) mine.push_back(c);
        if (mine.empty()) continue;
        const int keep = b->vec[cls], keep_dyn = b->dyn[cls];
        double best = 1e300;
        for (size_t ti = 0; ti < tiles.size() && s == LBM_OK; ++ti)
            for (int order = 0; order < 2 && s == LBM_OK; ++order) {
                b->vec[cls] = tiles[ti];
                b->dyn[cls] = order;
                double t_us = 0.0;
                s = trial(mine, t_us);
                b->vec[cls] = keep;
                b->dyn[cls] = keep_dyn;
                if (s != LBM_OK) break;
                if (us && (order == 0 || t_us < us[cls * 3 + ti])) us[cls * 3 + ti] = t_us;
                if (t_us < best) {
                    best = t_us;
                    chosen[cls] = tiles[ti];
                    chosen_dyn[cls] = order;
                }
            }
    }
    // The orders were chosen one class at a time. Together, dynamic order in
    // a smaller class can cost more than it saved alone (256 specimens:
    // 0.897-0.899 of the copy bandwidth with classes 2 or 3 dynamic, 0.902
    // with only the largest): the whole batch is timed with the chosen
    // orders and with static order for every class but the one with the
    // most nodes, and the faster is kept.
    int big = 0;
    for (int k = 1; k < NCLASS; ++k)
        if (cls_nodes[k] > cls_nodes[big]) big = k;
    bool small_dyn = false;
    for (int k = 0; k < NCLASS; ++k)
        if (k != big && cls_nodes[k] > 0 && chosen_dyn[k]) small_dyn = true;
    if (s == LBM_OK && small_dyn) {
        int keep_vec[NCLASS], keep_dyn[NCLASS];
        for (int k = 0; k < NCLASS; ++k) {
            keep_vec[k] = b->vec[k];
            keep_dyn[k] = b->dyn[k];
            b->vec[k] = chosen[k];
            b->dyn[k] = chosen_dyn[k];
        }
        double t_chosen = 0.0, t_static = 0.0;
        s = trial(all, t_chosen);
        for (int k = 0; k < NCLASS; ++k)
            if (k != big) b->dyn[k] = 0;
        if (s == LBM_OK) s = trial(all, t_static);
        for (int k = 0; k < NCLASS; ++k) {
            b->vec[k] = keep_vec[k];
            b->dyn[k] = keep_dyn[k];
        }
        if (s == LBM_OK && t_static < t_chosen)
            for (int k = 0; k < NCLASS; ++k)
                if (k != big) chosen_dyn[k] = 0;
    }
    b->m = all;
    b->n = n_all;
    cudaFreeAsync(scratch, b->st);
    cudaStreamSynchronize(b->st);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (s != LBM_OK) return s;
    for (int k = 0; k < NCLASS; ++k) {
        b->vec[k] = chosen[k];
        b->dyn[k] = chosen_dyn[k];
    }
    b->have_plan = false;  // the device arrays hold trial arguments now
    drop_graph(b);
    BK(b, cudaEventRecord(b->ev_out, b->st));
    return join_streams(b, false);
}

lbm_status lbm_batch_step(lbm_batch *b, int64_t nsteps, int32_t graph_steps, int32_t *member_status)
{
    Range range_("lbm_batch_step");
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "null batch");
    if (nsteps < 0) return bfail(b, LBM_ERR_ARG, "nsteps must be >= 0");
    if (graph_steps < 0 || (graph_steps & 1) || graph_steps > TIME_CHUNK)
        return bfail(b, LBM_ERR_ARG, "graph_steps must be 0 or even and at most 1024");
    BK(b, cudaSetDevice(b->device));
    lbm_status s = members_ready(b);
    if (s != LBM_OK) return s;
    s = join_streams(b, true);
    if (s != LBM_OK) return s;
    s = current_plan(b);
    if (s == LBM_OK) s = upload_plan(b, b->plan, nullptr, nullptr);
    if (s == LBM_OK && nsteps > 0) s = run_steps(b, nsteps, graph_steps);
    if (s != LBM_OK) {
        // a failed enqueue leaves an unknown number of steps done: the
        // members' states are undefined (documented for LBM_ERR_CUDA)
        cudaStreamSynchronize(b->st);
        return s;
    }
    for (lbm_ctx *c : b->m) {
        c->cur ^= (int)(nsteps & 1);
        c->step += nsteps;
    }
    BK(b, cudaEventRecord(b->ev_out, b->st));
    s = join_streams(b, false);
    if (s != LBM_OK) return s;
    return gather_status(b, member_status);
}

lbm_status lbm_batch_info(const lbm_batch *b, int64_t *nodes, int32_t *launches_per_step, int32_t *graphs)
{
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "null batch");
    if (nodes) {
        int64_t t = 0;
        for (const lbm_ctx *c : b->m) t += (int64_t)c->L.nx * c->L.ny;
        *nodes = t;
    }
    if (launches_per_step) {
        Plan p;
        lbm_batch *mb = const_cast<lbm_batch *>(b);
        const std::string keep = mb->err;
        if (make_plan(mb, p) == LBM_OK)
            *launches_per_step = (int)p.groups.size() + (p.timed ? 1 : 0);
        else
            *launches_per_step = 0;
        mb->err = keep;
    }
    if (graphs) *graphs = b->graphs;
    return LBM_OK;
}

} // extern "C"
