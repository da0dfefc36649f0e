// lbm_noalloc.cu -- diagnostics reduction that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: applications that hand
// out all device memory from their own pool and account for every byte, or
// latency-critical loops that must not pay for (or be serialised by) an
// allocation. For them lbm_diagnostics_state_noalloc reduces a caller-owned
// FP64 state field into caller-owned output, and keeps its per-block partial
// sums in the file-scope array below instead of allocated scratch.
//
// The array is fixed at NOALLOC_MAX_BLOCKS * 10 doubles (1.25 MiB); every
// GPU that loads this library holds it until the process exits. One block
// reduces NOALLOC_NODES_PER_BLOCK nodes, so a call accepts at most
// NOALLOC_MAX_BLOCKS * NOALLOC_NODES_PER_BLOCK = 67,108,864 nodes (8192^2).
// All calls share the array: two calls whose kernels overlap on the GPU (on
// different streams, or on one stream from different host threads) race on
// it. Each call overwrites every slot it later reads, so nothing needs
// clearing between calls. The material is the uniform closure the caller
// names; the call makes `device` current only while it runs and gives the
// calling thread back its previous current device on every return.
#include <cfloat>
#include <mutex>
#include <string>

#include "lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_NODES_PER_THREAD = 16;
constexpr long long NOALLOC_NODES_PER_BLOCK = (long long)NOALLOC_THREADS * NOALLOC_NODES_PER_THREAD;
constexpr int NOALLOC_MAX_BLOCKS = 16384;
constexpr int NOALLOC_SLOT = 10;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS * NOALLOC_SLOT];

struct NoallocArgs {
    const double *U;  // 6 x N, component-major (v1, v2, F11, F12, F21, F22)
    long long N;
    tlv::Material m;
    double dx;
    double *partial;  // device address of g_noalloc_partials
    double *out;      // 10 doubles
    int nblocks;
};

struct Acc {
    double s[7];
    double jmin, jmax, gmax;
};

__device__ __forceinline__ void acc_init(Acc &a)
{
    for (int i = 0; i < 7; ++i) a.s[i] = 0.0;
    a.jmin = DBL_MAX;
    a.jmax = -DBL_MAX;
    a.gmax = 0.0;
}

__device__ __forceinline__ void acc_add(Acc &a, const Acc &b)
{
    for (int i = 0; i < 7; ++i) a.s[i] += b.s[i];
    a.jmin = fmin(a.jmin, b.jmin);
    a.jmax = fmax(a.jmax, b.jmax);
    a.gmax = fmax(a.gmax, b.gmax);
}

// block-wide reduction; the result is valid in thread 0
__device__ Acc acc_block(Acc a)
{
    __shared__ double sh[NOALLOC_THREADS / 32][NOALLOC_SLOT];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int off = 16; off > 0; off >>= 1) {
        Acc o;
        for (int i = 0; i < 7; ++i) o.s[i] = __shfl_down_sync(0xffffffffu, a.s[i], off);
        o.jmin = __shfl_down_sync(0xffffffffu, a.jmin, off);
        o.jmax = __shfl_down_sync(0xffffffffu, a.jmax, off);
        o.gmax = __shfl_down_sync(0xffffffffu, a.gmax, off);
        acc_add(a, o);
    }
    if (lane == 0) {
        for (int i = 0; i < 7; ++i) sh[w][i] = a.s[i];
        sh[w][7] = a.jmin;
        sh[w][8] = a.jmax;
        sh[w][9] = a.gmax;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int ww = 1; ww < NOALLOC_THREADS / 32; ++ww) {
            Acc o;
            for (int i = 0; i < 7; ++i) o.s[i] = sh[ww][i];
            o.jmin = sh[ww][7];
            o.jmax = sh[ww][8];
            o.gmax = sh[ww][9];
            acc_add(a, o);
        }
    return a;
}

// block b reduces nodes [b * NODES_PER_BLOCK, (b + 1) * NODES_PER_BLOCK) into slot b
__global__ void __launch_bounds__(NOALLOC_THREADS) k_noalloc_partial(const NoallocArgs a)
{
    Acc acc;
    acc_init(acc);
    const long long base = (long long)blockIdx.x * NOALLOC_NODES_PER_BLOCK;
    for (int j = 0; j < NOALLOC_NODES_PER_THREAD; ++j) {
        const long long n = base + (long long)j * NOALLOC_THREADS + threadIdx.x;
        if (n >= a.N) break;
        const double v1 = a.U[n], v2 = a.U[a.N + n];
        const double G11 = a.U[2 * a.N + n] - 1.0, G12 = a.U[3 * a.N + n];
        const double G21 = a.U[4 * a.N + n], G22 = a.U[5 * a.N + n] - 1.0;
        const double J = 1.0 + (G11 + G22 + (G11 * G22 - G12 * G21));
        acc.s[0] += v1;
        acc.s[1] += v2;
        acc.s[2] += G11;
        acc.s[3] += G12;
        acc.s[4] += G21;
        acc.s[5] += G22;
        acc.s[6] += 0.5 * (v1 * v1 + v2 * v2) + tlv::energy_ofs(a.m.law, G11, G12, G21, G22, tlv::law_at(a.m, 0));
        acc.jmin = fmin(acc.jmin, J);
        acc.jmax = fmax(acc.jmax, J);
        acc.gmax = fmax(acc.gmax, sqrt(G11 * G11 + G12 * G12 + G21 * G21 + G22 * G22));
    }
    acc = acc_block(acc);
    if (threadIdx.x == 0) {
        double *p = a.partial + (long long)blockIdx.x * NOALLOC_SLOT;
        for (int i = 0; i < 7; ++i) p[i] = acc.s[i];
        p[7] = acc.jmin;
        p[8] = acc.jmax;
        p[9] = acc.gmax;
    }
}

__global__ void __launch_bounds__(NOALLOC_THREADS) k_noalloc_final(const NoallocArgs a)
{
    Acc acc;
    acc_init(acc);
    for (int b = threadIdx.x; b < a.nblocks; b += NOALLOC_THREADS) {
        const double *p = a.partial + (long long)b * NOALLOC_SLOT;
        Acc o;
        for (int i = 0; i < 7; ++i) o.s[i] = p[i];
        o.jmin = p[7];
        o.jmax = p[8];
        o.gmax = p[9];
        acc_add(acc, o);
    }
    acc = acc_block(acc);
    if (threadIdx.x == 0) {
        const double N = (double)a.N;
        a.out[0] = acc.s[0];
        a.out[1] = acc.s[1];
        a.out[2] = 1.0 + acc.s[2] / N;
        a.out[3] = acc.s[3] / N;
        a.out[4] = acc.s[4] / N;
        a.out[5] = 1.0 + acc.s[5] / N;
        a.out[6] = a.dx * a.dx * acc.s[6];
        a.out[7] = acc.jmin;
        a.out[8] = acc.jmax;
        a.out[9] = acc.gmax;
    }
}

// device address of g_noalloc_partials, looked up once per device
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// the message is read back with lbm_last_error(NULL)
lbm_status noalloc_fail(lbm_status s, const std::string &msg)
{
    tlv::set_thread_error(msg);
    return s;
}

// restores the calling thread's current device when the call returns
struct DeviceRestore {
    int prev = -1;
    DeviceRestore()
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            prev = -1;
            cudaGetLastError();
        }
    }
    ~DeviceRestore()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

} // namespace

extern "C" lbm_status lbm_diagnostics_state_noalloc(const double *U_dev, int32_t nx, int32_t ny, int32_t law,
                                                    const double *params, int32_t nparams, double dx,
                                                    double *out_dev, int32_t device, void *stream)
{
    if (!U_dev || !out_dev) return noalloc_fail(LBM_ERR_ARG, "U_dev and out_dev must be device pointers");
    if (nx < 1 || ny < 1) return noalloc_fail(LBM_ERR_ARG, "nx and ny must be >= 1");
    const long long N = (long long)nx * ny;
    const long long max_nodes = (long long)NOALLOC_MAX_BLOCKS * NOALLOC_NODES_PER_BLOCK;
    if (N > max_nodes)
        return noalloc_fail(LBM_ERR_ARG, "grid of " + std::to_string(N) + " nodes exceeds the static scratch "
                                         "capacity of " + std::to_string(max_nodes) + " nodes");
    static const int need[6] = {2, 2, 2, 3, 4, 3};
    if (law < LBM_LAW_SVK || law > LBM_LAW_GENT) return noalloc_fail(LBM_ERR_ARG, "unknown law");
    if (!params || nparams < need[law]) return noalloc_fail(LBM_ERR_ARG, "too few closure parameters");
    if (!(dx > 0.0)) return noalloc_fail(LBM_ERR_ARG, "dx must be > 0");
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) return noalloc_fail(LBM_ERR_ARG, "device ordinal out of range");
    DeviceRestore restore_;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return noalloc_fail(LBM_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    double *partial;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[device]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess)
                return noalloc_fail(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_noalloc_ptr[device] = static_cast<double *>(p);
        }
        partial = g_noalloc_ptr[device];
    }
    NoallocArgs a;
    a.U = U_dev;
    a.N = N;
    a.m.law = law;
    a.m.lam = params[0];
    a.m.mu = params[1];
    a.m.p2 = nparams > 2 ? params[2] : 0.0;
    a.m.p3 = nparams > 3 ? params[3] : 0.0;
    a.m.mufield = nullptr;
    a.m.lam_ratio = 0.0;
    a.dx = dx;
    a.partial = partial;
    a.out = out_dev;
    a.nblocks = (int)((N + NOALLOC_NODES_PER_BLOCK - 1) / NOALLOC_NODES_PER_BLOCK);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_noalloc_partial<<<a.nblocks, NOALLOC_THREADS, 0, st>>>(a);
    k_noalloc_final<<<1, NOALLOC_THREADS, 0, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(LBM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return LBM_OK;
}
