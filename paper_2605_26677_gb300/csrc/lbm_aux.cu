// lbm_aux.cu -- initialization, read-out and diagnostics kernels of the TL
// vectorial D2Q4x6 LBM. Read-out and diagnostics compute in FP64 whatever the
// storage; the initialization computes in FP64 for FP64 storage and in FP32
// otherwise (u* always in FP64).
#include <cfloat>

#include "lbm_init_core.cuh"
#include <type_traits>

namespace tlv {

// Initial populations (Sec. 3.4) followed by the collision of step 0, so the
// stored state is f*^0; u* receives u0 - (dt/2) v0 + dt v^0 (Eq. 22).
template <typename T>
__global__ void __launch_bounds__(128) k_init(const InitArgs a)
{
    using R = typename std::conditional<sizeof(T) == 8, double, float>::type;  // compute type
    const int nx = a.L.nx, ny = a.L.ny;
    const long long N = (long long)nx * ny;
    T *fout = static_cast<T *>(a.fout);
    const double dt = a.dt;
    const R c = (R)a.c, w = (R)a.omega;
    const long long n1 = (long long)a.y1 * nx;
    for (long long n = (long long)a.y0 * nx + (long long)blockIdx.x * blockDim.x + threadIdx.x; n < n1;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % nx), y = (int)(n / nx);
        R f[4][6];  // f^0 - f_rest
        const LawP<R> m = law_cast<R>(law_at(a.m, n));
        if (!init_node_ofs<R>(a, x, y, m, f)) atomicOr(a.status, ST_BAD_J);
        // step-0 collision (Eqs. 10, 12, 14) on the offsets from the rest
        // state, which the collision leaves fixed
        R Un[6], dJ;
#pragma unroll
        for (int k = 0; k < 6; ++k) Un[k] = (f[0][k] + f[2][k]) + (f[1][k] + f[3][k]);
        Un[0] += (R)(0.5 * dt * a.b1);
        Un[1] += (R)(0.5 * dt * a.b2);
        const R Gn[4] = {Un[2], Un[3], Un[4], Un[5]};
        R Pn[4], feq[4][6];
        piola_any_t<R>(a.m.law, Gn, m, Pn, dJ);
        feq_ofs<R>(Un, Pn, c, feq);
        const R src[2] = {(R)(dt * (2.0 - a.omega) * 0.125 * a.b1), (R)(dt * (2.0 - a.omega) * 0.125 * a.b2)};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                R fs = f[q][k] + w * (feq[q][k] - f[q][k]);
                if (k < 2) fs += src[k];
                fout[pidx(a.L, q, k, x, y)] = to_store<T>(fs);
            }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const double u0 = a.u0 ? a.u0[k * N + n] : 0.0;
            a.ustar[k * a.L.uplane + (long long)y * a.L.upitch + x] =
                (u0 - 0.5 * dt * a.U0[k * N + n]) + dt * (double)Un[k];
        }
    }
}

template <typename R>
__global__ void k_mu_plane(const double *mu, R *plane, Layout L)
{
    const long long N = (long long)L.nx * L.ny;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % L.nx), y = (int)(n / L.nx);
        plane[(long long)y * L.upitch + x] = (R)mu[n];
    }
}

// U^n = sum_q f*_q - (dt/2) B, P(F^n), sigma = J^{-1} P F^T, u^n = u* - (dt/2) v^n
// (the stored u* already holds u*^{n+1} = u*^n + dt v^n)
template <typename T>
__global__ void __launch_bounds__(128) k_read(const ReadArgs a)
{
    const int nx = a.L.nx, ny = a.L.ny;
    const long long N = (long long)nx * ny;
    const T *f = static_cast<const T *>(a.f);
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % nx), y = (int)(n / nx);
        double S[6];
        for (int k = 0; k < 6; ++k) {
            double s = 0.0;
            for (int q = 0; q < 4; ++q) s += (double)ld_r(f[pidx(a.L, q, k, x, y)]);
            S[k] = s;
        }
        const double v1 = S[0] - 0.5 * a.dt * a.b1, v2 = S[1] - 0.5 * a.dt * a.b2;
        const double G[4] = {S[2], S[3], S[4], S[5]};
        if (a.U) {
            a.U[0 * N + n] = v1;
            a.U[1 * N + n] = v2;
            a.U[2 * N + n] = 1.0 + G[0];
            a.U[3 * N + n] = G[1];
            a.U[4 * N + n] = G[2];
            a.U[5 * N + n] = 1.0 + G[3];
        }
        if (a.P || a.sigma) {
            double P[4], dJ;
            piola_any(a.m.law, G, law_at(a.m, n), P, dJ);
            if (a.P)
                for (int m = 0; m < 4; ++m) a.P[m * N + n] = P[m];
            if (a.sigma) {
                const double F[4] = {1.0 + G[0], G[1], G[2], 1.0 + G[3]};
                const double J = 1.0 + dJ;
                a.sigma[0 * N + n] = (P[0] * F[0] + P[1] * F[1]) / J;
                a.sigma[1 * N + n] = (P[0] * F[2] + P[1] * F[3]) / J;
                a.sigma[2 * N + n] = (P[2] * F[0] + P[3] * F[1]) / J;
                a.sigma[3 * N + n] = (P[2] * F[2] + P[3] * F[3]) / J;
            }
        }
        if (a.u) {
            const long long ui = (long long)y * a.L.upitch + x;
            a.u[0 * N + n] = a.ustar[ui] - 0.5 * a.dt * v1;
            a.u[1 * N + n] = a.ustar[a.L.uplane + ui] - 0.5 * a.dt * v2;
        }
    }
}

// ---------------------------------------------------------------- diagnostics
// Ten reduced values: 7 sums (v1, v2, G11, G12, G21, G22, energy density),
// min J, max J, max |F - I|_F. Per-block partials, then one block combines them
// in a fixed order, so the result does not depend on scheduling.
constexpr int DIAG_THREADS = 256;
constexpr int DIAG_MAX_BLOCKS = 1024;

struct Red {
    double s[7];
    double jmin, jmax, gmax;
};

static __device__ __forceinline__ void red_combine(Red &r, const Red &o)
{
    for (int i = 0; i < 7; ++i) r.s[i] += o.s[i];
    r.jmin = fmin(r.jmin, o.jmin);
    r.jmax = fmax(r.jmax, o.jmax);
    r.gmax = fmax(r.gmax, o.gmax);
}

static __device__ Red block_reduce(Red r)
{
    __shared__ double sh[DIAG_THREADS / 32][10];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int off = 16; off > 0; off >>= 1) {
        Red o;
        for (int i = 0; i < 7; ++i) o.s[i] = __shfl_down_sync(0xffffffffu, r.s[i], off);
        o.jmin = __shfl_down_sync(0xffffffffu, r.jmin, off);
        o.jmax = __shfl_down_sync(0xffffffffu, r.jmax, off);
        o.gmax = __shfl_down_sync(0xffffffffu, r.gmax, off);
        red_combine(r, o);
    }
    if (lane == 0) {
        for (int i = 0; i < 7; ++i) sh[w][i] = r.s[i];
        sh[w][7] = r.jmin;
        sh[w][8] = r.jmax;
        sh[w][9] = r.gmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int ww = 1; ww < DIAG_THREADS / 32; ++ww) {
            Red o;
            for (int i = 0; i < 7; ++i) o.s[i] = sh[ww][i];
            o.jmin = sh[ww][7];
            o.jmax = sh[ww][8];
            o.gmax = sh[ww][9];
            red_combine(r, o);
        }
    }
    return r;
}

template <typename T>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag_partial(const DiagArgs a)
{
    const int nx = a.L.nx, ny = a.L.ny;
    const long long N = (long long)nx * ny;
    const T *f = static_cast<const T *>(a.f);
    Red r;
    for (int i = 0; i < 7; ++i) r.s[i] = 0.0;
    r.jmin = DBL_MAX;
    r.jmax = -DBL_MAX;
    r.gmax = 0.0;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % nx), y = (int)(n / nx);
        double S[6];
        for (int k = 0; k < 6; ++k) {
            double s = 0.0;
            for (int q = 0; q < 4; ++q) s += (double)ld_r(f[pidx(a.L, q, k, x, y)]);
            S[k] = s;
        }
        const double v1 = S[0] - 0.5 * a.dt * a.b1, v2 = S[1] - 0.5 * a.dt * a.b2;
        const double dJ = S[2] + S[5] + (S[2] * S[5] - S[3] * S[4]);
        r.s[0] += v1;
        r.s[1] += v2;
        for (int m = 0; m < 4; ++m) r.s[2 + m] += S[2 + m];
        r.s[6] += 0.5 * (v1 * v1 + v2 * v2) + energy_ofs(a.m.law, S[2], S[3], S[4], S[5], law_at(a.m, n));
        r.jmin = fmin(r.jmin, 1.0 + dJ);
        r.jmax = fmax(r.jmax, 1.0 + dJ);
        r.gmax = fmax(r.gmax, sqrt(S[2] * S[2] + S[3] * S[3] + S[4] * S[4] + S[5] * S[5]));
    }
    r = block_reduce(r);
    if (threadIdx.x == 0) {
        double *p = a.partial + (long long)blockIdx.x * 10;
        for (int i = 0; i < 7; ++i) p[i] = r.s[i];
        p[7] = r.jmin;
        p[8] = r.jmax;
        p[9] = r.gmax;
    }
}

__global__ void __launch_bounds__(DIAG_THREADS) k_diag_final(const DiagArgs a, int nblocks)
{
    Red r;
    for (int i = 0; i < 7; ++i) r.s[i] = 0.0;
    r.jmin = DBL_MAX;
    r.jmax = -DBL_MAX;
    r.gmax = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double *p = a.partial + (long long)b * 10;
        Red o;
        for (int i = 0; i < 7; ++i) o.s[i] = p[i];
        o.jmin = p[7];
        o.jmax = p[8];
        o.gmax = p[9];
        red_combine(r, o);
    }
    r = block_reduce(r);
    if (threadIdx.x == 0) {
        const double N = (double)a.L.nx * (double)a.L.ny;
        a.out[0] = r.s[0];
        a.out[1] = r.s[1];
        a.out[2] = 1.0 + r.s[2] / N;
        a.out[3] = r.s[3] / N;
        a.out[4] = r.s[4] / N;
        a.out[5] = 1.0 + r.s[5] / N;
        a.out[6] = a.dx * a.dx * r.s[6];
        a.out[7] = r.jmin;
        a.out[8] = r.jmax;
        a.out[9] = r.gmax;
    }
}

// ---------------------------------------------------------------- launchers
static int grid_for(long long n, int threads)
{
    long long g = (n + threads - 1) / threads;
    if (g > 65535LL * 16) g = 65535LL * 16;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_init(int storage, const InitArgs &a, cudaStream_t st)
{
    // the kernel writes rows [y0, y1) and reads U0 around them: a range
    // outside the lattice is an error, an empty one a no-op
    if (a.y0 < 0 || a.y1 > a.L.ny || a.y1 < a.y0) return cudaErrorInvalidValue;
    if (a.y1 == a.y0) return cudaSuccess;
    const int g = grid_for((long long)a.L.nx * (a.y1 - a.y0), 128);
    return with_storage(storage, [&](auto tag) {
        k_init<decltype(tag)><<<g, 128, 0, st>>>(a);
        return cudaGetLastError();
    });
}

cudaError_t launch_read(int storage, const ReadArgs &a, cudaStream_t st)
{
    const int g = grid_for((long long)a.L.nx * a.L.ny, 128);
    return with_storage(storage, [&](auto tag) {
        k_read<decltype(tag)><<<g, 128, 0, st>>>(a);
        return cudaGetLastError();
    });
}

int diag_blocks(const Layout &L)
{
    const long long n = (long long)L.nx * L.ny;
    long long b = (n + DIAG_THREADS - 1) / DIAG_THREADS;
    if (b > DIAG_MAX_BLOCKS) b = DIAG_MAX_BLOCKS;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_diag(int storage, const DiagArgs &a, cudaStream_t st)
{
    const int nb = diag_blocks(a.L);
    with_storage(storage, [&](auto tag) {
        k_diag_partial<decltype(tag)><<<nb, DIAG_THREADS, 0, st>>>(a);
        return 0;
    });
    k_diag_final<<<1, DIAG_THREADS, 0, st>>>(a, nb);
    return cudaGetLastError();
}

cudaError_t launch_mu_plane(int storage, const double *mu, void *plane, const Layout &L, cudaStream_t st)
{
    const long long N = (long long)L.nx * L.ny;
    const int grid = (int)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096);
    if (storage == STORE_F64)
        k_mu_plane<double><<<grid, 256, 0, st>>>(mu, static_cast<double *>(plane), L);
    else
        k_mu_plane<float><<<grid, 256, 0, st>>>(mu, static_cast<float *>(plane), L);
    return cudaGetLastError();
}

constexpr int STATS_BLOCKS = 256;

__global__ void __launch_bounds__(256) k_field_stats(const double *v, long long n, double *partial)
{
    __shared__ double smin[256], smax[256], sbad[256];
    double lo = DBL_MAX, hi = -DBL_MAX, bad = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double x = v[i];
        if (!isfinite(x)) {
            bad += 1.0;
        } else {
            lo = fmin(lo, x);
            hi = fmax(hi, x);
        }
    }
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    sbad[threadIdx.x] = bad;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
            sbad[threadIdx.x] += sbad[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[3 * blockIdx.x] = smin[0];
        partial[3 * blockIdx.x + 1] = smax[0];
        partial[3 * blockIdx.x + 2] = sbad[0];
    }
}

cudaError_t launch_field_stats(const double *v, long long n, double out[3], cudaStream_t st)
{
    double *partial = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&partial, 3 * STATS_BLOCKS * sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_field_stats<<<STATS_BLOCKS, 256, 0, st>>>(v, n, partial);
    double h[3 * STATS_BLOCKS];
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, partial, sizeof h, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(partial, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    out[0] = DBL_MAX;
    out[1] = -DBL_MAX;
    out[2] = 0.0;
    for (int b = 0; b < STATS_BLOCKS; ++b) {
        out[0] = fmin(out[0], h[3 * b]);
        out[1] = fmax(out[1], h[3 * b + 1]);
        out[2] += h[3 * b + 2];
    }
    return cudaSuccess;
}

} // namespace tlv
