// lbm_internal.h -- host-side declarations shared by the library's
// translation units (kernel launchers); not part of the public C ABI.
#pragma once
#include <string>

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace tlv {

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
};
cudaError_t launch_init(int storage, const InitArgs &a, cudaStream_t st);

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

// lbm_api.cu: message returned by lbm_last_error(NULL) on this host thread
void set_thread_error(const std::string &msg);

} // namespace tlv
