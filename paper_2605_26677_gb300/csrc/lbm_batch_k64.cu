// lbm_batch_k64.cu -- batched step kernels for FP64 storage.
#include "lbm_batch_kernels.cuh"

namespace tlv {

const void *batch_kernel_f64(int law, int vec) { return batch_kernel<double>(law, vec); }

} // namespace tlv
