// lbm_batch_kf16.cu -- batched step kernels for FP16 storage.
#include "lbm_batch_kernels.cuh"

namespace tlv {

const void *batch_kernel_f16(int law, int vec) { return batch_kernel<__half>(law, vec); }

} // namespace tlv
