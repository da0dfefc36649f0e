// lbm_batch_k16.cu -- batched step kernels for BF16 storage.
#include "lbm_batch_kernels.cuh"

namespace tlv {

const void *batch_kernel_bf16(int law, int vec) { return batch_kernel<__nv_bfloat16>(law, vec); }

} // namespace tlv
