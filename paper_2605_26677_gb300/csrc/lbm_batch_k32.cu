// lbm_batch_k32.cu -- batched step kernels for FP32 storage (one translation
// unit per storage type, so that the build compiles them in parallel).
#include "lbm_batch_kernels.cuh"

namespace tlv {

const void *batch_kernel_f32(int law, int vec) { return batch_kernel<float>(law, vec); }

} // namespace tlv
