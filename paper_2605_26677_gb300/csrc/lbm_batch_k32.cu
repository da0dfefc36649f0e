// lbm_batch_k32.cu -- batched step kernels for FP64 and FP32 storage.
#include "lbm_batch_kernels.cuh"

namespace tlv {

const void *batch_kernel_wide(int storage, int law, int vec)
{
    return storage == STORE_F64 ? batch_kernel<double>(law, vec) : batch_kernel<float>(law, vec);
}

} // namespace tlv
