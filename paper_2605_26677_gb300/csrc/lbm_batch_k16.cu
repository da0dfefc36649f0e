// lbm_batch_k16.cu -- batched step kernels for BF16 and FP16 storage.
#include "lbm_batch_kernels.cuh"

namespace tlv {

const void *batch_kernel_16(int storage, int law, int vec)
{
    return storage == STORE_BF16 ? batch_kernel<__nv_bfloat16>(law, vec) : batch_kernel<__half>(law, vec);
}

} // namespace tlv
