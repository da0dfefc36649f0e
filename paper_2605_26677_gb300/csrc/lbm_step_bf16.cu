// lbm_step_bf16.cu -- step and ghost-refresh kernels for BF16 storage.
#include "lbm_step_kernels.cuh"

namespace tlv {

TLV_STEP_ENTRY_POINTS(bf16, __nv_bfloat16)

} // namespace tlv
