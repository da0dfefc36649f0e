// lbm_step_f16.cu -- step and ghost-refresh kernels for FP16 storage.
#include "lbm_step_kernels.cuh"

namespace tlv {

TLV_STEP_ENTRY_POINTS(f16, __half)

} // namespace tlv
