// lbm_step_f32.cu -- step and ghost-refresh kernels for FP32 storage.
#include "lbm_step_kernels.cuh"

namespace tlv {

TLV_STEP_ENTRY_POINTS(f32, float)

} // namespace tlv
