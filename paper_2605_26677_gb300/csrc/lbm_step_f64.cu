// lbm_step_f64.cu -- step and ghost-refresh kernels for FP64 storage.
#include "lbm_step_kernels.cuh"

namespace tlv {

TLV_STEP_ENTRY_POINTS(f64, double)

} // namespace tlv
