// mttkrp_f32_res.cu — residual-mode (fused completion gradient) MTTKRP kernel
// instantiations for f32 factors.
#include "dispatch.cuh"

AMPED_DEFINE_DTYPE_RESIDUAL_LAUNCHER(float, f32)
