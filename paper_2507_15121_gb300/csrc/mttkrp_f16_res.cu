// mttkrp_f16_res.cu — residual-mode (fused completion gradient) MTTKRP kernel
// instantiations for f16 factors.
#include "dispatch.cuh"

AMPED_DEFINE_DTYPE_RESIDUAL_LAUNCHER(__half, f16)
