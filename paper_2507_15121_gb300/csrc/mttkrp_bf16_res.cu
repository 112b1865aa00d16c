// mttkrp_bf16_res.cu — residual-mode (fused completion gradient) MTTKRP kernel
// instantiations for bf16 factors.
#include "dispatch.cuh"

AMPED_DEFINE_DTYPE_RESIDUAL_LAUNCHER(__nv_bfloat16, bf16)
