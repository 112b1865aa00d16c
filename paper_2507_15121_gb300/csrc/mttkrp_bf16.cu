// mttkrp_bf16.cu — MTTKRP and sampled-model kernel instantiations for bf16 factors.
#include "dispatch.cuh"

AMPED_DEFINE_DTYPE_LAUNCHERS(__nv_bfloat16, bf16)
