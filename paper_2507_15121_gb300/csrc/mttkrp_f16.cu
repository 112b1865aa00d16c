// mttkrp_f16.cu — MTTKRP and sampled-model kernel instantiations for f16 factors.
#include "dispatch.cuh"

AMPED_DEFINE_DTYPE_LAUNCHERS(__half, f16)
