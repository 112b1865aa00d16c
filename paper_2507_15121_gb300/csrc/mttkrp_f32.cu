// mttkrp_f32.cu — MTTKRP and sampled-model kernel instantiations for f32 factors.
#include "dispatch.cuh"

AMPED_DEFINE_DTYPE_LAUNCHERS(float, f32)
