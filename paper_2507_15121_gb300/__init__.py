"""GB300-native sparse MTTKRP (the hot path of AMPED, arXiv 2507.15121).

All-mode sparse MTTKRP for N-mode COO tensors on one GPU, written as
hand-tuned sm_103a CUDA behind a C ABI (``include/amped.h``,
``libamped.so``): a host-side reorder builds one output-row-ordered,
segmented copy per mode; a persistent kernel whose workers pull segments
from a device-wide ticket counter streams the coordinates with 128-bit
loads, gathers factor rows and accumulates each output row in registers.
Factors may be stored in fp32, bf16 or fp16 (arithmetic in fp32); tensors
have 2 to 8 modes, and their per-nonzero streams may stay in host memory
(out-of-core, read over the host link).  ``torch.autograd.Function``s give
the sampled CP model with an MTTKRP backward and a fused completion loss for
gradient-based CP completion; ``Tensor.cp_als`` runs CP decomposition by
alternating least squares (fp64 normal-equation solve on the GPU).
"""
from ._lib import AmpedError, kernel_launches, version  # noqa: F401
from .tensor import Tensor, plan_mode  # noqa: F401

try:
    from .autograd import (CPCompletionLoss, CPSampled, completion_loss, fused_completion_loss,  # noqa: F401
                           sampled_model)
except ImportError:  # torch missing: only the host planning query is usable
    pass
