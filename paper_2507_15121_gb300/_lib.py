"""ctypes binding of libamped.so (the C ABI declared in include/amped.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# AMPED_LIB selects another build of the same library (the bounds-checked one,
# for example); it must exist like the default one.
LIB_PATH = os.environ.get("AMPED_LIB") or os.path.join(_HERE, "libamped.so")

OK, ERR_INVALID, ERR_INDEX, ERR_OOM, ERR_CUDA, ERR_UNSUPPORTED, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
F32, BF16, F16 = 0, 1, 2
ALS_INIT = 1  # amped_cp_als_sweep flag: compute the Grams of the given factors first
MAX_MODES = 8

_STATUS = {OK: "ok", ERR_INVALID: "invalid argument", ERR_INDEX: "index out of range", ERR_OOM: "out of memory",
           ERR_CUDA: "CUDA error", ERR_UNSUPPORTED: "unsupported", ERR_TIMEOUT: "timeout"}


class AmpedError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("segment_items", ctypes.c_int32), ("keep_perm", ctypes.c_int32), ("keep_coo", ctypes.c_int32),
                ("max_rank", ctypes.c_int32), ("host_threads", ctypes.c_int32), ("inner_order", ctypes.c_int32),
                ("short_rows", ctypes.c_int32), ("stream_memory", ctypes.c_int32)]


class PlanSizes(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("nnz", "rows", "long_rows", "long_nnz", "short_rows", "long_segments",
                                              "short_segments", "split_rows")]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library (built by ``paper_2507_15121_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libamped.so is not built ({LIB_PATH}); run "
                              "`python -m paper_2507_15121_gb300.build` or __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        st = c_int
        sig = {
            "amped_tensor_create": ([i64, c_int, vp, vp, vp, ctypes.POINTER(Opts), ctypes.POINTER(vp)], st),
            "amped_tensor_destroy": ([vp], st),
            "amped_tensor_info": ([vp, ctypes.POINTER(i64), ctypes.POINTER(c_int), vp], st),
            "amped_mttkrp": ([vp, c_int, vp, c_int, c_int, vp, vp], st),
            "amped_mttkrp_all": ([vp, vp, c_int, c_int, vp, vp], st),
            "amped_mttkrp_noalloc": ([vp, c_int, vp, c_int, c_int, vp, vp], st),
            "amped_mttkrp_all_host": ([vp, vp, c_int, c_int, vp, vp], st),
            "amped_cp_sample": ([vp, vp, c_int, c_int, vp, vp], st),
            "amped_cp_grad": ([vp, vp, c_int, c_int, vp, vp, vp], st),
            "amped_cp_completion_grad": ([vp, vp, c_int, c_int, vp, vp, vp], st),
            "amped_plan_mode": ([i64, c_int, vp, vp, c_int, c_int, c_int, c_int, ctypes.POINTER(PlanSizes)]
                                + [vp] * 9, st),
            "amped_tensor_norm2": ([vp, ctypes.POINTER(ctypes.c_double)], st),
            "amped_norm2_host": ([i64, c_int, vp, vp, vp, c_int, ctypes.POINTER(ctypes.c_double)], st),
            "amped_cp_als_sweep": ([vp, vp, c_int, vp, vp, c_int, vp], st),
            "amped_cp_als_normalize": ([vp, vp, c_int, vp, vp, vp], st),
            "amped_cp_als_update": ([vp, c_int, vp, c_int, vp, vp, c_int, vp], st),
            "amped_set_kernel_events": ([vp, vp, vp], st),
            "amped_kernel_launches": ([], i64),
            "amped_last_error": ([], ctypes.c_char_p),
            "amped_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != OK:
        raise AmpedError(status, lib().amped_last_error().decode(errors="replace"))


def version() -> str:
    return lib().amped_version().decode()


def kernel_launches() -> int:
    return int(lib().amped_kernel_launches())


def ptr_array(ptrs) -> ctypes.Array:
    return (ctypes.c_void_p * len(ptrs))(*[ctypes.c_void_p(p) if p else None for p in ptrs])
