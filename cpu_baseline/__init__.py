"""All-cores FP64 CPU MTTKRP: the multithreaded CPU baseline the benchmark
times beside the single-threaded oracle.

Not the oracle and not the product: ``cpu_mttkrp.c`` is its own OpenMP
restatement of the elementwise MTTKRP (paper Sec. 3, Alg. 2) over a copy of
the nonzeros ordered by the output coordinate, each thread owning whole
output rows.  ``order`` (the sort) is preprocessing and is not timed;
``mttkrp`` is the timed part.  Checked against the oracle in
``tests/test_cpu_baseline.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_mttkrp.c")
_LIB = os.path.join(_HERE, "libcpumttkrp.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile libcpumttkrp.so in place (gcc -O2 -fopenmp)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, c_int, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.cpu_order.argtypes = [i64, c_int, vp, vp, c_int, vp, vp]
        lib.cpu_mttkrp.argtypes = [i64, c_int, vp, vp, vp, vp, c_int, c_int, vp, vp, vp, c_int]
        lib.cpu_order.restype = lib.cpu_mttkrp.restype = lib.cpu_threads.restype = c_int
        _lib = lib
    return _lib


def threads() -> int:
    """Threads the OpenMP runtime uses by default (all host cores unless OMP_NUM_THREADS says otherwise)."""
    return int(_L().cpu_threads())


def order(dims, idx, mode: int):
    """(perm, rowptr): the nonzeros ordered by coordinate `mode`."""
    dims_a = np.ascontiguousarray(np.asarray(dims, dtype=np.int64))
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    perm = np.empty(idx.shape[0], dtype=np.int32)
    rowptr = np.empty(int(dims_a[mode]) + 1, dtype=np.int64)
    if _L().cpu_order(idx.shape[0], idx.shape[1], dims_a.ctypes.data, idx.ctypes.data, mode, perm.ctypes.data,
                      rowptr.ctypes.data) != 0:
        raise MemoryError("cpu_order")
    return perm, rowptr


def mttkrp(dims, idx, vals, factors, mode: int, ordered, out=None, nthreads: int = 0) -> np.ndarray:
    """Mode-`mode` MTTKRP in FP64 with fp32 factors, on every host core."""
    dims_a = np.ascontiguousarray(np.asarray(dims, dtype=np.int64))
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float32)
    fs = [np.ascontiguousarray(f, dtype=np.float32) for f in factors]
    R = int(fs[0].shape[1])
    fp = (ctypes.c_void_p * len(fs))(*[f.ctypes.data for f in fs])
    perm, rowptr = ordered
    if out is None:
        out = np.empty((int(dims_a[mode]), R), dtype=np.float64)
    if _L().cpu_mttkrp(idx.shape[0], idx.shape[1], dims_a.ctypes.data, idx.ctypes.data, vals.ctypes.data, fp, R,
                       mode, perm.ctypes.data, rowptr.ctypes.data, out.ctypes.data, nthreads) != 0:
        raise ValueError("cpu_mttkrp: bad argument")
    return out
