"""FP64 CPU oracle for sparse MTTKRP, the sampled CP model and its gradient.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only callers.  The GPU
library (``paper_2507_15121_gb300``) never imports this package and this
package never imports it.

The arithmetic lives in ``oracle.c`` (plain single-threaded loops in double
precision, in the order the nonzeros are given); this module only marshals
numpy arrays.  What it follows:

* MTTKRP, mode d: the elementwise computation of Sec. 3 (one nonzero adds
  val * Hadamard product of the other modes' factor rows into row i_d of the
  output), generalised to N modes as in Alg. 2, summed over all nonzeros of
  a zero-initialised output; equal to X_(d) times the Khatri-Rao product of
  the other factors (Sec. 2.1, Eq. 1).
* Sampled CP model: m = sum_r prod_n A_n(i_n, r) at each nonzero, the CP
  model of Sec. 2.1 evaluated at the tensor's coordinates.
* Gradient of a per-nonzero loss: dL/dA_n = MTTKRP_n with the values
  replaced by dL/dm.  With the completion loss L = 1/2 sum_k (m_k - x_k)^2
  the per-nonzero derivative is m_k - x_k.

Pins (tests/test_oracle_pins.py): brute force through dense unfolding and an
explicit Khatri-Rao product, the closed form for an exact dense CP tensor,
the N=2 sparse-matrix product, a hand-worked fixture, invariances, and
central finite differences for the gradient.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

DTYPES = {"f32": 0, "bf16": 1, "f16": 2, "f64": 3}


def build(force: bool = False) -> str:
    """Compile liboracle.so in place (plain gcc, no OpenMP: single thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.oracle_mttkrp.argtypes = [i64, i32, vp, vp, vp, vp, vp, i32, i32, i32, vp]
        lib.oracle_mttkrp_rows.argtypes = [i64, i32, vp, vp, vp, vp, vp, i32, i32, i32, i64, vp, vp]
        lib.oracle_cp_sample.argtypes = [i64, i32, vp, vp, vp, i32, i32, vp]
        lib.oracle_cp_grad.argtypes = [i64, i32, vp, vp, vp, vp, i32, i32, vp]
        for f in (lib.oracle_mttkrp, lib.oracle_mttkrp_rows, lib.oracle_cp_sample, lib.oracle_cp_grad):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _storage(f: np.ndarray, dtype: str) -> np.ndarray:
    """Factor in its storage form: float32 / float64, or raw uint16 bits for bf16/f16."""
    if dtype in ("f32", "f64"):
        assert f.dtype == (np.float32 if dtype == "f32" else np.float64)
        return np.ascontiguousarray(f)
    assert f.dtype == np.uint16, "16-bit factors are passed as their raw uint16 bit patterns"
    return np.ascontiguousarray(f)


def _common(dims, idx, factors, dtype):
    dims_a = np.ascontiguousarray(np.asarray(dims, dtype=np.int64))
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    assert idx.ndim == 2 and idx.shape[1] == dims_a.shape[0]
    R = int(factors[0].shape[1]) if factors else 0
    fs = [_storage(f, dtype) for f in factors]
    fptrs = (ctypes.c_void_p * len(fs))(*[f.ctypes.data for f in fs])
    return dims_a, idx, fs, fptrs, R


def _rc(rc):
    if rc == -2:
        raise IndexError("oracle: coordinate out of range")
    if rc != 0:
        raise ValueError(f"oracle: invalid argument (rc={rc})")


def mttkrp(dims, idx, vals, factors, mode: int, dtype: str = "f32") -> np.ndarray:
    """Mode-`mode` MTTKRP in FP64.  vals float32 (or float64), factors list of
    [dims[n], R] arrays (float32, or uint16 bit patterns for bf16/f16)."""
    dims_a, idx, fs, fptrs, R = _common(dims, idx, factors, dtype)
    out = np.empty((int(dims_a[mode]), R), dtype=np.float64)
    vals = np.ascontiguousarray(vals)
    v32 = vals if vals.dtype == np.float32 else None
    v64 = np.ascontiguousarray(vals, dtype=np.float64) if v32 is None else None
    _rc(_L().oracle_mttkrp(idx.shape[0], len(dims_a), _ptr(dims_a), _ptr(idx), _ptr(v32), _ptr(v64), fptrs,
                           DTYPES[dtype], R, mode, _ptr(out)))
    return out


def mttkrp_rows(dims, idx, vals, factors, mode: int, rows, dtype: str = "f32") -> np.ndarray:
    """MTTKRP restricted to the (strictly increasing) output rows `rows`;
    vals float32 or float64."""
    dims_a, idx, fs, fptrs, R = _common(dims, idx, factors, dtype)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty((rows.shape[0], R), dtype=np.float64)
    vals = np.ascontiguousarray(vals)
    v32 = vals if vals.dtype == np.float32 else None
    v64 = np.ascontiguousarray(vals, dtype=np.float64) if v32 is None else None
    _rc(_L().oracle_mttkrp_rows(idx.shape[0], len(dims_a), _ptr(dims_a), _ptr(idx), _ptr(v32), _ptr(v64), fptrs,
                                DTYPES[dtype], R, mode, rows.shape[0], _ptr(rows), _ptr(out)))
    return out


def cp_sample(dims, idx, factors, dtype: str = "f32") -> np.ndarray:
    """m_k = sum_r prod_n A_n(i_n(k), r) for every nonzero k, FP64."""
    dims_a, idx, fs, fptrs, R = _common(dims, idx, factors, dtype)
    m = np.empty(idx.shape[0], dtype=np.float64)
    _rc(_L().oracle_cp_sample(idx.shape[0], len(dims_a), _ptr(dims_a), _ptr(idx), fptrs, DTYPES[dtype], R,
                              _ptr(m)))
    return m


def cp_grad(dims, idx, g, factors, dtype: str = "f32") -> list:
    """dL/dA_n for every mode n, given g_k = dL/dm_k (FP64)."""
    dims_a, idx, fs, fptrs, R = _common(dims, idx, factors, dtype)
    g = np.ascontiguousarray(g, dtype=np.float64)
    grads = [np.empty((int(d), R), dtype=np.float64) for d in dims_a]
    gp = (ctypes.c_void_p * len(grads))(*[a.ctypes.data for a in grads])
    _rc(_L().oracle_cp_grad(idx.shape[0], len(dims_a), _ptr(dims_a), _ptr(idx), _ptr(g), fptrs, DTYPES[dtype], R,
                            gp))
    return grads


def completion_loss(m: np.ndarray, x: np.ndarray) -> float:
    """L = 1/2 sum_k (m_k - x_k)^2 (no mean, no regulariser)."""
    d = np.asarray(m, dtype=np.float64) - np.asarray(x, dtype=np.float64)
    return 0.5 * float(np.dot(d, d))


def completion_grad(dims, idx, vals, factors, dtype: str = "f32"):
    """(loss, [dL/dA_n]) for the completion loss, all FP64."""
    m = cp_sample(dims, idx, factors, dtype)
    g = m - np.asarray(vals, dtype=np.float64)
    return completion_loss(m, vals), cp_grad(dims, idx, g, factors, dtype)


def row_error(gpu: np.ndarray, ref: np.ndarray, floor_frac: float = 0.0) -> float:
    """max_i ||g_i - o_i||_inf / ||o_i||_inf over rows with o_i != 0 (with
    floor_frac > 0 the denominator is max(||o_i||_inf, floor_frac * max_i ||o_i||_inf),
    for mixed-sign outputs).  Rows with o_i == 0 must match exactly; any
    difference there returns inf."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.size == 0:
        return 0.0
    num = np.abs(gpu - ref).max(axis=1)
    den = np.abs(ref).max(axis=1)
    if floor_frac > 0:
        den = np.maximum(den, floor_frac * den.max())
    zero = den == 0
    if np.any(num[zero] != 0):
        return float("inf")
    if np.all(zero):
        return 0.0
    return float((num[~zero] / den[~zero]).max())
