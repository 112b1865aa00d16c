"""Python face of the library: a sparse tensor handle with MTTKRP, the
sampled CP model and its gradient.  PyTorch provides device memory and
streams only; the work is done by the CUDA library behind the C ABI.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _lib

try:
    import torch
except ImportError:  # the planning query works without torch
    torch = None

# amped_opts.inner_order codes: the order of the nonzeros inside an output row
INNER_ORDERS = {
    "stable": 1,                     # caller order
    "lexicographic": 2,              # other coordinates, largest dimension most significant
    "lexicographic_ascending": 3,    # other coordinates, smallest dimension most significant
}


def _dtype_code(t) -> int:
    if t.dtype == torch.float32:
        return _lib.F32
    if t.dtype == torch.bfloat16:
        return _lib.BF16
    if t.dtype == torch.float16:
        return _lib.F16
    raise TypeError(f"factor dtype {t.dtype} is not one of float32, bfloat16, float16")


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Tensor:
    """An N-mode sparse COO tensor resident on the current CUDA device.

    ``idx`` is int32 [nnz, N] (0-based), ``vals`` float32 [nnz]; both host
    arrays (numpy or CPU torch).  Construction builds one output-row-ordered,
    segmented copy per mode (paper Sec. 3); it is synchronous.  With
    ``stream_memory="host"`` the per-nonzero streams of the copies stay in
    pinned host memory and the kernels read them over the host link
    (out-of-core); factors, outputs and row tables are always on the device.
    """

    def __init__(self, dims, idx, vals, *, segment_items: int = 0, keep_perm: bool = True, keep_coo: bool = True,
                 max_rank: int = 0, host_threads: int = 0, inner_order: str = "lexicographic",
                 short_rows: int = 0, stream_memory: str = "device"):
        L = _lib.lib()
        self.dims = tuple(int(d) for d in dims)
        idx = np.ascontiguousarray(idx.numpy() if hasattr(idx, "numpy") else idx, dtype=np.int32)
        vals = np.ascontiguousarray(vals.numpy() if hasattr(vals, "numpy") else vals, dtype=np.float32)
        if idx.ndim != 2 or idx.shape[1] != len(self.dims) or vals.shape != (idx.shape[0],):
            raise ValueError("idx must be [nnz, N] and vals [nnz]")
        self.nnz = int(idx.shape[0])
        dims_a = np.asarray(self.dims, dtype=np.int64)
        if inner_order not in INNER_ORDERS:
            raise ValueError(f"inner_order must be one of {sorted(INNER_ORDERS)}")
        if stream_memory not in ("device", "host"):
            raise ValueError("stream_memory must be 'device' or 'host'")
        opts = _lib.Opts(segment_items, 1 if keep_perm else 2, 1 if keep_coo else 2, max_rank, host_threads,
                         INNER_ORDERS[inner_order], short_rows, 2 if stream_memory == "host" else 1)
        h = ctypes.c_void_p()
        _lib.check(L.amped_tensor_create(self.nnz, len(self.dims), dims_a.ctypes.data,
                                         idx.ctypes.data if self.nnz else None,
                                         vals.ctypes.data if self.nnz else None, ctypes.byref(opts),
                                         ctypes.byref(h)))
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device()) if torch is not None else None

    # ------------------------------------------------------------------ lifetime
    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib.lib().amped_tensor_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def nmodes(self) -> int:
        return len(self.dims)

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise ValueError("tensor handle is closed")
        return self._h

    # ------------------------------------------------------------------ helpers
    def _factors(self, factors, skip=-1):
        if len(factors) != self.nmodes:
            raise ValueError(f"need {self.nmodes} factors")
        ref = next(f for n, f in enumerate(factors) if n != skip and f is not None)
        R = int(ref.shape[1])
        code = _dtype_code(ref)
        ptrs = []
        for n, f in enumerate(factors):
            if n == skip and f is None:
                ptrs.append(None)
                continue
            if f.dtype != ref.dtype or not f.is_cuda or not f.is_contiguous() or tuple(f.shape) != (self.dims[n], R):
                raise ValueError(f"factor {n} must be a contiguous CUDA [{self.dims[n]}, {R}] {ref.dtype} tensor")
            ptrs.append(f.data_ptr())
        return _lib.ptr_array(ptrs), code, R

    def _out(self, n, R, out):
        if out is None:
            return torch.empty((self.dims[n], R), dtype=torch.float32, device=self.device)
        if out.dtype != torch.float32 or not out.is_contiguous() or tuple(out.shape) != (self.dims[n], R):
            raise ValueError(f"output {n} must be a contiguous float32 [{self.dims[n]}, {R}] tensor")
        return out

    # ------------------------------------------------------------------ operations
    def mttkrp(self, mode: int, factors, out=None, stream=None):
        """Mode-`mode` MTTKRP: out[i] = sum over nonzeros with i_mode = i of
        val * Hadamard product of the other factors' rows (fp32 result)."""
        fp, code, R = self._factors(factors, skip=mode)
        out = self._out(mode, R, out)
        _lib.check(_lib.lib().amped_mttkrp(self.handle, mode, fp, code, R, out.data_ptr(), _stream_ptr(stream)))
        return out

    def mttkrp_all(self, factors, outs=None, stream=None):
        """MTTKRP for every mode with the same input factors."""
        fp, code, R = self._factors(factors)
        outs = [self._out(n, R, None if outs is None else outs[n]) for n in range(self.nmodes)]
        op = _lib.ptr_array([o.data_ptr() for o in outs])
        _lib.check(_lib.lib().amped_mttkrp_all(self.handle, fp, code, R, op, _stream_ptr(stream)))
        return outs

    def mttkrp_all_host(self, factors, outs=None, stream=None):
        """All-mode MTTKRP on host (CPU) tensors: the library copies the factors
        in, runs every mode and copies the outputs back before returning."""
        if len(factors) != self.nmodes:
            raise ValueError(f"need {self.nmodes} factors")
        R = int(factors[0].shape[1])
        code = _dtype_code(factors[0])
        for n, f in enumerate(factors):
            if f.is_cuda or not f.is_contiguous() or tuple(f.shape) != (self.dims[n], R) or f.dtype != factors[0].dtype:
                raise ValueError(f"host factor {n} must be a contiguous CPU [{self.dims[n]}, {R}] tensor")
        if outs is None:
            outs = [torch.empty((d, R), dtype=torch.float32) for d in self.dims]
        for n, o in enumerate(outs):
            if o.is_cuda or o.dtype != torch.float32 or not o.is_contiguous() or tuple(o.shape) != (self.dims[n], R):
                raise ValueError(f"host output {n} must be a contiguous CPU float32 [{self.dims[n]}, {R}] tensor")
        fp = _lib.ptr_array([f.data_ptr() for f in factors])
        op = _lib.ptr_array([o.data_ptr() for o in outs])
        _lib.check(_lib.lib().amped_mttkrp_all_host(self.handle, fp, code, R, op, _stream_ptr(stream)))
        return outs

    def cp_sample(self, factors, out=None, stream=None):
        """Sampled CP model m[k] = sum_r prod_n A_n(i_n(k), r), caller order."""
        fp, code, R = self._factors(factors)
        if out is None:
            out = torch.empty(self.nnz, dtype=torch.float32, device=self.device)
        _lib.check(_lib.lib().amped_cp_sample(self.handle, fp, code, R, out.data_ptr() if self.nnz else None,
                                              _stream_ptr(stream)))
        return out

    def cp_grad(self, factors, gvals, grads=None, stream=None):
        """d L / d A_n for every n given gvals[k] = dL/dm_k (caller order)."""
        fp, code, R = self._factors(factors)
        if gvals.dtype != torch.float32 or not gvals.is_cuda or gvals.numel() != self.nnz:
            raise ValueError("gvals must be a float32 CUDA tensor with one entry per nonzero")
        gvals = gvals.contiguous()
        grads = [self._out(n, R, None if grads is None else grads[n]) for n in range(self.nmodes)]
        gp = _lib.ptr_array([g.data_ptr() for g in grads])
        _lib.check(_lib.lib().amped_cp_grad(self.handle, fp, code, R, gvals.data_ptr() if self.nnz else None, gp,
                                            _stream_ptr(stream)))
        return grads

    def completion_grad(self, factors, grads=None, loss=None, stream=None):
        """Fused gradient of L = 1/2 sum_k (m_k - x_k)^2 over the tensor's own values x:
        returns (grads, loss) with loss a 0-dim float64 CUDA tensor."""
        fp, code, R = self._factors(factors)
        grads = [self._out(n, R, None if grads is None else grads[n]) for n in range(self.nmodes)]
        if loss is None:
            loss = torch.empty((), dtype=torch.float64, device=self.device)
        gp = _lib.ptr_array([g.data_ptr() for g in grads])
        _lib.check(_lib.lib().amped_cp_completion_grad(self.handle, fp, code, R, gp, loss.data_ptr(),
                                                       _stream_ptr(stream)))
        return grads, loss

    def norm2(self) -> float:
        """||X||^2 of the tensor, repeated coordinates summed into one entry."""
        v = ctypes.c_double()
        _lib.check(_lib.lib().amped_tensor_norm2(self.handle, ctypes.byref(v)))
        return v.value

    def _als_buffers(self, factors, grams, stats=None):
        fp, code, R = self._factors(factors)
        if code != _lib.F32:
            raise ValueError("CP-ALS keeps fp32 factors")
        for name, t, dt, shape in (("grams", grams, torch.float64, (self.nmodes, R, R)),
                                   ("stats", stats, torch.float64, (8,))):
            if t is None:
                continue
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != shape:
                raise ValueError(f"{name} must be a contiguous CUDA {dt} tensor of shape {shape}")
        return fp, R

    def cp_als_sweep(self, factors, grams, stats, init: bool = False, stream=None) -> None:
        """One CP-ALS sweep over modes 0..N-1: each fp32 factor is replaced by
        the least-squares update after its MTTKRP (columns not normalised).
        Updates `grams` [N, R, R] fp64 (the factors' Grams) and `stats` [8]
        fp64 in place (fit, residual^2, ||X||^2, <X, X^>, ||X^||^2, singular
        solves, first singular mode + 1).  init=True computes `grams` from the
        factors first."""
        fp, R = self._als_buffers(factors, grams, stats)
        _lib.check(_lib.lib().amped_cp_als_sweep(self.handle, fp, R, grams.data_ptr(), stats.data_ptr(),
                                                 _lib.ALS_INIT if init else 0, _stream_ptr(stream)))

    def cp_als_update(self, mode: int, factors, grams, stats, init: bool = False, stream=None) -> None:
        """One CP-ALS mode update: factors[mode] becomes the unnormalised
        least-squares update after the mode-`mode` MTTKRP; grams[mode] its
        Gram; stats the fit terms of the resulting model."""
        fp, R = self._als_buffers(factors, grams, stats)
        _lib.check(_lib.lib().amped_cp_als_update(self.handle, int(mode), fp, R, grams.data_ptr(), stats.data_ptr(),
                                                  _lib.ALS_INIT if init else 0, _stream_ptr(stream)))

    def cp_als_normalize(self, factors, grams, lam=None, stream=None):
        """Scale every factor's columns to unit norm in place; returns lambda
        (the products of the norms) and rescales `grams`."""
        fp, R = self._als_buffers(factors, grams)
        if lam is None:
            lam = torch.empty(R, dtype=torch.float32, device=self.device)
        _lib.check(_lib.lib().amped_cp_als_normalize(self.handle, fp, R, grams.data_ptr(), lam.data_ptr(),
                                                     _stream_ptr(stream)))
        return lam

    def cp_als(self, factors, sweeps: int = 25, tol: float = 1e-5, stream=None):
        """CP decomposition by alternating least squares, starting from the
        given fp32 factors (updated in place, unit-norm columns on return).
        Stops after `sweeps` sweeps or when the fit changes by less than
        `tol`.  Returns (lambda, fits)."""
        R = int(factors[0].shape[1])
        grams = torch.empty((self.nmodes, R, R), dtype=torch.float64, device=self.device)
        stats = torch.zeros(8, dtype=torch.float64, device=self.device)
        fits = []
        for s in range(sweeps):
            self.cp_als_sweep(factors, grams, stats, init=(s == 0), stream=stream)
            if stream is not None:
                stream.synchronize()
            st = stats.cpu()
            if st[5] > 0:
                raise _lib.AmpedError(_lib.ERR_INVALID, f"CP-ALS: the normal equations of mode {int(st[6]) - 1} "
                                      "are singular (a factor lost column rank)")
            fits.append(float(st[0]))
            if s > 0 and abs(fits[-1] - fits[-2]) < tol:
                break
        return self.cp_als_normalize(factors, grams, stream=stream), fits

    def set_kernel_events(self, start, stop) -> None:
        """Record torch.cuda.Event `start`/`stop` around the next MTTKRP kernel."""
        for ev in (start, stop):
            if ev is not None and not ev.cuda_event:
                ev.record()  # events are created lazily by torch
        _lib.check(_lib.lib().amped_set_kernel_events(self.handle, start.cuda_event if start else None,
                                                      stop.cuda_event if stop else None))


def plan_mode(dims, idx, mode: int, segment_items: int = 0, inner_order: str = "lexicographic",
              short_rows: int = 0) -> dict:
    """Host-only: the reorder, row classes and segment tables for one mode."""
    L = _lib.lib()
    dims_a = np.asarray(dims, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    nnz = int(idx.shape[0])
    io = INNER_ORDERS[inner_order]
    args = (nnz, len(dims_a), dims_a.ctypes.data, idx.ctypes.data if nnz else None, mode, segment_items, io,
            short_rows)
    sz = _lib.PlanSizes()
    _lib.check(L.amped_plan_mode(*args, ctypes.byref(sz), *([None] * 9)))
    out = {
        "perm": np.empty(nnz, np.int32),
        "rows_long": np.empty(sz.long_rows, np.int32),
        "rowptr_long": np.empty(sz.long_rows + 1, np.int32),
        "seg_row": np.empty(sz.long_segments + 1, np.int32),
        "seg_nz": np.empty(sz.long_segments + 1, np.int32),
        "splits": np.empty((max(sz.split_rows, 1), 3), np.int32),
        "rows_short": np.empty(sz.short_rows, np.int32),
        "rowptr_short": np.empty(sz.short_rows + 1, np.int32),
        "seg_short": np.empty(sz.short_segments + 1, np.int32),
    }
    ptrs = [a.ctypes.data if a.size else None for a in out.values()]
    _lib.check(L.amped_plan_mode(*args, ctypes.byref(sz), *ptrs))
    out["splits"] = out["splits"][: sz.split_rows]
    out["sizes"] = {f: getattr(sz, f) for f, _ in _lib.PlanSizes._fields_}
    out["items"] = segment_items if segment_items > 0 else 1024
    return out
