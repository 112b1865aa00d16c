"""Seeded synthetic sparse tensors for the MTTKRP tests and benchmark.

This package only draws random inputs (coordinates, values, dense factors);
it contains none of the MTTKRP / CP arithmetic, so the CPU oracle and the GPU
library can both be fed from it without sharing any code.  The random source
is a counter-based SplitMix64 stream and Zipf draws use rejection-inversion
(see ``synth.c``); results are identical for any thread count and on x86-64
and aarch64.

Workload recipes (``WORKLOADS``) restate the synthetic stand-ins for the
paper's billion-scale FROSTT/Twitch tensors (Sec. 5.1, Table 3): power-law
(Zipf over a random permutation of each mode's range) coordinates with FP32
values, plus a small uniform parity case and a planted-CP completion case.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

# stream ids (one independent counter stream per purpose)
_S_INDEX, _S_PERM, _S_VALUES, _S_FACTOR, _S_NOISE, _S_PLANTED, _S_SHUFFLE, _S_SUBSET = (
    100, 200, 300, 400, 500, 600, 700, 800)


def build(force: bool = False) -> str:
    """Compile libsynth.so in place (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, i64, vp = ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p
        lib.synth_permutation.argtypes = [u64, u64, i64, vp]
        lib.synth_index_uniform.argtypes = [u64, u64, i64, i64, vp, i64]
        lib.synth_index_zipf.argtypes = [u64, u64, i64, i64, ctypes.c_double, vp, vp, i64]
        lib.synth_values.argtypes = [u64, u64, i64, ctypes.c_int, ctypes.c_double, ctypes.c_double, vp]
        lib.synth_u64.argtypes = [u64, u64]
        lib.synth_u64.restype = u64
        lib.synth_key.argtypes = [u64, u64]
        lib.synth_key.restype = u64
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def permutation(n: int, seed: int, stream: int = _S_PERM) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    _L().synth_permutation(seed, stream, n, _p(out))
    return out


def values(n: int, seed: int, kind: str = "uniform", a: float = 0.0, b: float = 1.0,
           stream: int = _S_VALUES) -> np.ndarray:
    """kind 'uniform' U(a,b); 'lognormal' exp(N(a, b^2)); 'normal' N(a, b^2)."""
    code = {"uniform": 0, "lognormal": 1, "normal": 2}[kind]
    out = np.empty(n, dtype=np.float32)
    _L().synth_values(seed, stream, n, code, a, b, _p(out))
    return out


@dataclass
class Workload:
    """One synthetic tensor recipe."""
    name: str
    dims: tuple
    nnz: int
    index_dist: tuple  # per mode: ("uniform",) or ("zipf", s)
    values: tuple = ("uniform", 0.0, 1.0)
    rank: int = 32
    seed: int = 20250715
    merge_duplicates: bool = False
    planted_rank: int = 0        # >0: values come from a planted CP model plus noise
    noise_sd: float = 0.0
    factor_scale: float = 1.0    # factors U(0, factor_scale)
    note: str = ""

    def scaled(self, f: float) -> "Workload":
        """Same recipe with nnz and every dimension scaled by f (each at least 1)."""
        if f == 1.0:
            return self
        dims = tuple(max(1, int(round(d * f))) for d in self.dims)
        return Workload(self.name + f"@{f:g}", dims, max(0, int(round(self.nnz * f))), self.index_dist,
                        self.values, self.rank, self.seed, self.merge_duplicates, self.planted_rank,
                        self.noise_sd, self.factor_scale, self.note)


WORKLOADS = {
    "uniform3": Workload("uniform3", (1000, 800, 600), 100_000, (("uniform",),) * 3, rank=16,
                         seed=20250715 + 1, merge_duplicates=True,
                         note="3-mode uniform, duplicates merged by sum"),
    "zipf3": Workload("zipf3", (10_000_000, 5_000_000, 2_000_000), 200_000_000, (("zipf", 1.1),) * 3,
                      rank=32, seed=20250715 + 2, note="3-mode power-law, Zipf(1.1) over a permutation"),
    "zipf4": Workload("zipf4", (50_000_000, 20_000_000, 5_000_000, 1000), 1_000_000_000,
                      (("zipf", 1.2), ("zipf", 1.2), ("zipf", 1.2), ("uniform",)),
                      values=("lognormal", 0.0, 1.0), rank=32, seed=20250715 + 3,
                      note="4-mode billion-scale, modes 0-2 Zipf(1.2), mode 3 uniform, lognormal values"),
    "zipf3_r64": Workload("zipf3_r64", (10_000_000, 5_000_000, 2_000_000), 200_000_000,
                          (("zipf", 1.1),) * 3, rank=64, seed=20250715 + 2,
                          note="same tensor as zipf3 at R=64 for 16-bit factor storage"),
    "zipf5": Workload("zipf5", (15_500_000, 6_200_000, 784_000, 6_100, 6_100), 500_000_000,
                      (("zipf", 1.1),) * 5, rank=32, seed=20250715 + 6,
                      note="5-mode power-law with the shape of the paper's Twitch tensor (Table 3)"),
    "planted3": Workload("planted3", (5_000_000, 2_000_000, 1_000_000), 100_000_000, (("zipf", 1.1),) * 3,
                         rank=32, seed=20250715 + 5, planted_rank=16, noise_sd=0.01, factor_scale=0.5,
                         note="completion: planted rank-16 CP values plus N(0, 0.01^2) noise"),
}


@dataclass
class Coo:
    dims: tuple
    idx: np.ndarray   # int32 [nnz, N], 0-based
    vals: np.ndarray  # float32 [nnz]
    extra: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.idx.shape[0])

    @property
    def nmodes(self) -> int:
        return len(self.dims)


def coordinates(dims, nnz: int, index_dist, seed: int) -> np.ndarray:
    """int32 [nnz, N] coordinates; each mode drawn from its own stream."""
    N = len(dims)
    idx = np.empty((nnz, N), dtype=np.int32)
    lib = _L()
    for n, (d, dist) in enumerate(zip(dims, index_dist)):
        col = idx[:, n:]  # view starting at column n; stride N
        if nnz == 0:
            continue
        if dist[0] == "uniform":
            lib.synth_index_uniform(seed, _S_INDEX + n, nnz, d, _p(col), N)
        elif dist[0] == "zipf":
            perm = permutation(d, seed, _S_PERM + n)
            lib.synth_index_zipf(seed, _S_INDEX + n, nnz, d, float(dist[1]), _p(perm), _p(col), N)
        else:
            raise ValueError(dist)
    return idx


def factors(dims, rank: int, seed: int, scale: float = 1.0, stream: int = _S_FACTOR) -> list:
    """Dense factors A_n, float32 [dims[n], rank], entries U(0, scale)."""
    return [values(int(d) * rank, seed, "uniform", 0.0, scale, stream + n).reshape(int(d), rank)
            for n, d in enumerate(dims)]


def make(w: Workload, with_values: bool = True) -> Coo:
    """Draw the tensor of a recipe.  For planted recipes the values are NOT
    filled in here (computing a CP model is the method's arithmetic); the
    planted factors and the noise are returned in ``extra`` instead, and
    ``vals`` holds the noise only."""
    idx = coordinates(w.dims, w.nnz, w.index_dist, w.seed)
    if w.planted_rank:
        vals = values(w.nnz, w.seed, "normal", 0.0, w.noise_sd, _S_NOISE)
        planted = factors(w.dims, w.planted_rank, w.seed, 1.0, _S_PLANTED)
        return Coo(w.dims, idx, vals, {"planted_factors": planted, "noise": vals.copy()})
    kind, a, b = w.values
    vals = values(w.nnz, w.seed, kind, a, b, _S_VALUES) if with_values else np.zeros(w.nnz, np.float32)
    if w.merge_duplicates and w.nnz:
        idx, vals = merge_duplicates(w.dims, idx, vals, w.seed)
    return Coo(w.dims, idx, vals)


def merge_duplicates(dims, idx: np.ndarray, vals: np.ndarray, seed: int):
    """Sum the values of repeated coordinates (COO semantics), then shuffle
    the merged nonzeros with a seeded permutation so the order stays random."""
    key = np.zeros(idx.shape[0], dtype=np.int64)
    for n, d in enumerate(dims):
        key = key * int(d) + idx[:, n].astype(np.int64)
    uk, inv = np.unique(key, return_inverse=True)
    merged = np.zeros(uk.shape[0], dtype=np.float64)
    np.add.at(merged, inv, vals.astype(np.float64))
    out = np.empty((uk.shape[0], len(dims)), dtype=np.int32)
    rem = uk.copy()
    for n in range(len(dims) - 1, -1, -1):
        out[:, n] = (rem % int(dims[n])).astype(np.int32)
        rem //= int(dims[n])
    p = permutation(uk.shape[0], seed, _S_SHUFFLE)
    return np.ascontiguousarray(out[p]), merged.astype(np.float32)[p]


def subset(n: int, k: int, seed: int, stream: int = _S_SUBSET) -> np.ndarray:
    """k distinct indices of [0, n), sorted (seeded)."""
    k = min(int(k), int(n))
    if k == 0:
        return np.zeros(0, dtype=np.int64)
    draws = np.empty(4 * k + 64, dtype=np.int32)
    _L().synth_index_uniform(seed, stream, draws.shape[0], n, _p(draws), 1)
    _, first = np.unique(draws, return_index=True)
    picked = draws[np.sort(first)][:k]
    if picked.shape[0] < k:  # tiny n: fall back to a seeded permutation
        picked = permutation(n, seed, stream)[:k]
    return np.sort(picked.astype(np.int64))
