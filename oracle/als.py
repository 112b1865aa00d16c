"""FP64 CPU oracle for CP decomposition by alternating least squares.

TEST INFRASTRUCTURE ONLY: the same callers as the rest of this package (the
tests, the smoke check and the benchmark's CPU legs).  The GPU library never
imports it.

Sec. 2.1 computes the CPD by ALS, performing the mode-wise MTTKRPs of Eq. 1
in turn and iterating.  The paper stops at the MTTKRP; the factor update that
follows it is the least-squares solve of CP-ALS (Kolda & Bader, "Tensor
Decompositions and Applications", SIAM Review 2009, Sec. 3.4), written here
step by step:

  for d = 0 .. N-1 (each step sees the factors updated before it):
    M   = MTTKRP_d(X; A_n, n != d)                  (Sec. 3 elementwise form)
    V   = Hadamard product over n != d of A_n^T A_n  (R x R)
    B   = M V^+                                      (pseudo-inverse)
    lam = 2-norms of the columns of B;  A_d = B with its columns scaled to unit
          norm (a zero column stays zero and gets lam = 0)
  model  X^ = sum_r lam_r a_r^(0) o ... o a_r^(N-1)   (lam from the last update)
  fit    = 1 - ||X - X^|| / ||X||

X is the sparse tensor: zero at every coordinate that is not listed, and
repeated coordinates in the list add up into one entry.  ||X - X^||^2 is
expanded as ||X||^2 - 2<X, X^> + ||X^||^2 with <X, X^> = sum_k x_k X^(i_k)
over the listed nonzeros and ||X^||^2 = lam^T (Hadamard of all A_n^T A_n) lam.

Library primitives used as steps: numpy matmul, pinv, unique and bincount;
the MTTKRP and the sampled model are the C oracle's loops, with fp64 factors.
"""
from __future__ import annotations

import numpy as np

from . import cp_sample, mttkrp


def gram(A: np.ndarray) -> np.ndarray:
    """A^T A in fp64."""
    A = np.asarray(A, dtype=np.float64)
    return A.T @ A


def hadamard_others(grams, d: int) -> np.ndarray:
    """Elementwise product of the Gram matrices of every mode except d."""
    V = np.ones_like(grams[0])
    for n, G in enumerate(grams):
        if n != d:
            V = V * G
    return V


def normalize_columns(B: np.ndarray):
    """(B with unit-norm columns, the column norms); zero columns stay zero."""
    lam = np.sqrt((B * B).sum(axis=0))
    return B / np.where(lam > 0, lam, 1.0), lam


def update_mode(dims, idx, vals, A, d: int):
    """Least-squares update of factor d with the other factors fixed.
    Returns (normalised A_d, lam)."""
    M = mttkrp(dims, idx, vals, A, d, "f64")
    V = hadamard_others([gram(a) for a in A], d)
    return normalize_columns(M @ np.linalg.pinv(V))


def norm2(idx, vals) -> float:
    """||X||^2 of the sparse tensor, repeated coordinates summed first."""
    idx = np.asarray(idx)
    vals = np.asarray(vals, dtype=np.float64)
    if vals.size == 0:
        return 0.0
    _, inv = np.unique(idx, axis=0, return_inverse=True)
    s = np.bincount(inv.ravel(), weights=vals)
    return float(np.dot(s, s))


def fit_terms(dims, idx, vals, A, lam):
    """(||X||^2, <X, X^>, ||X^||^2) for the model [[lam; A_0, ..., A_{N-1}]]."""
    A = [np.asarray(a, dtype=np.float64) for a in A]
    lam = np.asarray(lam, dtype=np.float64)
    xx = norm2(idx, vals)
    scaled = [A[0] * lam[None, :]] + A[1:]
    xy = float(np.dot(np.asarray(vals, dtype=np.float64), cp_sample(dims, idx, scaled, "f64")))
    W = np.outer(lam, lam)
    for a in A:
        W = W * gram(a)
    return xx, xy, float(W.sum())


def fit(dims, idx, vals, A, lam) -> float:
    """1 - ||X - X^|| / ||X|| (the squared residual is clamped at 0)."""
    xx, xy, yy = fit_terms(dims, idx, vals, A, lam)
    return 1.0 - np.sqrt(max(xx - 2.0 * xy + yy, 0.0)) / np.sqrt(xx)


def sweep(dims, idx, vals, factors):
    """One ALS sweep over modes 0..N-1 from `factors` (copied, fp64).
    Returns (factors, lam, fit)."""
    A = [np.array(f, dtype=np.float64) for f in factors]
    lam = None
    for d in range(len(dims)):
        A[d], lam = update_mode(dims, idx, vals, A, d)
    return A, lam, fit(dims, idx, vals, A, lam)


def run(dims, idx, vals, factors, sweeps: int):
    """`sweeps` ALS sweeps; returns (factors, lam, [fit after each sweep])."""
    A, lam, fits = list(factors), None, []
    for _ in range(sweeps):
        A, lam, f = sweep(dims, idx, vals, A)
        fits.append(f)
    return A, lam, fits
