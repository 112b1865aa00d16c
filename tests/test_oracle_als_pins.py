"""Pins for the FP64 CP-ALS oracle (oracle/als.py), each against something
other than the oracle itself:

* every mode update is the least-squares solution of the unfolded problem,
  computed by numpy's lstsq on a dense unfolding with an explicit
  Khatri-Rao product (no normal equations, no Hadamard identity);
* the fit equals 1 - ||X - X^|| / ||X|| computed on dense arrays, with
  repeated coordinates summed into X;
* an exactly rank-R dense tensor started at its own factors is a fixed
  point: fit 1, factors unchanged up to column scaling;
* the dense residual never grows from one mode update to the next (each
  update is an exact least-squares step);
* a hand-worked fixture (tests/golden/tiny_als.txt): two mode-0 updates and
  the fit terms of the updated models, worked out by hand;
* planted mistakes in the oracle (the mode's own Gram in V, a matrix
  product for the Hadamard product, repeated coordinates not summed, lam left
  out of the model) each fail one of these.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import als


def densify(dims, idx, vals):
    X = np.zeros(dims)
    np.add.at(X, tuple(np.asarray(idx).T), np.asarray(vals, dtype=np.float64))
    return X


def unfold(X, d):
    """Mode-d unfolding, the remaining indices swept with the first one fastest."""
    return np.reshape(np.moveaxis(X, d, 0), (X.shape[d], -1), order="F")


def khatri_rao(mats):
    """Columnwise Kronecker product; the last matrix's row index runs fastest."""
    K = mats[0]
    for B in mats[1:]:
        K = (K[:, None, :] * B[None, :, :]).reshape(-1, K.shape[1])
    return K


def kr_others(A, d):
    """Khatri-Rao product matching unfold(): the other modes in decreasing order."""
    return khatri_rao([A[n] for n in reversed(range(len(A))) if n != d])


def dense_model(A, lam):
    N = len(A)
    letters = "abcdefgh"[:N]
    expr = "r," + ",".join(f"{c}r" for c in letters) + "->" + letters
    return np.einsum(expr, lam, *A)


def random_sparse(dims, nnz, seed, dup_frac=0.2):
    rng = np.random.default_rng(seed)
    idx = np.stack([rng.integers(0, d, nnz) for d in dims], axis=1).astype(np.int32)
    ndup = int(nnz * dup_frac)
    idx[nnz - ndup:] = idx[rng.integers(0, nnz - ndup, ndup)]  # repeated coordinates
    vals = rng.uniform(0.1, 1.0, nnz)
    return idx, vals


def ls_error(dims, idx, vals, A, d):
    """max relative difference between the oracle's mode-d update (scaled back
    by lam) and the dense least-squares solution."""
    X = densify(dims, idx, vals)
    K = kr_others(A, d)
    Bt, *_ = np.linalg.lstsq(K, unfold(X, d).T, rcond=None)
    An, lam = als.update_mode(dims, idx, vals, A, d)
    got = An * lam[None, :]
    return np.abs(got - Bt.T).max() / np.abs(Bt).max()


def fit_error(dims, idx, vals, A, lam):
    X = densify(dims, idx, vals)
    ref = 1.0 - np.linalg.norm(X - dense_model(A, lam)) / np.linalg.norm(X)
    return abs(als.fit(dims, idx, vals, A, lam) - ref)


CASES = [((6, 5, 4), 60, 3, 11), ((5, 4, 3, 3), 90, 2, 12), ((7, 6), 25, 3, 13), ((4, 3, 3, 2, 2), 80, 2, 14)]


@pytest.mark.parametrize("dims,nnz,R,seed", CASES)
def test_mode_update_is_the_least_squares_solution(dims, nnz, R, seed):
    idx, vals = random_sparse(dims, nnz, seed)
    rng = np.random.default_rng(seed + 100)
    A = [rng.uniform(0, 1, (d, R)) for d in dims]
    for d in range(len(dims)):
        assert ls_error(dims, idx, vals, A, d) < 1e-10


@pytest.mark.parametrize("dims,nnz,R,seed", CASES)
def test_fit_matches_the_dense_residual(dims, nnz, R, seed):
    idx, vals = random_sparse(dims, nnz, seed)
    rng = np.random.default_rng(seed + 200)
    A = [rng.uniform(0, 1, (d, R)) for d in dims]
    lam = rng.uniform(0.5, 2.0, R)
    assert fit_error(dims, idx, vals, A, lam) < 1e-12
    A2, lam2, f = als.sweep(dims, idx, vals, A)
    assert abs(f - (1.0 - np.linalg.norm(densify(dims, idx, vals) - dense_model(A2, lam2))
                    / np.linalg.norm(densify(dims, idx, vals)))) < 1e-10


def test_norm_sums_repeated_coordinates():
    idx = np.array([[0, 1, 2], [0, 1, 2], [1, 0, 0]], dtype=np.int32)
    vals = np.array([1.0, 2.0, 4.0])
    assert als.norm2(idx, vals) == 9.0 + 16.0  # (1 + 2)^2 + 4^2


@pytest.mark.parametrize("dims,R", [((6, 5, 4), 3), ((4, 3, 5, 2), 2)])
def test_exact_rank_tensor_is_a_fixed_point(dims, R):
    rng = np.random.default_rng(7)
    B = [rng.uniform(0.2, 1.0, (d, R)) for d in dims]
    X = dense_model(B, np.ones(R))
    idx = np.argwhere(np.ones(dims, dtype=bool)).astype(np.int32)  # every entry listed
    vals = X[tuple(idx.T)]
    A, lam, f = als.sweep(dims, idx, vals, B)
    assert f > 1 - 1e-6
    for n in range(len(dims)):
        ref = B[n] / np.linalg.norm(B[n], axis=0)
        np.testing.assert_allclose(A[n], ref, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(lam, np.prod([np.linalg.norm(b, axis=0) for b in B], axis=0), rtol=1e-9)


def test_dense_residual_never_grows_between_mode_updates():
    dims, R = (8, 7, 6), 3
    idx, vals = random_sparse(dims, 120, 21)
    X = densify(dims, idx, vals)
    rng = np.random.default_rng(22)
    A = [rng.uniform(0, 1, (d, R)) for d in dims]
    prev = np.inf
    for _ in range(4):
        for d in range(3):
            A[d], lam = als.update_mode(dims, idx, vals, A, d)
            res = np.linalg.norm(X - dense_model(A, lam))
            assert res <= prev * (1 + 1e-12)
            prev = res


def test_run_returns_one_fit_per_sweep():
    dims = (6, 5, 4)
    idx, vals = random_sparse(dims, 50, 31)
    A0 = [np.random.default_rng(32 + n).uniform(0, 1, (d, 2)) for n, d in enumerate(dims)]
    A, lam, fits = als.run(dims, idx, vals, A0, 3)
    assert len(fits) == 3 and np.all(np.diff(fits) >= -1e-12)
    assert all(a.dtype == np.float64 for a in A) and lam.shape == (2,)


# --- planted mistakes: each must be caught by a pin above -------------------------------

def _with(monkeypatch, name, fn):
    monkeypatch.setattr(als, name, fn)


def test_mutant_own_gram_in_v_is_caught(monkeypatch):
    dims, (idx, vals) = (6, 5, 4), random_sparse((6, 5, 4), 60, 41)
    A = [np.random.default_rng(42 + n).uniform(0, 1, (d, 3)) for n, d in enumerate(dims)]

    def bad(grams, d):
        V = np.ones_like(grams[0])
        for G in grams:
            V = V * G
        return V
    _with(monkeypatch, "hadamard_others", bad)
    assert ls_error(dims, idx, vals, A, 0) > 1e-3


def test_mutant_matrix_product_for_hadamard_is_caught(monkeypatch):
    dims, (idx, vals) = (6, 5, 4), random_sparse((6, 5, 4), 60, 43)
    A = [np.random.default_rng(44 + n).uniform(0, 1, (d, 3)) for n, d in enumerate(dims)]

    def bad(grams, d):
        V = np.eye(grams[0].shape[0])
        for n, G in enumerate(grams):
            if n != d:
                V = V @ G
        return V
    _with(monkeypatch, "hadamard_others", bad)
    assert ls_error(dims, idx, vals, A, 1) > 1e-3


def test_mutant_unsummed_duplicates_is_caught(monkeypatch):
    dims, (idx, vals) = (6, 5, 4), random_sparse((6, 5, 4), 60, 45, dup_frac=0.4)
    A = [np.random.default_rng(46 + n).uniform(0, 1, (d, 3)) for n, d in enumerate(dims)]
    _with(monkeypatch, "norm2", lambda idx, vals: float(np.dot(vals, vals)))
    assert fit_error(dims, idx, vals, A, np.ones(3)) > 1e-3


def test_mutant_model_without_lambda_is_caught(monkeypatch):
    dims, (idx, vals) = (6, 5, 4), random_sparse((6, 5, 4), 60, 47)
    A = [np.random.default_rng(48 + n).uniform(0, 1, (d, 3)) for n, d in enumerate(dims)]
    real = als.fit_terms
    _with(monkeypatch, "fit_terms", lambda dims, idx, vals, A, lam: real(dims, idx, vals, A, np.ones_like(lam)))
    assert fit_error(dims, idx, vals, A, np.array([0.5, 2.0, 1.5])) > 1e-3


def test_mttkrp_accepts_fp64_factors_exactly():
    dims = (5, 4, 3)
    idx, vals = random_sparse(dims, 30, 51)
    A = [np.random.default_rng(52 + n).uniform(0, 1, (d, 2)) for n, d in enumerate(dims)]
    got = oracle.mttkrp(dims, idx, vals, A, 0, "f64")
    ref = unfold(densify(dims, idx, vals), 0) @ kr_others(A, 0)
    np.testing.assert_allclose(got, ref, rtol=1e-13)


# --- hand-worked fixture ------------------------------------------------------------------

GOLDEN_ALS = os.path.join(os.path.dirname(__file__), "golden", "tiny_als.txt")


def load_golden_als():
    """{'dims', 'idx', 'vals', 'cases': {name: {'R', 'A1', 'A2', 'A0new', 'terms'}}}."""
    g = {"idx": [], "vals": [], "cases": {}}
    cur = None
    for line in open(GOLDEN_ALS):
        tok = line.split()
        if not tok or tok[0].startswith("#"):
            continue
        if tok[0] == "dims":
            g["dims"] = tuple(int(x) for x in tok[1:])
        elif tok[0] == "nz":
            g["idx"].append([int(x) for x in tok[1:-1]])
            g["vals"].append(float(tok[-1]))
        elif tok[0] == "case":
            cur = g["cases"].setdefault(tok[1], {"R": int(tok[2]), "A1": [], "A2": [], "A0new": []})
        elif tok[0] in ("A1", "A2", "A0new"):
            cur[tok[0]].append([float(x) for x in tok[1:]])
        elif tok[0] == "terms":
            cur["terms"] = [float(x) for x in tok[1:]]
    g["idx"] = np.array(g["idx"], dtype=np.int32)
    g["vals"] = np.array(g["vals"])
    return g


@pytest.mark.parametrize("case", ["r1", "r2"])
def test_golden_hand_worked_als(case):
    g = load_golden_als()
    c = g["cases"][case]
    R = c["R"]
    A1, A2, expect = np.array(c["A1"]), np.array(c["A2"]), np.array(c["A0new"])
    A0_start = np.ones((g["dims"][0], R))  # not read by the mode-0 update
    An, lam = als.update_mode(g["dims"], g["idx"], g["vals"], [A0_start, A1, A2], 0)
    np.testing.assert_allclose(An * lam[None, :], expect, atol=1e-12)
    xx, xy, yy = als.fit_terms(g["dims"], g["idx"], g["vals"], [expect, A1, A2], np.ones(R))
    np.testing.assert_allclose([xx, xy, yy, xx - 2 * xy + yy], c["terms"], rtol=1e-12)
