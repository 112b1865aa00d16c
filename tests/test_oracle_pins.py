"""Pins for the FP64 oracle: what the paper and the mathematics fix, checked
without trusting the oracle's own formula.

* brute force: densify, unfold (Kolda-Bader: first remaining index fastest),
  explicit Khatri-Rao product, matrix product -- Sec. 2.1 Eq. 1;
* closed form for an exact dense CP tensor X = [[B_0..B_{N-1}]]:
  X_(m) (KR of A_n, n != m) = B_m (Hadamard over n != m of B_n^T A_n);
* N = 2 reduces to a sparse-times-dense matrix product (scipy.sparse);
* a hand-worked fixture (tests/golden/tiny_mttkrp.txt);
* invariances: nonzero order, duplicate splitting, linearity, empty rows;
* the sampled CP model against a dense CP tensor read at the coordinates;
* the gradient against central finite differences in FP64;
* plausible mistakes (mutants, written here in Python) each fail a pin.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_mttkrp.txt")


# ----------------------------------------------------------------------------- helpers
def rand_coo(dims, nnz, seed, dup_frac=0.2, signed=False):
    rng = np.random.default_rng(seed)
    idx = np.stack([rng.integers(0, d, nnz) for d in dims], axis=1).astype(np.int32)
    ndup = int(nnz * dup_frac)
    if ndup:
        idx[-ndup:] = idx[rng.integers(0, nnz - ndup, ndup)]
    vals = rng.uniform(-1 if signed else 0, 1, nnz).astype(np.float32)
    return idx, vals


def rand_factors(dims, R, seed, signed=False):
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1 if signed else 0, 1, (d, R)).astype(np.float32) for d in dims]


def densify(dims, idx, vals):
    X = np.zeros(dims, dtype=np.float64)
    np.add.at(X, tuple(idx[:, n] for n in range(len(dims))), vals.astype(np.float64))
    return X


def unfold(X, n):
    """Mode-n unfolding, columns ordered with the first remaining index fastest."""
    return np.reshape(np.moveaxis(X, n, 0), (X.shape[n], -1), order="F")


def khatri_rao(mats):
    """Column-wise Kronecker product; the LAST matrix's row index varies fastest."""
    R = mats[0].shape[1]
    cols = []
    for r in range(R):
        v = np.ones(1)
        for M in mats:
            v = np.kron(v, M[:, r].astype(np.float64))
        cols.append(v)
    return np.stack(cols, axis=1)


def brute_mttkrp(dims, idx, vals, factors, m):
    X = densify(dims, idx, vals)
    rest = [n for n in range(len(dims)) if n != m]
    # unfolding has rest[0] fastest, so the Khatri-Rao product lists rest in reverse
    KR = khatri_rao([factors[n] for n in reversed(rest)])
    return unfold(X, m) @ KR


def load_golden():
    d = {"nz": [], "model": None}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        key, *rest = line.split()
        if key == "nz":
            d["nz"].append([float(x) for x in rest])
        elif key in ("dims", "rank"):
            d[key] = [int(x) for x in rest]
        elif key in ("model", "loss"):
            d[key] = [float(x) for x in rest]
        else:
            d.setdefault(key, []).append([float(x) for x in rest])
    nz = np.array(d["nz"])
    d["idx"] = nz[:, :3].astype(np.int32)
    d["vals"] = nz[:, 3].astype(np.float32)
    return d


# ----------------------------------------------------------------------------- pins
PIN_CASES = [((6, 5, 4), 40, 3), ((5, 4, 3, 3), 50, 4), ((7, 1, 3), 12, 2), ((4, 6), 15, 5)]


@pytest.mark.parametrize("dims,nnz,R", PIN_CASES)
def test_brute_force_unfold_khatri_rao(dims, nnz, R):
    idx, vals = rand_coo(dims, nnz, seed=sum(dims) + nnz, signed=True)
    F = rand_factors(dims, R, seed=nnz, signed=True)
    for m in range(len(dims)):
        ref = brute_mttkrp(dims, idx, vals, F, m)
        got = oracle.mttkrp(dims, idx, vals, F, m)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_golden_hand_worked():
    g = load_golden()
    F = [np.array(g[k], dtype=np.float32) for k in ("A0", "A1", "A2")]
    for m in range(3):
        got = oracle.mttkrp(g["dims"], g["idx"], g["vals"], F, m)
        np.testing.assert_array_equal(got, np.array(g[f"M{m}"]))
    model = oracle.cp_sample(g["dims"], g["idx"], F)
    np.testing.assert_array_equal(model, np.array(g["model"]))
    loss, grads = oracle.completion_grad(g["dims"], g["idx"], g["vals"], F)
    assert loss == g["loss"][0]
    np.testing.assert_array_equal(grads[0], np.array(g["G0"]))


@pytest.mark.parametrize("dims,RB,RA", [((4, 3, 5), 2, 3), ((3, 4, 2, 3), 3, 2)])
def test_closed_form_exact_cp_tensor(dims, RB, RA):
    """All entries of X = [[B_0..B_{N-1}]] stored as COO; the MTTKRP must equal
    B_m * (Hadamard over n != m of B_n^T A_n) (multilinearity of the CP model)."""
    B = rand_factors(dims, RB, seed=11, signed=True)
    A = rand_factors(dims, RA, seed=12, signed=True)
    coords = np.array(list(itertools.product(*[range(d) for d in dims])), dtype=np.int32)
    # entry values: sum_r prod_n B_n(i_n, r), evaluated with numpy einsum (not the oracle)
    letters = "abcdefgh"[: len(dims)]
    X = np.einsum(",".join(f"{l}z" for l in letters) + "->" + letters, *[b.astype(np.float64) for b in B])
    vals = X[tuple(coords[:, n] for n in range(len(dims)))]
    for m in range(len(dims)):
        V = np.ones((RB, RA))
        for n in range(len(dims)):
            if n != m:
                V *= B[n].astype(np.float64).T @ A[n].astype(np.float64)
        ref = B[m].astype(np.float64) @ V
        got = oracle.mttkrp(dims, coords, vals, A, m)  # float64 values path
        np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11)
    # with A = B this is the form A_m (Hadamard of A_n^T A_n)
    got = oracle.mttkrp(dims, coords, vals, B, 0)
    V = np.ones((RB, RB))
    for n in range(1, len(dims)):
        V *= B[n].astype(np.float64).T @ B[n].astype(np.float64)
    np.testing.assert_allclose(got, B[0].astype(np.float64) @ V, rtol=1e-11, atol=1e-11)


def test_two_modes_is_spmm():
    scipy_sparse = pytest.importorskip("scipy.sparse")
    dims = (30, 20)
    idx, vals = rand_coo(dims, 200, seed=3, signed=True)
    F = rand_factors(dims, 7, seed=4, signed=True)
    S = scipy_sparse.coo_matrix((vals.astype(np.float64), (idx[:, 0], idx[:, 1])), shape=dims).tocsr()
    np.testing.assert_allclose(oracle.mttkrp(dims, idx, vals, F, 0), S @ F[1].astype(np.float64), rtol=1e-12)
    np.testing.assert_allclose(oracle.mttkrp(dims, idx, vals, F, 1), S.T @ F[0].astype(np.float64), rtol=1e-12)


def test_invariances():
    dims = (40, 30, 20)
    idx, vals = rand_coo(dims, 500, seed=5)
    F = rand_factors(dims, 8, seed=6)
    rng = np.random.default_rng(7)
    p = rng.permutation(idx.shape[0])
    # split every nonzero into two halves at the same coordinate
    idx2 = np.concatenate([idx, idx])
    half = (vals.astype(np.float64) / 2)
    for m in range(3):
        base = oracle.mttkrp(dims, idx, vals, F, m)
        np.testing.assert_allclose(oracle.mttkrp(dims, idx[p], vals[p], F, m), base, rtol=1e-13)
        np.testing.assert_allclose(oracle.mttkrp(dims, idx2, np.concatenate([half, half]), F, m), base, rtol=1e-13)
        np.testing.assert_allclose(oracle.mttkrp(dims, idx, vals.astype(np.float64) * 2.5, F, m), 2.5 * base,
                                   rtol=1e-13)
        touched = np.zeros(dims[m], bool)
        touched[idx[:, m]] = True
        assert np.all(base[~touched] == 0.0)
        assert np.all(np.abs(base[touched]).max(axis=1) > 0)


def test_rows_subset_matches_full():
    w = synth.WORKLOADS["zipf3"].scaled(0.0005)
    c = synth.make(w)
    F = synth.factors(c.dims, 8, w.seed)
    for m in range(3):
        full = oracle.mttkrp(c.dims, c.idx, c.vals, F, m)
        rows = synth.subset(c.dims[m], 50, seed=m)
        np.testing.assert_array_equal(oracle.mttkrp_rows(c.dims, c.idx, c.vals, F, m, rows), full[rows])
        # fp64 values (residuals) take the same path
        v64 = c.vals.astype(np.float64) - 0.5
        full64 = oracle.mttkrp(c.dims, c.idx, v64, F, m)
        np.testing.assert_array_equal(oracle.mttkrp_rows(c.dims, c.idx, v64, F, m, rows), full64[rows])


def test_16bit_factor_widening_exact():
    """bf16 / fp16 factors are widened exactly: the oracle on the raw bit
    patterns equals the oracle on numpy's own float32 decoding of them."""
    dims = (9, 8, 7)
    idx, vals = rand_coo(dims, 60, seed=8)
    F = rand_factors(dims, 5, seed=9, signed=True)
    F[0][0, 0] = 6.1e-5 / 2  # an fp16 subnormal
    h = [f.astype(np.float16) for f in F]
    hbits = [a.view(np.uint16) for a in h]
    b = [(f.view(np.uint32) >> 16).astype(np.uint16) for f in F]  # bf16 by truncation
    bf = [(x.astype(np.uint32) << 16).view(np.float32) for x in b]
    for m in range(3):
        np.testing.assert_array_equal(oracle.mttkrp(dims, idx, vals, hbits, m, "f16"),
                                      oracle.mttkrp(dims, idx, vals, [a.astype(np.float32) for a in h], m))
        np.testing.assert_array_equal(oracle.mttkrp(dims, idx, vals, b, m, "bf16"),
                                      oracle.mttkrp(dims, idx, vals, bf, m))


def test_sampled_model_against_dense_cp():
    dims = (5, 4, 6, 3)
    F = rand_factors(dims, 4, seed=10, signed=True)
    idx, _ = rand_coo(dims, 70, seed=11)
    X = np.einsum("az,bz,cz,dz->abcd", *[f.astype(np.float64) for f in F])
    np.testing.assert_allclose(oracle.cp_sample(dims, idx, F), X[tuple(idx.T)], rtol=1e-12, atol=1e-13)


def test_gradient_central_differences():
    dims = (6, 5, 4)
    idx, vals = rand_coo(dims, 80, seed=12)
    F = rand_factors(dims, 3, seed=13)
    F64 = [f.astype(np.float64) for f in F]

    def loss(fs):
        X = np.einsum("az,bz,cz->abc", *fs)
        d = X[tuple(idx.T)] - vals.astype(np.float64)
        return 0.5 * np.dot(d, d)

    L, grads = oracle.completion_grad(dims, idx, vals, F)
    assert abs(L - loss(F64)) < 1e-10 * max(1, L)
    h = 1e-6
    for n in range(3):
        for i in range(dims[n]):
            for r in range(3):
                fp = [f.copy() for f in F64]
                fm = [f.copy() for f in F64]
                fp[n][i, r] += h
                fm[n][i, r] -= h
                fd = (loss(fp) - loss(fm)) / (2 * h)
                assert abs(fd - grads[n][i, r]) <= 1e-6 * max(1.0, abs(fd)), (n, i, r, fd, grads[n][i, r])


def test_synthetic_zipf_frequencies():
    """The generator's Zipf(s) draws follow P(rank k) = k^-s / H (chi-square on the head)."""
    n, s, draws = 1000, 1.1, 400_000
    col = synth.coordinates((n,), draws, (("zipf", s),), seed=99)[:, 0]
    perm = synth.permutation(n, 99, 200)
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    counts = np.bincount(inv[col], minlength=n)
    p = np.arange(1, n + 1, dtype=np.float64) ** -s
    p /= p.sum()
    head = 50
    exp = p[:head] * draws
    chi2 = ((counts[:head] - exp) ** 2 / exp).sum()
    assert chi2 < 100, chi2  # 49 dof: mean 49, sd ~10


# ----------------------------------------------------------------------------- mutants
def _loop_mttkrp(dims, idx, vals, F, m, mutant):
    N = len(dims)
    R = F[0].shape[1]
    out = np.zeros((dims[m], R))
    for k in range(idx.shape[0]):
        ell = np.full(R, float(vals[k])) if mutant != "no_value" else np.ones(R)
        for w in range(N):
            if w == m and mutant != "own_factor":
                continue
            if mutant == "drop_last" and w == (N - 1 if m != N - 1 else N - 2):
                continue
            i = idx[k, w] if mutant != "wrong_index" else idx[k, (w + 1) % N] % dims[w]
            if mutant == "transposed":
                flat = F[w].astype(np.float64).T.reshape(-1)  # column-major read of a row-major factor
                row = np.array([flat[(i * R + r) % flat.size] for r in range(R)])
            else:
                row = F[w][i].astype(np.float64)
            ell = ell * row
        tgt = idx[k, m] if mutant != "wrong_row" else idx[k, (m + 1) % N] % dims[m]
        out[tgt] += ell if mutant != "sign" else -ell if k % 2 else ell
    return out


@pytest.mark.parametrize("mutant", ["no_value", "own_factor", "drop_last", "wrong_index", "transposed",
                                    "wrong_row", "sign"])
def test_pins_reject_mutants(mutant):
    """A plausible mistake in an MTTKRP implementation fails the brute-force
    pin (a reference for how the pins above discriminate)."""
    dims = (6, 5, 4)
    idx, vals = rand_coo(dims, 40, seed=21)
    F = rand_factors(dims, 3, seed=22)
    ok = []
    for m in range(3):
        ref = brute_mttkrp(dims, idx, vals, F, m)
        ok.append(np.allclose(_loop_mttkrp(dims, idx, vals, F, m, mutant), ref, rtol=1e-9))
        assert np.allclose(_loop_mttkrp(dims, idx, vals, F, m, None), ref, rtol=1e-9)
    assert not all(ok), mutant


# ----------------------------------------------------------------------------- the parity metric
# oracle.row_error is the metric every GPU parity assertion goes through: the
# max relative row error of the MTTKRP output (the row-wise reading of the
# error bound on X_(d) times the Khatri-Rao product, Sec. 2.1 Eq. 1).  Its
# cases are worked by hand, so a slip in the function (wrong axis, a missing
# absolute value, a mean for the max, a lenient rule for empty rows, the
# floor taken on the wrong side) changes at least one expected number.
ROW_ERROR_CASES = [
    # (gpu, ref, floor_frac, expected, what the case fixes)
    ([[10.0, 0.2], [1.0, 1.0]], [[10.0, 0.1], [1.0, 1.0]], 0.0, 0.01,
     "row 0: |0.2-0.1| / max(10, 0.1) = 0.01; row 1 exact; the max over rows is 0.01"),
    ([[2.0, 3.0]], [[2.0, 4.0]], 0.0, 0.25, "gpu below ref: |3-4| / 4"),
    ([[-3.0, 1.0]], [[-4.0, 1.0]], 0.0, 0.25, "negative reference entry: |(-3)-(-4)| / |-4|"),
    ([[1.0, 1.0], [2.0, 5.0], [0.5, 0.5]], [[1.0, 1.0], [2.0, 4.0], [0.5, 0.25]], 0.0, 0.5,
     "row 1: |5-4| / 4 = 0.25; row 2: |0.5-0.25| / 0.5 = 0.5; the max over rows is 0.5"),
    ([[0.0, 0.0], [1.0, 1.5]], [[0.0, 0.0], [1.0, 1.0]], 0.0, 0.5, "empty row matched exactly is skipped"),
    ([[0.0, 1e-30], [1.0, 1.0]], [[0.0, 0.0], [1.0, 1.0]], 0.0, float("inf"),
     "any value in a row whose reference is empty is an error"),
    ([[0.0, 0.0]], [[0.0, 0.0]], 0.0, 0.0, "all-zero reference matched exactly"),
    ([[0.0, -2.0]], [[0.0, 0.0]], 0.0, float("inf"), "all-zero reference, nonzero result"),
    ([[2e-9, -1e-9], [2.0, -1.0]], [[1e-9, -1e-9], [2.0, -1.0]], 0.0, 1.0,
     "tiny mixed-sign row without a floor: 1e-9 / 1e-9"),
    ([[2e-9, -1e-9], [2.0, -1.0]], [[1e-9, -1e-9], [2.0, -1.0]], 1e-6, 5e-4,
     "with floor_frac 1e-6 the denominator is 1e-6 * max row norm 2 = 2e-6: 1e-9 / 2e-6"),
    ([[0.0, 3e-6], [-4.0, 2.0]], [[0.0, 0.0], [-4.0, 2.0]], 1e-6, 3e-6 / 4e-6,
     "the floor also covers an empty reference row: 3e-6 / (1e-6 * 4)"),
]


@pytest.mark.parametrize("case", range(len(ROW_ERROR_CASES)))
def test_row_error_hand_worked(case):
    gpu, ref, ff, expected, why = ROW_ERROR_CASES[case]
    got = oracle.row_error(np.array(gpu), np.array(ref), floor_frac=ff)
    if np.isinf(expected):
        assert np.isinf(got), why
    else:
        assert got == pytest.approx(expected, rel=1e-12, abs=0.0), why


def test_row_error_inputs_and_shapes():
    # float32 inputs are widened before the difference (no fp32 rounding of the error)
    a = np.array([[1.0 + 2 ** -23]], dtype=np.float32)
    b = np.array([[1.0]], dtype=np.float64)
    assert oracle.row_error(a, b) == pytest.approx(2 ** -23, rel=1e-12)
    assert oracle.row_error(np.zeros((0, 4)), np.zeros((0, 4))) == 0.0
    # symmetric in which rows are hit: the error of the worst row, wherever it is
    rng = np.random.default_rng(5)
    ref = rng.uniform(0.5, 1.0, (50, 8))
    for r in (0, 17, 49):
        gpu = ref.copy()
        gpu[r, 3] *= 1 + 1e-3
        assert oracle.row_error(gpu, ref) == pytest.approx(1e-3 * ref[r, 3] / ref[r].max(), rel=1e-9)


# mutants of the metric, written here; each must give a different answer on some hand-worked case
def _re_axis0(gpu, ref, floor_frac=0.0):
    gpu, ref = np.asarray(gpu, float), np.asarray(ref, float)
    num, den = np.abs(gpu - ref).max(axis=0), np.abs(ref).max(axis=0)
    z = den == 0
    return float("inf") if np.any(num[z] != 0) else (float((num[~z] / den[~z]).max()) if np.any(~z) else 0.0)


def _re_no_abs(gpu, ref, floor_frac=0.0):
    gpu, ref = np.asarray(gpu, float), np.asarray(ref, float)
    num, den = (gpu - ref).max(axis=1), ref.max(axis=1)
    if floor_frac > 0:
        den = np.maximum(den, floor_frac * den.max())
    z = den == 0
    return float("inf") if np.any(num[z] != 0) else (float((num[~z] / den[~z]).max()) if np.any(~z) else 0.0)


def _re_mean(gpu, ref, floor_frac=0.0):
    gpu, ref = np.asarray(gpu, float), np.asarray(ref, float)
    num, den = np.abs(gpu - ref).max(axis=1), np.abs(ref).max(axis=1)
    if floor_frac > 0:
        den = np.maximum(den, floor_frac * den.max())
    z = den == 0
    return float("inf") if np.any(num[z] != 0) else (float((num[~z] / den[~z]).mean()) if np.any(~z) else 0.0)


def _re_lenient_empty(gpu, ref, floor_frac=0.0):
    gpu, ref = np.asarray(gpu, float), np.asarray(ref, float)
    num, den = np.abs(gpu - ref).max(axis=1), np.abs(ref).max(axis=1)
    if floor_frac > 0:
        den = np.maximum(den, floor_frac * den.max())
    z = den == 0
    return float((num[~z] / den[~z]).max()) if np.any(~z) else 0.0


def _re_floor_min(gpu, ref, floor_frac=0.0):
    gpu, ref = np.asarray(gpu, float), np.asarray(ref, float)
    num, den = np.abs(gpu - ref).max(axis=1), np.abs(ref).max(axis=1)
    if floor_frac > 0:
        den = np.minimum(den, floor_frac * den.max())
    z = den == 0
    return float("inf") if np.any(num[z] != 0) else (float((num[~z] / den[~z]).max()) if np.any(~z) else 0.0)


@pytest.mark.parametrize("mutant", [_re_axis0, _re_no_abs, _re_mean, _re_lenient_empty, _re_floor_min])
def test_row_error_cases_reject_mutants(mutant, monkeypatch):
    # the mutant stands in for the oracle's function; the hand-worked cases must notice
    monkeypatch.setattr(oracle, "row_error", mutant)
    caught = False
    for gpu, ref, ff, expected, _ in ROW_ERROR_CASES:
        got = oracle.row_error(np.array(gpu), np.array(ref), floor_frac=ff)
        if np.isinf(expected) != np.isinf(got) or (not np.isinf(expected) and abs(got - expected) > 1e-12 * max(
                1.0, abs(expected))):
            caught = True
            break
    assert caught, mutant.__name__
