"""CPU-side checks of the CUDA library: it loads, exports every symbol the
header declares, rejects bad arguments before touching the GPU, and its host
reorder / merge-path segment plan satisfies the invariants the kernel relies
on.  A Python walk of the plan with the kernel's flush rules (complete rows
stored, head/tail partials of split rows combined in order) reproduces the
FP64 oracle, which checks the split-row bookkeeping without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth
from paper_2507_15121_gb300 import _lib, plan_mode

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "amped.h")


@pytest.fixture(scope="module")
def L():
    from paper_2507_15121_gb300 import build
    build.build()
    return _lib.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(amped_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert "amped_mttkrp" in names and "amped_tensor_create" in names and "amped_cp_grad" in names
    for n in names:
        assert hasattr(L, n), n
    assert L.amped_version().decode().startswith("amped-gb300")


def test_checked_build_compiles_and_loads(tmp_path):
    """The bounds-checked variant (-DAMPED_CHECKS=1) cross-compiles for sm_103a, exports the same
    entry points and identifies itself; its kernels run in the GPU tests."""
    from paper_2507_15121_gb300 import build
    path = build.build(flags=["-DAMPED_CHECKS=1"], lib_path=str(tmp_path / "libamped_checked.so"),
                       build_dir=str(tmp_path / "_build"))
    C = ctypes.CDLL(path)
    C.amped_version.restype = ctypes.c_char_p
    assert C.amped_version().decode().endswith("(sm_103a, checked)")
    for n in declared_functions():
        assert hasattr(C, n), n


def test_header_is_plain_c(tmp_path):
    """The boundary header compiles as strict ISO C (no C++ or CUDA types leak into it), and a C
    program that calls every declared entry point links against the library."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    names = declared_functions()
    src = tmp_path / "use_amped.c"
    src.write_text('#include "amped.h"\n#include <stdio.h>\ntypedef void (*fn_t)(void);\nint main(void) {\n'
                   "    amped_opts o = {0};\n    (void)o;\n    fn_t fns[] = {\n"
                   + "".join(f"        (fn_t){n},\n" for n in names)
                   + '    };\n    printf("%d\\n", (int)(sizeof fns / sizeof fns[0]));\n'
                   + "    return (int)AMPED_OK;\n}\n")
    lib_dir = os.path.join(ROOT, "paper_2507_15121_gb300")
    subprocess.check_call([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.dirname(HEADER),
                           str(src), "-o", str(tmp_path / "use_amped"), "-L", lib_dir, "-lamped",
                           f"-Wl,-rpath,{lib_dir}"])


def _create(L, nnz, dims, idx, vals):
    dims_a = np.asarray(dims, dtype=np.int64)
    h = ctypes.c_void_p()
    rc = L.amped_tensor_create(nnz, len(dims), dims_a.ctypes.data if len(dims) else None,
                               None if idx is None else idx.ctypes.data, None if vals is None else vals.ctypes.data,
                               None, ctypes.byref(h))
    return rc, h


def test_argument_errors_without_gpu(L):
    idx = np.array([[0, 1], [2, 0]], dtype=np.int32)
    vals = np.ones(2, np.float32)
    assert _create(L, 2, (), idx, vals)[0] == _lib.ERR_INVALID
    assert _create(L, -1, (3, 2), idx, vals)[0] == _lib.ERR_INVALID
    assert _create(L, 2, (0, 2), idx, vals)[0] == _lib.ERR_INVALID
    assert _create(L, 2, (3, 2), None, vals)[0] == _lib.ERR_INVALID
    assert _create(L, 2, tuple([2] * 9), np.zeros((2, 9), np.int32), vals)[0] == _lib.ERR_INVALID
    bad = np.array([[0, 1], [3, 0]], dtype=np.int32)  # 3 is outside dims[0] = 3
    rc, h = _create(L, 2, (3, 2), bad, vals)
    assert rc == _lib.ERR_INDEX and not h.value
    assert b"nonzero 1" in L.amped_last_error()
    neg = np.array([[0, -1]], dtype=np.int32)
    assert _create(L, 1, (3, 2), neg, vals[:1])[0] == _lib.ERR_INDEX
    # stream_memory must be 0, 1 or 2 (checked before anything is allocated)
    opts = _lib.Opts(0, 0, 0, 0, 0, 0, 0, 3)
    dims_a = np.asarray((3, 2), dtype=np.int64)
    h = ctypes.c_void_p()
    assert L.amped_tensor_create(2, 2, dims_a.ctypes.data, idx.ctypes.data, vals.ctypes.data, ctypes.byref(opts),
                                 ctypes.byref(h)) == _lib.ERR_INVALID
    assert b"stream_memory" in L.amped_last_error()
    # inner_order must be 0..3 (create and the host-only planning queries)
    opts = _lib.Opts(0, 0, 0, 0, 0, 4, 0, 0)
    assert L.amped_tensor_create(2, 2, dims_a.ctypes.data, idx.ctypes.data, vals.ctypes.data, ctypes.byref(opts),
                                 ctypes.byref(h)) == _lib.ERR_INVALID
    assert b"inner_order" in L.amped_last_error()
    sz = _lib.PlanSizes()
    assert L.amped_plan_mode(2, 2, dims_a.ctypes.data, idx.ctypes.data, 0, 0, -1, 0, ctypes.byref(sz),
                             *([None] * 9)) == _lib.ERR_INVALID
    n2 = ctypes.c_double()
    assert L.amped_norm2_host(2, 2, dims_a.ctypes.data, idx.ctypes.data, vals.ctypes.data, 5,
                              ctypes.byref(n2)) == _lib.ERR_INVALID
    # calls on a NULL handle fail cleanly
    assert L.amped_mttkrp(None, 0, None, 0, 32, None, None) == _lib.ERR_INVALID
    assert L.amped_tensor_destroy(None) == _lib.OK


def check_plan(dims, idx, mode, items, inner_order="lexicographic", short_rows=0):
    p = plan_mode(dims, idx, mode, items, inner_order, short_rows)
    nnz, I = idx.shape[0], dims[mode]
    keys = idx[:, mode]
    if inner_order == "stable":  # by the mode's coordinate, ties in caller order
        base = np.argsort(keys, kind="stable")
    else:  # by the mode coordinate, then the other coordinates (largest dimension first, or smallest
        # first for the ascending order; ties by lower mode index), ties in caller order
        sign = 1 if inner_order == "lexicographic_ascending" else -1
        others = sorted((n for n in range(len(dims)) if n != mode), key=lambda n: (sign * dims[n], n))
        base = np.lexsort(tuple([np.arange(nnz)] + [idx[:, n] for n in reversed(others)] + [keys]))
    lens = np.bincount(keys, minlength=I)
    rp = np.concatenate([[0], np.cumsum(lens)])
    thr = 32 if short_rows == 0 else (1 if short_rows < 0 else min(short_rows, 125))
    long_rows = np.flatnonzero(lens >= thr)
    short = np.flatnonzero(lens < thr)
    short = short[np.lexsort((short, -lens[short]))]  # decreasing length, ties by id
    np.testing.assert_array_equal(p["rows_long"], long_rows)
    np.testing.assert_array_equal(p["rows_short"], short)
    order = [base[rp[r]:rp[r + 1]] for r in long_rows] + [base[rp[r]:rp[r + 1]] for r in short]
    exp_perm = np.concatenate(order) if order else np.zeros(0, np.int64)
    np.testing.assert_array_equal(p["perm"], exp_perm)
    nnz_L = int(lens[long_rows].sum())
    np.testing.assert_array_equal(p["rowptr_long"], np.concatenate([[0], np.cumsum(lens[long_rows])]))
    np.testing.assert_array_equal(p["rowptr_short"], nnz_L + np.concatenate([[0], np.cumsum(lens[short])]))
    # long part: merge path over the long rows
    L = len(long_rows)
    sr, sz, S = p["seg_row"].astype(np.int64), p["seg_nz"].astype(np.int64), p["sizes"]["long_segments"]
    total = L + nnz_L
    assert S == -(-total // p["items"])
    d = np.minimum(np.arange(S + 1, dtype=np.int64) * p["items"], total)
    np.testing.assert_array_equal(sr + sz, d)
    assert sr[0] == 0 and sz[0] == 0 and sr[-1] == L and sz[-1] == nnz_L
    assert np.all(np.diff(sr) >= 0) and np.all(np.diff(sz) >= 0)
    rpl = p["rowptr_long"].astype(np.int64)
    for s in range(S + 1):  # rows before seg_row are complete, the current row is partly consumed
        r = sr[s]
        if r < L:
            assert rpl[r] <= sz[s] <= rpl[r + 1]
        if r > 0:
            assert rpl[r] <= sz[s]
    straddled = [(int(sr[s]), s) for s in range(1, S) if sr[s] < L and sz[s] > rpl[sr[s]]]
    exp = []
    for r, s in straddled:
        if exp and exp[-1][0] == r and exp[-1][2] == s - 1:
            exp[-1][2] = s
        else:
            exp.append([r, s, s])
    np.testing.assert_array_equal(p["splits"].reshape(-1, 3), np.array(exp, dtype=np.int32).reshape(-1, 3))
    # short part: greedy segments of at most 31 rows and 124 nonzeros covering every short row
    ss = p["seg_short"].astype(np.int64)
    rps = p["rowptr_short"].astype(np.int64)
    assert ss[0] == 0 and ss[-1] == len(short) and np.all(np.diff(ss) > 0) or len(short) == 0
    for t in range(len(ss) - 1):
        a, b = ss[t], ss[t + 1]
        assert b - a <= 31 and rps[b] - rps[a] <= 124
        if b < len(short):  # greedy: the next row would not have fitted
            assert b - a == 31 or rps[b + 1] - rps[a] > 124
    return p


def simulate_kernel(p, dims, idx, vals, F, mode):
    """The MTTKRP kernel in plain Python (fp64): long segments walk their rows
    with the flush rules (complete rows stored, head/tail partials of split
    rows), short segments store their rows whole, then the split rows are
    combined in segment order."""
    I = dims[mode]
    R = F[0].shape[1]
    perm = p["perm"]
    contrib = vals[perm].astype(np.float64)[:, None] * np.ones((1, R))
    for n in range(len(dims)):
        if n != mode:
            contrib = contrib * F[n][idx[perm, n]].astype(np.float64)
    out = np.full((I, R), np.nan)
    rows_L, rp = p["rows_long"], p["rowptr_long"].astype(np.int64)
    L = len(rows_L)
    H, T = {}, {}
    sr, sz = p["seg_row"], p["seg_nz"]
    for s in range(p["sizes"]["long_segments"]):
        row_s, nz_s, row_e, nz_e = int(sr[s]), int(sz[s]), int(sr[s + 1]), int(sz[s + 1])
        cont = rp[row_s] < nz_s
        st = {"i": row_s, "acc": np.zeros(R), "touched": False}

        def rend():
            return rp[st["i"] + 1] if st["i"] < row_e else nz_e

        def flush(row):
            if row == row_s and cont:
                assert s not in H
                H[s] = st["acc"].copy()
            elif row < row_e:
                assert np.isnan(out[rows_L[row], 0]), "row written twice"
                out[rows_L[row]] = st["acc"]
            else:
                assert s not in T
                T[s] = st["acc"].copy()
            st["acc"][:] = 0
            st["touched"] = False

        for k in range(nz_s, nz_e):
            while k >= rend():
                flush(st["i"])
                st["i"] += 1
            st["acc"] += contrib[k]
            st["touched"] = True
        while st["i"] < row_e:
            flush(st["i"])
            st["i"] += 1
        if st["i"] < L and st["touched"]:
            flush(st["i"])
    rows_S, rps, ss = p["rows_short"], p["rowptr_short"].astype(np.int64), p["seg_short"]
    for t in range(p["sizes"]["short_segments"]):
        for j in range(int(ss[t]), int(ss[t + 1])):
            assert np.isnan(out[rows_S[j], 0]), "row written twice"
            out[rows_S[j]] = contrib[rps[j]:rps[j + 1]].sum(axis=0)
    for row, s_a, s_b in p["splits"]:
        assert np.isnan(out[rows_L[row], 0])
        out[rows_L[row]] = T[s_a - 1] + sum(H[s] for s in range(s_a, s_b + 1))
    assert not np.any(np.isnan(out)), "a row was never written"
    return out


CASES = [
    ("uniform-small", (30, 20, 10), 400, 1),
    ("one-long-row", (50, 6, 5), 300, 2),
    ("hypersparse", (5000, 7, 3), 40, 3),
    ("four-modes", (12, 9, 8, 5), 500, 4),
    ("two-modes", (40, 30), 250, 5),
    ("six-modes", (9, 8, 7, 6, 5, 4), 400, 6),
    ("eight-modes", (6, 5, 5, 4, 4, 3, 3, 2), 300, 7),
]


def make_case(name, dims, nnz, seed):
    rng = np.random.default_rng(seed)
    idx = np.stack([rng.integers(0, d, nnz) for d in dims], axis=1).astype(np.int32)
    if name == "one-long-row":
        idx[: nnz * 2 // 3, 0] = 7  # most nonzeros in one output row of mode 0
    vals = rng.uniform(0, 1, nnz).astype(np.float32)
    return idx, vals


@pytest.mark.parametrize("name,dims,nnz,seed", CASES)
@pytest.mark.parametrize("items", [1, 7, 32, 1024, 10 ** 6])
@pytest.mark.parametrize("inner_order,short_rows", [("lexicographic", 0), ("stable", 0), ("lexicographic", -1),
                                                    ("stable", 5), ("lexicographic", 200),
                                                    ("lexicographic_ascending", 0)])
def test_plan_and_simulated_kernel_match_oracle(name, dims, nnz, seed, items, inner_order, short_rows):
    idx, vals = make_case(name, dims, nnz, seed)
    F = [np.random.default_rng(seed + n).uniform(0, 1, (d, 3)).astype(np.float32) for n, d in enumerate(dims)]
    for mode in range(len(dims)):
        p = check_plan(dims, idx, mode, items, inner_order, short_rows)
        got = simulate_kernel(p, dims, idx, vals, F, mode)
        np.testing.assert_allclose(got, oracle.mttkrp(dims, idx, vals, F, mode), rtol=1e-12, atol=1e-12)


def test_plan_empty_tensor_and_zipf():
    dims = (10, 4, 3)
    p = check_plan(dims, np.zeros((0, 3), np.int32), 0, 4)
    assert p["sizes"]["long_segments"] == 0 and p["sizes"]["short_rows"] == 10 and len(p["splits"]) == 0
    w = synth.WORKLOADS["zipf3"].scaled(0.0002)
    c = synth.make(w)
    for mode in range(3):
        check_plan(c.dims, c.idx, mode, 256)


def _norm2_host(L, dims, idx, vals, inner_order):
    dims_a = np.asarray(dims, dtype=np.int64)
    out = ctypes.c_double()
    rc = L.amped_norm2_host(idx.shape[0], len(dims), dims_a.ctypes.data, idx.ctypes.data if idx.size else None,
                            vals.ctypes.data if vals.size else None, inner_order, ctypes.byref(out))
    return rc, out.value


@pytest.mark.parametrize("dims", [(30, 20, 10), (12, 9, 8, 5), (40, 30), (6, 5, 4, 3, 3, 2)])
@pytest.mark.parametrize("inner_order", [0, 1, 2, 3])
def test_tensor_norm_sums_repeated_coordinates(L, dims, inner_order):
    """The host norm ||X||^2 with repeated coordinates summed (the ALS fit's ||X||) equals the
    oracle's, for every inner order, with many repeats (some rows hold most of the nonzeros)."""
    from oracle import als
    rng = np.random.default_rng(len(dims) * 10 + inner_order)
    nnz = 3000
    idx = np.stack([rng.integers(0, d, nnz) for d in dims], axis=1).astype(np.int32)
    idx[: nnz // 3, 0] = 2  # a hot row
    idx[nnz // 2:] = idx[rng.integers(0, nnz // 2, nnz - nnz // 2)]  # repeated coordinates
    vals = rng.uniform(-1, 1, nnz).astype(np.float32)
    rc, v = _norm2_host(L, dims, idx, vals, inner_order)
    assert rc == _lib.OK
    assert v == pytest.approx(als.norm2(idx, vals), rel=1e-12)
    assert v != pytest.approx(float(np.dot(vals.astype(np.float64), vals)), rel=1e-3)  # repeats matter here
    rc, v0 = _norm2_host(L, dims, idx[:0], vals[:0], inner_order)
    assert rc == _lib.OK and v0 == 0.0
    bad = idx.copy()
    bad[5, 0] = dims[0]
    assert _norm2_host(L, dims, bad, vals, inner_order)[0] == _lib.ERR_INDEX
