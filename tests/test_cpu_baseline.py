"""The all-cores FP64 CPU baseline computes what the oracle computes."""
import numpy as np
import pytest

import cpu_baseline
import oracle
import synth


@pytest.mark.parametrize("name,scale", [("uniform3", 1.0), ("zipf3", 0.0002), ("zipf4", 0.00005)])
def test_openmp_baseline_matches_oracle(name, scale):
    w = synth.WORKLOADS[name].scaled(scale)
    c = synth.make(w)
    F = synth.factors(c.dims, w.rank, w.seed)
    for m in range(c.nmodes):
        ref = oracle.mttkrp(c.dims, c.idx, c.vals, F, m)
        got = cpu_baseline.mttkrp(c.dims, c.idx, c.vals, F, m, cpu_baseline.order(c.dims, c.idx, m), nthreads=4)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
        assert np.array_equal(got == 0, ref == 0)  # empty rows are exactly zero on both sides


def test_order_is_a_stable_counting_sort():
    idx = np.array([[2, 0], [0, 1], [2, 1], [1, 0], [0, 0]], dtype=np.int32)
    perm, rowptr = cpu_baseline.order((3, 2), idx, 0)
    assert rowptr.tolist() == [0, 2, 3, 5]
    assert perm.tolist() == [1, 4, 3, 0, 2]
