"""Failure handling of the C ABI under host-side fault injection.

AMPED_FAULT=alloc:K makes the K-th device allocation inside one entry-point
call fail as cudaMalloc does on an exhausted device.  Every K from the first
allocation of amped_tensor_create to its last must give AMPED_ERR_OOM with a
message, free whatever the call had built (the device's free memory is the
same afterwards), and leave the library usable.  No GPU fault is involved:
the failure is made on the host, before the allocation is attempted.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_15121_gb300 as amped  # noqa: E402
from paper_2507_15121_gb300 import _lib  # noqa: E402


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_every_allocation_of_create_can_fail_cleanly(monkeypatch):
    w = synth.WORKLOADS["zipf3"].scaled(0.0005)  # 100k nonzeros, 3 modes
    c = synth.make(w)
    monkeypatch.delenv("AMPED_FAULT", raising=False)
    amped.Tensor(c.dims, c.idx, c.vals).close()  # warm-up: modules and the static scratch are loaded
    free0 = _free()
    K = 1
    while True:
        monkeypatch.setenv("AMPED_FAULT", f"alloc:{K}")
        try:
            t = amped.Tensor(c.dims, c.idx, c.vals)
        except _lib.AmpedError as e:
            assert e.status == _lib.ERR_OOM, (K, str(e))
            assert len(str(e)) > len("out of memory: "), K
            assert _free() == free0, f"allocation {K} failed but device memory was not released"
            K += 1
            assert K < 1000
            continue
        t.close()
        break
    # every allocation of the create was hit once: 10 per mode (row tables, streams, segment and
    # combine tables), the caller-order coordinates and 3 for the scratch
    assert K - 1 >= 3 * 10 + 1 + 3, K
    monkeypatch.delenv("AMPED_FAULT")
    assert _free() == free0


def test_failed_scratch_growth_is_reported_and_recovered(monkeypatch):
    w = synth.WORKLOADS["zipf3"].scaled(0.0005)
    c = synth.make(w)
    R = 32
    F = synth.factors(c.dims, R, w.seed)
    Fd = [torch.from_numpy(f).cuda() for f in F]
    monkeypatch.delenv("AMPED_FAULT", raising=False)
    t = amped.Tensor(c.dims, c.idx, c.vals, max_rank=8)  # scratch sized for R = 8
    out = torch.full((c.dims[0], R), float("nan"), device="cuda")
    monkeypatch.setenv("AMPED_FAULT", "alloc:1")  # the growth to R = 32 fails
    with pytest.raises(_lib.AmpedError) as ei:
        t.mttkrp(0, Fd, out=out)
    assert ei.value.status == _lib.ERR_OOM
    torch.cuda.synchronize()
    assert torch.isnan(out).all().item()  # nothing was launched
    monkeypatch.delenv("AMPED_FAULT")
    t.mttkrp(0, Fd, out=out)  # the next call grows the scratch and computes
    ref = oracle.mttkrp(c.dims, c.idx, c.vals, F, 0)
    assert oracle.row_error(out.cpu().numpy(), ref) <= 1e-5
    t.close()
