"""The allocation-free MTTKRP entry point (amped_mttkrp_noalloc).

Some callers cannot allocate device memory while they run (their memory pool
owns the whole GPU, or their budget was fixed up front, or cudaMalloc's
implicit synchronisation is not acceptable in their loop).  For them the
library keeps its scratch in one fixed static device array.  This file checks,
through the C ABI, that two calls in a row give the same result as the regular
entry point (amped_mttkrp) and as the FP64 oracle, that the calls leave the
device's free memory unchanged, and that a mode too large for the fixed
buffer is refused with an error instead of launching.  It is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_15121_gb300 as amped  # noqa: E402
from paper_2507_15121_gb300 import _lib  # noqa: E402


def _call(L, fn, t, mode, F, code, R, out):
    fp = _lib.ptr_array([f.data_ptr() for f in F])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(t.handle, mode, fp, code, R, out.data_ptr(), stream)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_noalloc_matches_regular_entry_twice(dtype):
    L = _lib.lib()
    w = synth.WORKLOADS["zipf3"].scaled(0.002)  # 400k nonzeros, 20000 x 10000 x 4000
    c = synth.make(w)
    R = 32
    F = [torch.from_numpy(f).to("cuda", dtype) for f in synth.factors(c.dims, R, w.seed)]
    code = _lib.F32 if dtype == torch.float32 else _lib.BF16
    # the oracle reads the factors exactly as the GPU stores them (16-bit: the rounded bits)
    if dtype == torch.float32:
        Fo, odt = [f.cpu().numpy() for f in F], "f32"
    else:
        Fo, odt = [f.cpu().view(torch.int16).numpy().view(np.uint16) for f in F], "bf16"
    t = amped.Tensor(c.dims, c.idx, c.vals)
    for mode in range(3):
        ref = torch.empty((c.dims[mode], R), device="cuda")
        assert _call(L, L.amped_mttkrp, t, mode, F, code, R, ref) == _lib.OK
        ref = ref.cpu().numpy()
        exact = oracle.mttkrp(c.dims, c.idx, c.vals, Fo, mode, dtype=odt)
        outs = [torch.full((c.dims[mode], R), float("nan"), device="cuda") for _ in range(2)]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for out in outs:  # the static buffer keeps the last call's contents: reuse must be safe
            rc = _call(L, L.amped_mttkrp_noalloc, t, mode, F, code, R, out)
            assert rc == _lib.OK, L.amped_last_error()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "an allocation-free call changed the free device memory"
        for out in outs:
            got = out.cpu().numpy()
            assert oracle.row_error(got, ref) <= 1e-5
            assert oracle.row_error(got, exact) <= 1e-5
    t.close()


def test_noalloc_honours_kernel_events():
    L = _lib.lib()
    w = synth.WORKLOADS["zipf3"].scaled(0.0005)
    c = synth.make(w)
    R = 32
    F = [torch.from_numpy(f).cuda() for f in synth.factors(c.dims, R, w.seed)]
    t = amped.Tensor(c.dims, c.idx, c.vals)
    out = torch.empty((c.dims[0], R), device="cuda")
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t.set_kernel_events(start, stop)  # records each once first: torch creates events lazily
    torch.cuda.synchronize()
    assert _call(L, L.amped_mttkrp_noalloc, t, 0, F, _lib.F32, R, out) == _lib.OK, L.amped_last_error()
    torch.cuda.synchronize()
    assert start.elapsed_time(stop) > 0.0  # both events were recorded around the kernel
    t.close()


def test_noalloc_rejects_modes_beyond_the_static_buffer():
    L = _lib.lib()
    w = synth.WORKLOADS["zipf3"].scaled(0.001)  # 200k nonzeros
    c = synth.make(w)
    R = 64
    # one work item per segment: 2 * S * R * 4 bytes of partials exceed 32 MiB
    t = amped.Tensor(c.dims, c.idx, c.vals, segment_items=1)
    F = [torch.ones((d, R), device="cuda") for d in c.dims]
    out = torch.zeros((c.dims[0], R), device="cuda")
    rc = _call(L, L.amped_mttkrp_noalloc, t, 0, F, _lib.F32, R, out)
    assert rc == _lib.ERR_UNSUPPORTED
    assert b"static buffer" in L.amped_last_error()
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0  # nothing was launched
    t.close()
