"""Child process of test_gpu_checked.py.  Runs with AMPED_LIB pointing at the
bounds-checked build of the library (-DAMPED_CHECKS=1).

    python tests/checked_child.py valid     every kernel path on valid inputs: no check fires,
                                            results match the FP64 oracle
    python tests/checked_child.py corrupt   with AMPED_FAULT=coord:K: mode 0's copy holds one
                                            out-of-range coordinate; the MTTKRP call reports the
                                            failed check, the other modes still compute
"""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402
import paper_2507_15121_gb300 as amped  # noqa: E402
from paper_2507_15121_gb300 import _lib  # noqa: E402

BAR = 1e-5


def bits(t):
    return t.detach().cpu().view(torch.int16).numpy().view(np.uint16)


def valid():
    # 3- and 4-mode power-law tensors: long rows (factored and chunk paths), short rows,
    # split rows (small segments), 16-bit factors, the sampled model, both gradient forms
    for name, scale in (("zipf3", 0.0005), ("zipf4", 0.0001)):
        w = synth.WORKLOADS[name].scaled(scale)
        c = synth.make(w)
        F = synth.factors(c.dims, 32, w.seed)
        Fd = [torch.from_numpy(f).cuda() for f in F]
        for items in (0, 64):
            t = amped.Tensor(c.dims, c.idx, c.vals, segment_items=items)
            outs = t.mttkrp_all(Fd)
            for m in range(c.nmodes):
                err = oracle.row_error(outs[m].cpu().numpy(), oracle.mttkrp(c.dims, c.idx, c.vals, F, m))
                assert err <= BAR, (name, items, m, err)
            Fb = [f.to(torch.bfloat16) for f in Fd]
            outs = t.mttkrp_all(Fb)
            for m in range(c.nmodes):
                ref = oracle.mttkrp(c.dims, c.idx, c.vals, [bits(f) for f in Fb], m, "bf16")
                assert oracle.row_error(outs[m].cpu().numpy(), ref) <= BAR, (name, items, m)
            m_gpu = t.cp_sample(Fd).cpu().numpy()
            m_ref = oracle.cp_sample(c.dims, c.idx, F)
            assert np.max(np.abs(m_gpu - m_ref) / np.abs(m_ref)) <= BAR
            g = (m_ref - c.vals).astype(np.float32)
            grads = t.cp_grad(Fd, torch.from_numpy(g).cuda())
            ref = oracle.cp_grad(c.dims, c.idx, g.astype(np.float64), F)
            for n in range(c.nmodes):
                assert oracle.row_error(grads[n].cpu().numpy(), ref[n], floor_frac=1e-6) <= 1e-4, (name, n)
            grads, loss = t.completion_grad(Fd)
            loss_ref, ref = oracle.completion_grad(c.dims, c.idx, c.vals, F)
            assert abs(loss.item() - loss_ref) <= 1e-5 * abs(loss_ref)
            for n in range(c.nmodes):
                assert oracle.row_error(grads[n].cpu().numpy(), ref[n], floor_frac=1e-6) <= 1e-4, (name, n)
            t.close()
    # 6 and 8 modes (32-byte staged records, one nonzero per group step) with 16-bit factors
    rng = np.random.default_rng(5)
    for dims, R, dt, kind in (((30, 20, 12, 9, 7, 5), 16, torch.float32, "f32"),
                              ((12, 10, 9, 8, 7, 6, 5, 4), 32, torch.float16, "f16")):
        nnz = 20000
        idx = np.stack([rng.integers(0, d, nnz) for d in dims], axis=1).astype(np.int32)
        vals = rng.uniform(0, 1, nnz).astype(np.float32)
        F = [rng.uniform(0, 1, (d, R)).astype(np.float32) for d in dims]
        Fd = [torch.from_numpy(f).to(dt).cuda() for f in F]
        Fo = F if kind == "f32" else [bits(f) for f in Fd]
        t = amped.Tensor(dims, idx, vals)
        outs = t.mttkrp_all(Fd)
        for m in range(len(dims)):
            assert oracle.row_error(outs[m].cpu().numpy(), oracle.mttkrp(dims, idx, vals, Fo, m, kind)) <= BAR, (dims, m)
        m_gpu = t.cp_sample(Fd).cpu().numpy()
        m_ref = oracle.cp_sample(dims, idx, Fo, kind)
        assert np.max(np.abs(m_gpu - m_ref) / np.abs(m_ref)) <= BAR
        t.close()
    print("checked build, valid inputs: ok")


def corrupt():
    assert os.environ.get("AMPED_FAULT", "").startswith("coord:")
    w = synth.WORKLOADS["zipf3"].scaled(0.0005)
    c = synth.make(w)
    F = synth.factors(c.dims, 32, w.seed)
    Fd = [torch.from_numpy(f).cuda() for f in F]
    t = amped.Tensor(c.dims, c.idx, c.vals)  # coordinates are valid; the copy is altered afterwards
    out = torch.empty((c.dims[0], 32), device="cuda")
    try:
        t.mttkrp(0, Fd, out=out)
    except _lib.AmpedError as e:
        assert e.status == _lib.ERR_INDEX, str(e)
        assert "bounds check failed: gather coordinate" in str(e), str(e)
    else:
        raise AssertionError("the corrupted coordinate was not reported")
    # the error word was cleared and only mode 0's copy is altered: the other modes compute
    for m in (1, 2):
        o = t.mttkrp(m, Fd)
        assert oracle.row_error(o.cpu().numpy(), oracle.mttkrp(c.dims, c.idx, c.vals, F, m)) <= BAR, m
    t.close()
    print("checked build, corrupted copy: reported")


if __name__ == "__main__":
    assert "checked" in amped.version(), amped.version()
    {"valid": valid, "corrupt": corrupt}[sys.argv[1]]()
