"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Also: tensors of 2 to 8 modes, host-resident (out-of-core) streams against
device-resident ones (identical bits), the end-to-end host-buffer entry, and
full-size runs checked on sampled rows.

Bars: fp32 factors -> max relative row error <= 1e-5; bf16/fp16 factors ->
<= 1e-5 against the oracle run on the same rounded factors (kernel
arithmetic) and <= 2e-2 against the oracle on the original fp32 factors
(storage rounding included); gradients (mixed-sign values) -> <= 1e-4 with
the denominator floored at 1e-6 of the largest row.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_15121_gb300 as amped  # noqa: E402

FP32_BAR = 1e-5
LOWP_BAR = 2e-2
GRAD_BAR = 1e-4


def dev(a, dtype=torch.float32):
    # rounded to the storage type on the host, then uploaded: the device holds the same bits
    # that host_bits() gives the oracle
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).to("cuda")


def host_bits(t):
    """raw uint16 bit patterns of a bf16/fp16 tensor made by dev() (oracle input: the host
    rounding, read back unchanged)."""
    return t.detach().cpu().view(torch.int16).numpy().view(np.uint16)


def run_all(c, F, dtype=torch.float32, items=0, R=None):
    t = amped.Tensor(c.dims, c.idx, c.vals, segment_items=items)
    Fd = [dev(f, dtype) for f in F]
    outs = t.mttkrp_all(Fd)
    torch.cuda.synchronize()
    res = [o.cpu().numpy() for o in outs]
    t.close()
    return res, Fd


def check_fp32(c, F, items=0, bar=FP32_BAR):
    got, _ = run_all(c, F, items=items)
    for m in range(c.nmodes):
        ref = oracle.mttkrp(c.dims, c.idx, c.vals, F, m)
        err = oracle.row_error(got[m], ref)
        assert err <= bar, (m, err)


# --------------------------------------------------------------------------- configs at test size
def test_uniform3_full_size_fp32():
    """3-mode 1000x800x600, 100k uniform nonzeros (duplicates merged), R=16."""
    w = synth.WORKLOADS["uniform3"]
    c = synth.make(w)
    F = synth.factors(c.dims, w.rank, w.seed)
    check_fp32(c, F)


@pytest.mark.parametrize("scale", [0.001, 0.005])
def test_zipf3_reduced_fp32(scale):
    w = synth.WORKLOADS["zipf3"].scaled(scale)
    c = synth.make(w)
    F = synth.factors(c.dims, 32, w.seed)
    check_fp32(c, F)


def test_zipf4_reduced_fp32():
    w = synth.WORKLOADS["zipf4"].scaled(0.0003)
    c = synth.make(w)
    F = synth.factors(c.dims, 32, w.seed)
    check_fp32(c, F)


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_zipf5_five_modes(dt):
    """5-mode power-law tensor with the Twitch tensor's shape (scaled), all modes."""
    w = synth.WORKLOADS["zipf5"].scaled(0.0004)
    c = synth.make(w)
    F = synth.factors(c.dims, 32, w.seed)
    got, Fd = run_all(c, F, dtype=dt)
    if dt == torch.float32:
        refs = [oracle.mttkrp(c.dims, c.idx, c.vals, F, m) for m in range(5)]
    else:
        bits = [host_bits(f) for f in Fd]
        refs = [oracle.mttkrp(c.dims, c.idx, c.vals, bits, m, "bf16") for m in range(5)]
    for m in range(5):
        assert oracle.row_error(got[m], refs[m]) <= FP32_BAR, m
    t = amped.Tensor(c.dims, c.idx, c.vals)
    m_gpu = t.cp_sample([dev(f) for f in F]).cpu().numpy()
    m_ref = oracle.cp_sample(c.dims, c.idx, F)
    assert np.max(np.abs(m_gpu - m_ref) / np.abs(m_ref)) <= FP32_BAR


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("R", [32, 64])
def test_zipf3_16bit_factors(dt, R):
    w = synth.WORKLOADS["zipf3_r64"].scaled(0.001)
    c = synth.make(w)
    F = synth.factors(c.dims, R, w.seed)
    got, Fd = run_all(c, F, dtype=dt)
    name = "bf16" if dt == torch.bfloat16 else "f16"
    bits = [host_bits(f) for f in Fd]
    for m in range(3):
        ref_rounded = oracle.mttkrp(c.dims, c.idx, c.vals, bits, m, name)
        ref_fp32 = oracle.mttkrp(c.dims, c.idx, c.vals, F, m)
        assert oracle.row_error(got[m], ref_rounded) <= FP32_BAR
        assert oracle.row_error(got[m], ref_fp32) <= LOWP_BAR


# --------------------------------------------------------------------------- shapes and edge cases
@pytest.mark.parametrize("items", [1, 7, 32, 1024, 10 ** 7])
def test_segment_length_sweep(items):
    rng = np.random.default_rng(items)
    dims = (300, 200, 100)
    nnz = 20000
    idx = np.stack([rng.integers(0, d, nnz) for d in dims], axis=1).astype(np.int32)
    idx[:5000, 0] = 17  # one long row in mode 0
    c = synth.Coo(dims, idx, rng.uniform(0, 1, nnz).astype(np.float32))
    F = [rng.uniform(0, 1, (d, 32)).astype(np.float32) for d in dims]
    check_fp32(c, F, items=items)


@pytest.mark.parametrize("R", [1, 3, 8, 16, 24, 32, 48, 64, 128])
def test_rank_sweep_fp32(R):
    rng = np.random.default_rng(R)
    dims = (500, 300, 200)
    nnz = 30000
    idx = np.stack([rng.integers(0, d, nnz) for d in dims], axis=1).astype(np.int32)
    c = synth.Coo(dims, idx, rng.uniform(0, 1, nnz).astype(np.float32))
    F = [rng.uniform(0, 1, (d, R)).astype(np.float32) for d in dims]
    check_fp32(c, F, items=512)


@pytest.mark.parametrize("R", [5, 8, 16, 32, 128, 256])
def test_rank_sweep_bf16(R):
    rng = np.random.default_rng(100 + R)
    dims = (400, 300, 200)
    nnz = 20000
    idx = np.stack([rng.integers(0, d, nnz) for d in dims], axis=1).astype(np.int32)
    c = synth.Coo(dims, idx, rng.uniform(0, 1, nnz).astype(np.float32))
    F = [rng.uniform(0, 1, (d, R)).astype(np.float32) for d in dims]
    got, Fd = run_all(c, F, dtype=torch.bfloat16)
    bits = [host_bits(f) for f in Fd]
    for m in range(3):
        assert oracle.row_error(got[m], oracle.mttkrp(c.dims, c.idx, c.vals, bits, m, "bf16")) <= FP32_BAR


def test_unsupported_rank_is_an_error():
    c = synth.Coo((4, 4, 4), np.zeros((1, 3), np.int32), np.ones(1, np.float32))
    t = amped.Tensor(c.dims, c.idx, c.vals)
    F = [torch.ones((4, 130), device="cuda") for _ in range(3)]  # fp32 R=130: no kernel
    with pytest.raises(amped.AmpedError) as e:
        t.mttkrp(0, F)
    assert e.value.status == -5


def test_edge_cases():
    rng = np.random.default_rng(5)
    R = 32
    # empty tensor: every output row is exactly zero
    c = synth.Coo((7, 5, 3), np.zeros((0, 3), np.int32), np.zeros(0, np.float32))
    got, _ = run_all(c, [np.ones((d, R), np.float32) for d in c.dims])
    assert all(np.all(g == 0) for g in got)
    # single nonzero
    c = synth.Coo((7, 5, 3), np.array([[6, 0, 2]], np.int32), np.array([2.5], np.float32))
    check_fp32(c, [rng.uniform(0, 1, (d, R)).astype(np.float32) for d in c.dims])
    # one row holds every nonzero; a mode of size 1
    nnz = 50000
    idx = np.stack([np.full(nnz, 3), rng.integers(0, 1, nnz), rng.integers(0, 900, nnz)], 1).astype(np.int32)
    c = synth.Coo((10, 1, 900), idx, rng.uniform(0, 1, nnz).astype(np.float32))
    check_fp32(c, [rng.uniform(0, 1, (d, R)).astype(np.float32) for d in c.dims], items=256)
    # two modes (sparse matrix times dense)
    dims = (700, 500)
    idx = np.stack([rng.integers(0, d, 9000) for d in dims], 1).astype(np.int32)
    c = synth.Coo(dims, idx, rng.uniform(0, 1, 9000).astype(np.float32))
    check_fp32(c, [rng.uniform(0, 1, (d, R)).astype(np.float32) for d in dims])
    # hyper-sparse: 40 nonzeros over a million rows
    dims = (1_000_000, 20, 30)
    idx = np.stack([rng.integers(0, d, 40) for d in dims], 1).astype(np.int32)
    c = synth.Coo(dims, idx, rng.uniform(0, 1, 40).astype(np.float32))
    check_fp32(c, [rng.uniform(0, 1, (d, R)).astype(np.float32) for d in dims])


def test_repeat_calls_and_single_mode_entry():
    w = synth.WORKLOADS["zipf3"].scaled(0.0005)
    c = synth.make(w)
    F = synth.factors(c.dims, 32, w.seed)
    t = amped.Tensor(c.dims, c.idx, c.vals)
    Fd = [dev(f) for f in F]
    a = [t.mttkrp(m, Fd).cpu().numpy() for m in range(3)]
    b = [o.cpu().numpy() for o in t.mttkrp_all(Fd)]
    for m in range(3):  # the split-row combine is deterministic: identical results
        np.testing.assert_array_equal(a[m], b[m])
    host = t.mttkrp_all_host([torch.from_numpy(f) for f in F])
    for m in range(3):
        np.testing.assert_array_equal(host[m].numpy(), b[m])
    # 16-bit host factors (pinned, so the copies overlap the kernels) against the device entry
    Fh = [torch.from_numpy(f).to(torch.bfloat16).pin_memory() for f in F]
    outs_h = [torch.empty((d, 32), dtype=torch.float32).pin_memory() for d in c.dims]
    t.mttkrp_all_host(Fh, outs_h)
    dev_b = t.mttkrp_all([f.cuda() for f in Fh])
    for m in range(3):
        np.testing.assert_array_equal(outs_h[m].numpy(), dev_b[m].cpu().numpy())
    assert amped.kernel_launches() > 0


# --------------------------------------------------------------------------- sampled model and gradient
def test_cp_sample_and_grad_against_oracle():
    w = synth.WORKLOADS["planted3"].scaled(0.0005)
    c = synth.make(w)
    # planted values: the oracle evaluates the planted CP model, plus the noise
    x = (oracle.cp_sample(c.dims, c.idx, c.extra["planted_factors"]) + c.extra["noise"]).astype(np.float32)
    F = synth.factors(c.dims, 32, w.seed, scale=w.factor_scale)
    t = amped.Tensor(c.dims, c.idx, x)
    Fd = [dev(f) for f in F]
    m = t.cp_sample(Fd).cpu().numpy()
    m_ref = oracle.cp_sample(c.dims, c.idx, F)
    assert np.max(np.abs(m - m_ref) / np.abs(m_ref)) <= FP32_BAR
    g = (m_ref - x.astype(np.float64))
    grads = t.cp_grad(Fd, dev(g.astype(np.float32)))
    ref = oracle.cp_grad(c.dims, c.idx, g.astype(np.float32).astype(np.float64), F)
    for n in range(3):
        assert oracle.row_error(grads[n].cpu().numpy(), ref[n], floor_frac=1e-6) <= GRAD_BAR


def test_autograd_completion_step_gradient_check():
    """Planted rank-16 CP tensor; on a 1k-nonzero subset the autograd gradient
    of L = 1/2 sum (m - x)^2 matches the FP64 oracle gradient and FP64
    central finite differences of the oracle loss."""
    w = synth.WORKLOADS["planted3"].scaled(0.0002)
    c = synth.make(w)
    sub = synth.subset(c.nnz, 1000, w.seed)
    idx = np.ascontiguousarray(c.idx[sub])
    x = (oracle.cp_sample(c.dims, idx, c.extra["planted_factors"]) + c.extra["noise"][sub]).astype(np.float32)
    F = synth.factors(c.dims, 32, w.seed, scale=w.factor_scale)
    t = amped.Tensor(c.dims, idx, x)
    Fd = [dev(f).requires_grad_(True) for f in F]
    loss = amped.completion_loss(t, Fd, dev(x))
    loss.backward()
    L_ref, G_ref = oracle.completion_grad(c.dims, idx, x, F)
    assert abs(loss.item() - L_ref) <= 1e-5 * L_ref
    for n in range(3):
        assert oracle.row_error(Fd[n].grad.cpu().numpy(), G_ref[n], floor_frac=1e-6) <= GRAD_BAR
    # finite differences of the FP64 oracle loss on entries touched by the subset
    rng = np.random.default_rng(0)
    F64 = [f.astype(np.float64) for f in F]
    for n in range(3):
        rows = np.unique(idx[:, n])
        for _ in range(4):
            i, r = int(rng.choice(rows)), int(rng.integers(0, 32))
            h = 1e-6 * max(1.0, abs(F64[n][i, r]))
            Fp = [f.copy() for f in F64]
            Fm = [f.copy() for f in F64]
            Fp[n][i, r] += h
            Fm[n][i, r] -= h
            lp = oracle.completion_loss(oracle_cp_sample64(c.dims, idx, Fp), x)
            lm = oracle.completion_loss(oracle_cp_sample64(c.dims, idx, Fm), x)
            fd = (lp - lm) / (2 * h)
            gpu = float(Fd[n].grad[i, r])
            assert abs(gpu - fd) <= 1e-4 * max(1.0, abs(fd)), (n, i, r, gpu, fd)


def oracle_cp_sample64(dims, idx, F64):
    """The sampled model for fp64 factors: the oracle's fp32 interface would
    round the perturbed factors, so evaluate the definition with numpy here."""
    p = np.ones((idx.shape[0], F64[0].shape[1]))
    for n in range(len(dims)):
        p *= F64[n][idx[:, n]]
    return p.sum(axis=1)


def test_planted_model_residual_is_noise():
    """With the planted factors as the model, the residual is the added noise."""
    w = synth.WORKLOADS["planted3"].scaled(0.0002)
    c = synth.make(w)
    B = c.extra["planted_factors"]
    x = (oracle.cp_sample(c.dims, c.idx, B) + c.extra["noise"]).astype(np.float32)
    t = amped.Tensor(c.dims, c.idx, x)
    m = t.cp_sample([dev(b) for b in B]).cpu().numpy()
    resid = m - x
    assert abs(resid.std() - w.noise_sd) < 0.1 * w.noise_sd


def _planted(scale, dims_override=None):
    w = synth.WORKLOADS["planted3"].scaled(scale)
    c = synth.make(w)
    x = (oracle.cp_sample(c.dims, c.idx, c.extra["planted_factors"]) + c.extra["noise"]).astype(np.float32)
    F = synth.factors(c.dims, 32, w.seed, scale=w.factor_scale)
    return w, c, x, F


@pytest.mark.parametrize("short_rows", [0, -1])
def test_fused_completion_grad_against_oracle(short_rows):
    """amped_cp_completion_grad: one fused pass per mode (model value rebuilt from the
    output-mode row) against the FP64 oracle's completion gradient and loss."""
    w, c, x, F = _planted(0.0005)
    t = amped.Tensor(c.dims, c.idx, x, short_rows=short_rows)
    Fd = [dev(f) for f in F]
    grads, loss = t.completion_grad(Fd)
    L_ref, G_ref = oracle.completion_grad(c.dims, c.idx, x, F)
    assert abs(loss.item() - L_ref) <= 1e-5 * L_ref
    for n in range(3):
        assert oracle.row_error(grads[n].cpu().numpy(), G_ref[n], floor_frac=1e-6) <= GRAD_BAR
    # the generic gradient with residual values gives the same result
    m = t.cp_sample(Fd)
    generic = t.cp_grad(Fd, (m - dev(x)).contiguous())
    for n in range(3):
        assert oracle.row_error(grads[n].cpu().numpy(), generic[n].cpu().numpy().astype(np.float64),
                                floor_frac=1e-6) <= GRAD_BAR


def test_fused_completion_grad_bf16_and_autograd():
    w, c, x, F = _planted(0.0003)
    t = amped.Tensor(c.dims, c.idx, x)
    Fb = [dev(f, torch.bfloat16) for f in F]
    grads, loss = t.completion_grad(Fb)
    bits = [host_bits(f) for f in Fb]
    m = oracle.cp_sample(c.dims, c.idx, bits, "bf16")
    G_ref = oracle.cp_grad(c.dims, c.idx, m - x.astype(np.float64), bits, "bf16")
    for n in range(3):
        assert oracle.row_error(grads[n].cpu().numpy(), G_ref[n], floor_frac=1e-6) <= GRAD_BAR
    # autograd through the fused loss equals the two-kernel autograd path
    Fa = [dev(f).requires_grad_(True) for f in F]
    Fg = [dev(f).requires_grad_(True) for f in F]
    la = amped.fused_completion_loss(t, Fa)
    la.backward()
    lg = amped.completion_loss(t, Fg, dev(x))
    lg.backward()
    assert abs(la.item() - lg.item()) <= 1e-5 * lg.item()
    for n in range(3):
        assert oracle.row_error(Fa[n].grad.cpu().numpy(), Fg[n].grad.cpu().numpy().astype(np.float64),
                                floor_frac=1e-6) <= GRAD_BAR


# --------------------------------------------------------------------------- full size, sampled rows
@pytest.mark.parametrize("dims,R,dt", [((40, 30, 20, 12, 9, 7), 16, torch.float32),
                                         ((30, 20, 15, 10, 8, 6, 5), 32, torch.float32),
                                         ((25, 20, 12, 10, 8, 6, 5, 4), 8, torch.float32),
                                         ((30, 20, 15, 10, 8, 6, 5), 32, torch.bfloat16),
                                         ((25, 20, 12, 10, 8, 6, 5, 4), 3, torch.float32)])
def test_six_to_eight_modes(dims, R, dt):
    """Tensors of 6 to 8 modes (5 to 7 input modes per MTTKRP): every mode, the sampled
    model, the gradient and the fused completion gradient against the oracle."""
    rng = np.random.default_rng(len(dims) * 100 + R)
    nnz = 20000
    idx = np.stack([rng.integers(0, d, nnz) for d in dims], axis=1).astype(np.int32)
    idx[: nnz // 4, 0] = 3  # one long row in mode 0
    vals = rng.uniform(0, 1, nnz).astype(np.float32)
    F32 = [rng.uniform(0, 1, (d, R)).astype(np.float32) for d in dims]
    t = amped.Tensor(dims, idx, vals)
    Fd = [dev(f, dt) for f in F32]
    F = F32 if dt == torch.float32 else [host_bits(f) for f in Fd]
    code = "f32" if dt == torch.float32 else "bf16"
    outs = t.mttkrp_all(Fd)
    m = t.cp_sample(Fd)
    m_ref = oracle.cp_sample(dims, idx, F, code)
    g = (m_ref - vals.astype(np.float64)).astype(np.float32)  # residuals of the oracle's model
    grads = t.cp_grad(Fd, torch.from_numpy(g).cuda())
    fg, loss = t.completion_grad(Fd)
    torch.cuda.synchronize()
    for n in range(len(dims)):
        ref = oracle.mttkrp(dims, idx, vals, F, n, code)
        assert oracle.row_error(outs[n].cpu().numpy(), ref) <= FP32_BAR, n
    assert np.max(np.abs(m.cpu().numpy() - m_ref) / np.abs(m_ref)) <= FP32_BAR
    g_ref = oracle.cp_grad(dims, idx, g.astype(np.float64), F, code)
    x_ref = oracle.cp_grad(dims, idx, m_ref - vals.astype(np.float64), F, code)
    for n in range(len(dims)):
        assert oracle.row_error(grads[n].cpu().numpy(), g_ref[n], floor_frac=1e-6) <= GRAD_BAR, n
        assert oracle.row_error(fg[n].cpu().numpy(), x_ref[n], floor_frac=1e-6) <= GRAD_BAR, n
    assert loss.item() == pytest.approx(oracle.completion_loss(m_ref, vals), rel=1e-5)
    t.close()


@pytest.mark.parametrize("name,scale", [("zipf3", 0.002), ("zipf5", 0.0002)])
def test_host_resident_streams_match_device(name, scale):
    """Out-of-core form: the per-nonzero streams in mapped pinned host memory, read by the
    same kernels over the host link, give the same bits as device-resident streams."""
    w = synth.WORKLOADS[name].scaled(scale)
    c = synth.make(w)
    R = 16
    F = [dev(f) for f in synth.factors(c.dims, R, w.seed)]
    g = torch.from_numpy(np.random.default_rng(3).standard_normal(c.nnz).astype(np.float32)).cuda()
    res = {}
    for where in ("device", "host"):
        t = amped.Tensor(c.dims, c.idx, c.vals, stream_memory=where)
        outs = t.mttkrp_all(F)
        m = t.cp_sample(F)
        grads = t.cp_grad(F, g)
        fg, loss = t.completion_grad(F)
        A = [f.clone() for f in F]
        grams = torch.empty((c.nmodes, R, R), dtype=torch.float64, device="cuda")
        stats = torch.zeros(8, dtype=torch.float64, device="cuda")
        t.cp_als_sweep(A, grams, stats, init=True)
        torch.cuda.synchronize()
        res[where] = ([o.cpu() for o in outs], m.cpu(), [x.cpu() for x in grads], [x.cpu() for x in fg],
                      loss.item(), [a.cpu() for a in A], stats.cpu())
        t.close()
    d, h = res["device"], res["host"]
    for a, b in zip(d[0] + [d[1]] + d[2] + d[3], h[0] + [h[1]] + h[2] + h[3]):
        assert torch.equal(a, b)  # deterministic kernels, same data: identical bits
    assert h[4] == pytest.approx(d[4], rel=1e-12)  # fp64 loss, atomics in any order
    for a, b in zip(d[5], h[5]):
        torch.testing.assert_close(b, a, rtol=1e-5, atol=1e-7)  # fp64 Gram atomics feed the solve
    assert h[6][0].item() == pytest.approx(d[6][0].item(), abs=1e-9)


def oracle_rows_all_modes(c, F, rows):
    """The oracle's sampled-row pass for every mode; the single-threaded passes of
    different modes run side by side (ctypes releases the GIL during each call)."""
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=len(rows)) as ex:
        futs = [ex.submit(oracle.mttkrp_rows, c.dims, c.idx, c.vals, F, m, rows[m]) for m in range(len(rows))]
        return [f.result() for f in futs]


def sampled_rows(c, mode, k, seed):
    counts = np.bincount(c.idx[:, mode], minlength=c.dims[mode])
    hot = np.argsort(-counts, kind="stable")[:16]
    rows = np.unique(np.concatenate([hot, synth.subset(c.dims[mode], k, seed + mode)]))
    return rows


@pytest.mark.slow
def test_zipf3_full_size_sampled_rows():
    """10M x 5M x 2M, 200M Zipf(1.1) nonzeros, R=32, fp32 and bf16 factors, in the
    launch configuration the benchmark times; the oracle recomputes 4096 seeded
    rows per mode (plus the 16 hottest) in one pass over the COO."""
    w = synth.WORKLOADS["zipf3"]
    c = synth.make(w)
    F = synth.factors(c.dims, 32, w.seed)
    t = amped.Tensor(c.dims, c.idx, c.vals)
    Fd = [dev(f) for f in F]
    outs = [o.cpu().numpy() for o in t.mttkrp_all(Fd)]
    Fb = [f.to(torch.bfloat16) for f in Fd]
    outs_b = [o.cpu().numpy() for o in t.mttkrp_all(Fb)]
    del Fd, Fb
    t.close()
    rows = [sampled_rows(c, m, 4096, w.seed) for m in range(3)]
    refs = oracle_rows_all_modes(c, F, rows)
    for m in range(3):
        ref = refs[m]
        assert oracle.row_error(outs[m][rows[m]], ref) <= FP32_BAR, m
        assert oracle.row_error(outs_b[m][rows[m]], ref) <= LOWP_BAR, m
        # rows that no nonzero touches are exactly zero
        counts = np.bincount(c.idx[:, m], minlength=c.dims[m])
        empty = np.flatnonzero(counts == 0)[:1000]
        assert np.all(outs[m][empty] == 0)


@pytest.mark.slow
def test_zipf4_billion_full_size_sampled_rows():
    """50M x 20M x 5M x 1000, 1.0B nonzeros (modes 0-2 Zipf(1.2), mode 3 uniform,
    lognormal values), R=32 fp32 factors: all-mode MTTKRP with the four mode copies
    resident in HBM, and again with the copies' streams in host memory; 2048 seeded rows
    per mode (plus the 16 hottest) of both against the oracle."""
    w = synth.WORKLOADS["zipf4"]
    c = synth.make(w)
    F = synth.factors(c.dims, 32, w.seed)
    rows = [sampled_rows(c, m, 2048, w.seed) for m in range(4)]

    def run(**kw):  # sampled rows and a digest of every output (host memory stays bounded)
        import hashlib
        t = amped.Tensor(c.dims, c.idx, c.vals, **kw)
        outs = t.mttkrp_all(Fd)
        torch.cuda.synchronize()
        got = [(o[torch.from_numpy(rows[m]).cuda()].cpu().numpy(), hashlib.sha256(o.cpu().numpy()).hexdigest())
               for m, o in enumerate(outs)]
        del outs
        t.close()
        torch.cuda.empty_cache()
        return got

    Fd = [dev(f) for f in F]
    dev_res = run()
    # out-of-core form (paper Sec. 4, host-resident shards): the four copies' per-nonzero
    # streams (64 GB) in pinned host memory, read by the kernels over the host link
    host_res = run(stream_memory="host", keep_perm=False, keep_coo=False)
    del Fd
    refs = oracle_rows_all_modes(c, F, rows)
    for m in range(4):
        assert oracle.row_error(dev_res[m][0], refs[m]) <= FP32_BAR, m
        assert oracle.row_error(host_res[m][0], refs[m]) <= FP32_BAR, m
        assert host_res[m][1] == dev_res[m][1], m  # same kernels, same order: identical bits


@pytest.mark.slow
def test_zipf3_r64_full_size_16bit_sampled_rows():
    """The precision configuration at full size: 10M x 5M x 2M, 200M nonzeros, R=64, factors
    stored in bf16 and in fp16 (rounded on the host from the same fp32 draws).  2048 seeded
    rows per mode (plus the 16 hottest): each 16-bit result against the oracle on its own
    rounded factors (kernel arithmetic) and against the oracle on the fp32 factors."""
    w = synth.WORKLOADS["zipf3_r64"]
    c = synth.make(w)
    F = synth.factors(c.dims, 64, w.seed)
    rows = [sampled_rows(c, m, 2048, w.seed) for m in range(3)]
    t = amped.Tensor(c.dims, c.idx, c.vals)
    got, bits = {}, {}
    for name, dt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        Fd = [dev(f, dt) for f in F]
        bits[name] = [host_bits(f) for f in Fd]
        got[name] = [o.cpu().numpy()[rows[m]] for m, o in enumerate(t.mttkrp_all(Fd))]
        del Fd
    t.close()
    torch.cuda.empty_cache()
    ref32 = oracle_rows_all_modes(c, F, rows)
    for name in ("bf16", "f16"):
        import concurrent.futures as cf
        with cf.ThreadPoolExecutor(max_workers=3) as ex:
            futs = [ex.submit(oracle.mttkrp_rows, c.dims, c.idx, c.vals, bits[name], m, rows[m], name)
                    for m in range(3)]
            ref16 = [f.result() for f in futs]
        for m in range(3):
            assert oracle.row_error(got[name][m], ref16[m]) <= FP32_BAR, (name, m)
            assert oracle.row_error(got[name][m], ref32[m]) <= LOWP_BAR, (name, m)


@pytest.mark.slow
def test_planted3_full_size_fused_completion_gradient():
    """The differentiation configuration at full size: 5M x 2M x 1M, 100M nonzeros drawn from
    a planted rank-16 CP model plus N(0, 0.01^2) noise at Zipf positions, R=32 fp32 factors.
    The fused loss against the oracle's over all 100M nonzeros, and 2048 seeded gradient rows
    per mode (plus the 16 hottest) against the oracle's MTTKRP of its own residuals."""
    import concurrent.futures as cf
    w = synth.WORKLOADS["planted3"]
    c = synth.make(w)
    chunks = np.array_split(np.arange(c.nnz), 16)

    def sample(F):  # the oracle's sampled model over all nonzeros, in parallel slices
        with cf.ThreadPoolExecutor(max_workers=16) as ex:
            return np.concatenate(list(ex.map(lambda ix: oracle.cp_sample(c.dims, c.idx[ix], F), chunks)))
    x = (sample(c.extra["planted_factors"]) + c.extra["noise"]).astype(np.float32)
    F = synth.factors(c.dims, 32, w.seed, scale=w.factor_scale)
    t = amped.Tensor(c.dims, c.idx, x)
    grads, loss = t.completion_grad([dev(f) for f in F])
    rows = [sampled_rows(c, m, 2048, w.seed) for m in range(3)]
    got = [g.cpu().numpy()[rows[m]] for m, g in enumerate(grads)]
    loss = loss.item()
    del grads
    t.close()
    torch.cuda.empty_cache()
    r = sample(F) - x.astype(np.float64)  # the oracle's residuals
    assert loss == pytest.approx(oracle.completion_loss(r + x, x), rel=1e-5)
    with cf.ThreadPoolExecutor(max_workers=3) as ex:
        futs = [ex.submit(oracle.mttkrp_rows, c.dims, c.idx, r, F, m, rows[m]) for m in range(3)]
        refs = [f.result() for f in futs]
    for m in range(3):
        assert oracle.row_error(got[m], refs[m], floor_frac=1e-6) <= GRAD_BAR, m


@pytest.mark.parametrize("nmodes", [3, 4])
@pytest.mark.parametrize("runs", ["long", "short", "duplicates"])
@pytest.mark.parametrize("items", [0, 300])
@pytest.mark.parametrize("dt,R", [(torch.float32, 32), (torch.bfloat16, 32), (torch.float16, 32),
                                  (torch.bfloat16, 64)])
def test_factored_path_run_structures(nmodes, runs, items, dt, R):
    """Rows long enough for whole 128-nonzero batches (the factored path: outer slots gathered
    at run starts, innermost per nonzero) with controlled runs of the leading coordinates: long
    runs (few distinct leading values), runs of length one (every nonzero starts new runs), and
    repeated full coordinates; rows end inside batches and, with 300-item segments, rows span
    segments.  fp32 factors against the oracle; 16-bit factors (16 ranks per lane: 16 lane
    groups at R = 32, 8 at R = 64) against the oracle on the same rounded factors."""
    rng = np.random.default_rng(31 + nmodes)
    dims = (40, 300, 200, 150)[:nmodes]
    rows = [3, 17, 29]  # three long output rows of mode 0, plus scattered short rows
    lens = [2000, 777, 131]
    parts = []
    for r, n in zip(rows, lens):
        c = np.zeros((n, nmodes), np.int32)
        c[:, 0] = r
        for m in range(1, nmodes):
            if runs == "long":
                c[:, m] = rng.integers(0, 4, n)
            elif runs == "short":
                c[:, m] = rng.permutation(np.arange(n) % dims[m])
            else:
                c[:, m] = rng.integers(0, 3, n)
        parts.append(c)
    short = np.stack([rng.integers(0, d, 500) for d in dims], axis=1).astype(np.int32)
    idx = np.concatenate(parts + [short])
    idx = idx[rng.permutation(len(idx))]
    vals = rng.uniform(0, 1, len(idx)).astype(np.float32)
    F = [rng.uniform(0, 1, (d, R)).astype(np.float32) for d in dims]
    t = amped.Tensor(dims, idx, vals, segment_items=items)
    Fd = [dev(f, dt) for f in F]
    outs = t.mttkrp_all(Fd)
    torch.cuda.synchronize()
    if dt == torch.float32:
        Fo, kind = F, "f32"
    else:
        Fo, kind = [host_bits(f) for f in Fd], ("bf16" if dt == torch.bfloat16 else "f16")
    for m in range(nmodes):
        ref = oracle.mttkrp(dims, idx, vals, Fo, m, kind)
        assert oracle.row_error(outs[m].cpu().numpy(), ref) <= FP32_BAR, (m, runs, kind)
    t.close()
