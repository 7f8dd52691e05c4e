"""Learned shrinkage: the FP64 oracle against finite differences (CPU), and the GPU
training and inference kernels against the oracle (GPU)."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from oracle import shearlet_oracle as O
from paper_1402_5670_b300 import synth
from tests.conftest import oracle_system


def _random_problem(ndim, seed=0):
    dims = (16, 16) if ndim == 2 else (8, 8, 8)
    R = 7
    r = np.random.default_rng(seed)
    C = r.standard_normal((R,) + dims) * 3.0
    Cc = C * (np.abs(C) > 2.0)
    s = r.uniform(0.5, 2.0, R)
    n = 40
    j = r.integers(1, R, n)
    m = np.stack([r.integers(0, d, n) for d in dims], 1)
    p = M.unflatten(synth.mlp_init(ndim, R, seed).astype(np.float64), ndim, R)
    p["b1"] = r.standard_normal(64) * 0.1
    p["b2"] = r.standard_normal(64) * 0.1
    return p, C, Cc, s, j, m


@pytest.mark.parametrize("ndim", [2, 3])
def test_oracle_gradients_match_finite_differences(ndim):
    """The analytic backward pass of the oracle equals central differences of its loss
    (FP64), for every parameter tensor including the subband embedding, which enters
    through the features."""
    p, C, Cc, s, j, m = _random_problem(ndim)
    c = C[(j,) + tuple(m.T)]
    cc = Cc[(j,) + tuple(m.T)]

    def loss_of(pp):
        return M.loss(pp, M.features(C, j, m, s, pp["E"]), c, cc, s[j])

    L, g = M.backward(p, M.features(C, j, m, s, p["E"]), c, cc, s[j], j)
    assert abs(loss_of(p) - L) < 1e-12
    r = np.random.default_rng(1)
    h = 1e-6
    for k in M.ORDER:
        flat = p[k].ravel()
        for i in r.choice(flat.size, min(6, flat.size), replace=False):
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k].ravel()[i] += h
            Lp = loss_of(q)
            q[k].ravel()[i] -= 2 * h
            Lm = loss_of(q)
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[k].ravel()[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, i)


def test_pin_catches_wrong_relu_derivative():
    """Planted mistake: the ReLU derivative taken as 1 everywhere (gradient flowing
    through inactive units). Finite differences of the loss separate it from the
    oracle's gradient."""
    p, C, Cc, s, j, m = _random_problem(2)
    c = C[(j,) + tuple(m.T)]
    cc = Cc[(j,) + tuple(m.T)]
    X = M.features(C, j, m, s, p["E"])
    L, g = M.backward(p, X, c, cc, s[j], j)
    gv, _ = M.forward(p, X)
    dz3 = 2 * (gv * c - cc) / s[j] * c / s[j] / len(c) * gv * (1 - gv)
    wrong_b2 = np.outer(dz3, p["w3"]).sum(0)
    h = 1e-6
    fd = np.zeros(64)
    for i in range(64):
        q = {kk: vv.copy() for kk, vv in p.items()}
        q["b2"][i] += h
        Lp = M.loss(q, X, c, cc, s[j])
        q["b2"][i] -= 2 * h
        fd[i] = (Lp - M.loss(q, X, c, cc, s[j])) / (2 * h)
    assert np.max(np.abs(g["b2"] - fd)) < 1e-8
    assert np.max(np.abs(wrong_b2 - fd)) > 1e-6


def test_features_neighbourhood_order():
    """x_1..x_9 are |C| over the 3x3 neighbourhood in row-major order with periodic
    wrap, scaled by 1/s; x_0 is the signed centre."""
    C = np.zeros((2, 4, 5))
    C[1] = np.arange(20).reshape(4, 5) - 7.0
    E = np.zeros((2, 8))
    X = M.features(C, np.array([1]), np.array([[0, 0]]), np.array([1.0, 2.0]), E)
    want = [C[1, 0, 0] / 2] + [abs(C[1, a % 4, b % 5]) / 2 for a in (-1, 0, 1) for b in (-1, 0, 1)]
    assert np.allclose(X[0, :10], want)


def test_bf16_rounding_is_round_to_nearest_even():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.14159])
    assert list(M.bf16(v)) == [1.0, 1.0, 1.0 + 2 ** -6, -2.5, 3.140625]


# ------------------------------------------------------------------- GPU ---

torch = pytest.importorskip("torch")


def _gpu_setup(dims, J, sl, seed):
    from paper_1402_5670_b300.build import build
    from paper_1402_5670_b300.shearlet import MLP, Bank
    build()
    b = Bank(dims, J, sl, device=0)
    clean = (synth.piecewise_smooth_image(dims, seed) if len(dims) == 2
             else synth.moving_ellipses_volume(dims, seed))
    noisy = synth.add_noise(clean, 20.0, seed + 1)
    Cn = b.forward(torch.from_numpy(noisy).cuda())
    Cc = b.forward(torch.from_numpy(clean).cuda())
    mlp = MLP(b)
    flat = synth.mlp_init(len(dims), b.R, seed + 2)
    mlp.set_params(flat)
    return b, mlp, flat, Cn, Cc


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


@pytest.mark.gpu
@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync"])
@pytest.mark.parametrize("case", [((64, 64), 2, (1, 1)), ((16, 16, 16), 1, (0,))], ids=str)
def test_gpu_gradients_match_oracle(case, engine):
    """The tensor-core backward pass against the oracle: within 1e-2 of the oracle with
    the same BF16 operand rounding (FP32 vs FP64 accumulation, rare rounding-boundary
    flips), and within 5e-2 of the exact FP64 gradients (the BF16 effect itself). The
    tcgen05 engine also rounds the operands of the bias and w3 sums (dz2, dz1, h2, dz3)
    to BF16, inside the same bounds."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dims, J, sl = case
    b, mlp, flat, Cn, Cc = _gpu_setup(dims, J, sl, 3)
    mlp.set_engine(engine)
    s_sys = oracle_system(dims, J, sl)
    r = np.random.default_rng(5)
    n = 2048
    q = r.integers(b.N, b.R * b.N, n)
    idx = torch.from_numpy(q.astype(np.int32)).cuda()
    sigma = 20.0
    L_gpu, g_gpu = mlp.gradients(Cn, Cc, sigma, idx)
    C = Cn.cpu().numpy().astype(np.float64)
    CC = Cc.cpu().numpy().astype(np.float64)
    j = q // b.N
    m = np.stack(np.unravel_index(q % b.N, dims), 1)
    s = sigma * s_sys.norms
    p = M.unflatten(flat.astype(np.float64), len(dims), b.R)
    X = M.features(C, j, m, s, p["E"])
    c = C[(j,) + tuple(m.T)]
    cc = CC[(j,) + tuple(m.T)]
    L_q, g_q = M.backward(p, X, c, cc, s[j], j, bf16_operands=True)
    L_x, g_x = M.backward(p, X, c, cc, s[j], j)
    gq, gx = M.flatten(g_q), M.flatten(g_x)
    assert abs(L_gpu - L_q) <= 1e-3 * L_q
    off = 0
    for k, sh in M.param_shapes(len(dims), b.R).items():
        sz = int(np.prod(sh))
        e1 = _rel(g_gpu[off:off + sz], gq[off:off + sz])
        e2 = _rel(g_gpu[off:off + sz], gx[off:off + sz])
        assert e1 < 1e-2, (k, e1)
        assert e2 < 5e-2, (k, e2)
        off += sz
    mlp.check()


@pytest.mark.gpu
def test_training_engines_agree_and_descend():
    """Thirty Adam steps from the same start on the same samples (65,536 per step, 512
    tiles: several per CTA): the tcgen05 and mma.sync engines give parameters within
    2e-2 of each other (relative L2 per tensor; BF16 products summed in other orders),
    and both lower the loss."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dims, J, sl = (256, 256), 3, (1, 1, 2)
    b, mlp, flat, Cn, Cc = _gpu_setup(dims, J, sl, 4)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(9)
    idxs = [(torch.randint(0, (b.R - 1) * b.N, (65536,), generator=gen, device="cuda")
             + b.N).to(torch.int32) for _ in range(30)]
    out = {}
    for engine in ("tcgen05", "mma_sync"):
        mlp.set_params(flat)
        mlp.set_engine(engine)
        loss = torch.zeros(1, device="cuda")
        hist = []
        for idx in idxs:
            mlp.train_step(Cn, Cc, 20.0, idx, 2e-3, loss_out=loss)
            hist.append(float(loss.item()))
        mlp.check()
        assert hist[-1] < 0.9 * hist[0], (engine, hist[0], hist[-1])
        out[engine] = mlp.get_params().astype(np.float64)
    off = 0
    for k, sh in M.param_shapes(2, b.R).items():
        sz = int(np.prod(sh))
        a_, c_ = out["tcgen05"][off:off + sz], out["mma_sync"][off:off + sz]
        assert _rel(a_, c_) < 2e-2, (k, _rel(a_, c_))
        off += sz


@pytest.mark.gpu
def test_training_wait_timeout_is_reported_and_recovers(monkeypatch):
    """The tcgen05 trainer's bounded waits, made to run out at once (SL_MLP_WAIT_CYCLES=0,
    a test hook): the call returns, sl_mlp_check reports the flag and clears it, and
    the next call with the normal limit gives the gradients from before, exactly except
    for the embedding's (summed with shared-memory atomics in any order) to 1e-6."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5670_b300.shearlet import ShearletError
    dims, J, sl = (64, 64), 2, (1, 1)
    b, mlp, flat, Cn, Cc = _gpu_setup(dims, J, sl, 7)
    mlp.set_engine("tcgen05")
    r = np.random.default_rng(3)
    idx = torch.from_numpy(r.integers(b.N, b.R * b.N, 1024).astype(np.int32)).cuda()
    L0, g0 = mlp.gradients(Cn, Cc, 20.0, idx)
    mlp.check()
    monkeypatch.setenv("SL_MLP_WAIT_CYCLES", "0")
    mlp.gradients(Cn, Cc, 20.0, idx)
    with pytest.raises(ShearletError):
        mlp.check()
    monkeypatch.delenv("SL_MLP_WAIT_CYCLES")
    mlp.check()  # the flag was cleared
    L1, g1 = mlp.gradients(Cn, Cc, 20.0, idx)
    mlp.check()
    nE = b.R * M.EMBED
    assert L1 == L0
    assert np.array_equal(g1[:-nE], g0[:-nE])
    assert _rel(g1[-nE:], g0[-nE:]) < 1e-6


@pytest.mark.gpu
@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync"])
@pytest.mark.parametrize("case", [((64, 64), 2, (1, 1)), ((16, 16, 16), 1, (0,))], ids=str)
def test_gpu_apply_matches_oracle(case, engine):
    """Inference on both engines (tcgen05 tiles of 128 rows with TMEM accumulators,
    and warp-level mma.sync) against the oracle with the same BF16 operand rounding.
    Supported sizes make (R - 1) N a multiple of 128, so every tcgen05 tile is full."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dims, J, sl = case
    b, mlp, flat, Cn, Cc = _gpu_setup(dims, J, sl, 4)
    mlp.set_engine(engine)
    s_sys = oracle_system(dims, J, sl)
    out = mlp.apply(Cn, 20.0)
    mlp.check()
    out = out.cpu().numpy()
    p = M.unflatten(flat.astype(np.float64), len(dims), b.R)
    ref = M.apply(p, Cn.cpu().numpy().astype(np.float64), 20.0 * s_sys.norms, bf16_operands=True)
    assert np.array_equal(out[0], Cn[0].cpu().numpy())
    assert np.max(np.abs(out - ref)) <= 2e-3 * np.max(np.abs(ref))


@pytest.mark.gpu
def test_gpu_apply_engines_agree_at_full_size():
    """512^2, 49 subbands: the two engines agree coefficient by coefficient (same BF16
    operands, FP32 sums in another order), and sampled coefficients match the oracle
    computed one by one."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dims, J, sl = (512, 512), 4, (1, 1, 2, 2)
    b, mlp, flat, Cn, Cc = _gpu_setup(dims, J, sl, 6)
    mlp.set_engine("tcgen05")
    a = mlp.apply(Cn, 20.0)
    mlp.check()
    mlp.set_engine("mma_sync")
    m = mlp.apply(Cn, 20.0)
    torch.cuda.synchronize()
    scale = float(Cn.abs().max())
    assert float((a - m).abs().max()) <= 2e-3 * scale
    assert torch.equal(a[0], Cn[0])
    s_sys = oracle_system(dims, J, sl)
    r = np.random.default_rng(9)
    q = r.integers(b.N, b.R * b.N, 4096)
    j = q // b.N
    mm = np.stack(np.unravel_index(q % b.N, dims), 1)
    p = M.unflatten(flat.astype(np.float64), 2, b.R)
    C = Cn.cpu().numpy().astype(np.float64)
    s = 20.0 * s_sys.norms
    X = M.features(C, j, mm, s, p["E"])
    g, _ = M.forward(p, X, bf16_operands=True)
    want = g * C[(j,) + tuple(mm.T)]
    got = a.cpu().numpy()[(j,) + tuple(mm.T)]
    assert np.max(np.abs(got - want)) <= 2e-3 * scale


@pytest.mark.gpu
def test_apply_in_a_graph_follows_parameter_updates():
    """A CUDA graph that captured sl_mlp_apply repacks the tcgen05 weight tiles at
    every replay, so a parameter update between replays is seen, bit for bit as an
    eager call with the new parameters."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dims, J, sl = (64, 64), 2, (1, 1)
    b, mlp, flat, Cn, Cc = _gpu_setup(dims, J, sl, 5)
    out = torch.empty_like(Cn)
    mlp.apply(Cn, 20.0, out=out)  # packs on the current stream first
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        mlp.apply(Cn, 20.0, out=out)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, mlp.apply(Cn, 20.0))
    mlp.set_params(0.5 * flat)
    g.replay()
    torch.cuda.synchronize()
    want = mlp.apply(Cn, 20.0)
    mlp.check()
    assert torch.equal(out, want)
    assert not torch.equal(want[1:], Cn[1:])


@pytest.mark.gpu
def test_tensor_core_wait_timeout_is_reported_and_recovers(monkeypatch):
    """The bounded tensor-core waits of the tcgen05 engine, made to run out at once
    (SL_MLP_WAIT_CYCLES=0, a test hook): the call returns, sl_mlp_check reports the
    flag (and clears it), and the next call with the normal limit matches the
    result from before bit for bit. Nothing here faults or hangs: the kernel drains
    the MMAs it issued, with the normal limit, before it frees tensor memory."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5670_b300.shearlet import ShearletError
    dims, J, sl = (64, 64), 2, (1, 1)
    b, mlp, flat, Cn, Cc = _gpu_setup(dims, J, sl, 7)
    mlp.set_engine("tcgen05")
    ref = mlp.apply(Cn, 20.0).clone()
    mlp.check()
    monkeypatch.setenv("SL_MLP_WAIT_CYCLES", "0")
    mlp.apply(Cn, 20.0)
    with pytest.raises(ShearletError):
        mlp.check()
    monkeypatch.delenv("SL_MLP_WAIT_CYCLES")
    mlp.check()  # the flag was cleared
    again = mlp.apply(Cn, 20.0)
    mlp.check()
    assert torch.equal(again, ref)


@pytest.mark.gpu
def test_learned_shrinkage_beats_hard_thresholding():
    """Trained on the GPU from transform-generated pairs (20,000 Adam steps of 65,536
    samples on 12 cartoons x 4 noise levels), the learned gain must denoise held-out
    synthetic images better (PSNR) than the paper's hard threshold at every tested
    noise level: each gain above 0.08 dB and their mean above 0.2 dB (measured on a
    B300: 0.16 to 0.41 dB, mean 0.28)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5670_b300 import learned
    from paper_1402_5670_b300.shearlet import MLP, Bank
    dims, J, sl = (256, 256), 2, (1, 1)
    b = Bank(dims, J, sl, device=0)
    mlp = MLP(b)
    mlp.set_params(synth.mlp_init(2, b.R, 11))
    pairs = learned.make_pairs(b, [10.0, 20.0, 30.0, 40.0], seeds=list(range(100, 112)))
    hist = learned.train(mlp, pairs, steps=20000, batch=65536, lr=2e-3, seed=1)
    assert hist[-1] < hist[0]
    K = [2.5, 3.8]
    gains = []
    for sg in (10.0, 20.0, 30.0, 40.0):
        for sd in (500, 501):
            clean = synth.piecewise_smooth_image(dims, sd)
            noisy = synth.add_noise(clean, sg, sd + 9)
            xg = torch.from_numpy(noisy).cuda()
            hard = b.denoise(xg, sg, K).cpu().numpy()
            lrn = mlp.denoise(xg, sg).cpu().numpy()
            gains.append(O.psnr(clean, lrn) - O.psnr(clean, hard))
    print("PSNR gain of learned over hard thresholding (dB):", np.round(gains, 2))
    assert min(gains) > 0.08
    assert float(np.mean(gains)) > 0.2


@pytest.mark.gpu
def test_checkpoint_resume(tmp_path):
    """Save after 3 Adam steps, keep training; a fresh MLP loaded from the checkpoint
    holds the same parameters and continues to the same place (up to the summation
    order of the gradient reduction); a checkpoint of another shape is refused."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5670_b300.shearlet import MLP, Bank, ShearletError
    dims, J, sl = (64, 64), 2, (1, 1)
    b, mlp, flat, Cn, Cc = _gpu_setup(dims, J, sl, 6)
    r = np.random.default_rng(7)
    idxs = [torch.from_numpy(r.integers(b.N, b.R * b.N, 1024).astype(np.int32)).cuda()
            for _ in range(5)]
    for i in range(3):
        mlp.train_step(Cn, Cc, 20.0, idxs[i], 1e-3)
    ck = str(tmp_path / "mlp.ckpt")
    mlp.save(ck)
    saved = mlp.get_params()
    for i in range(3, 5):
        mlp.train_step(Cn, Cc, 20.0, idxs[i], 1e-3)
    after = mlp.get_params()
    m2 = MLP(b)
    m2.load(ck)
    assert np.array_equal(m2.get_params(), saved)
    for i in range(3, 5):
        m2.train_step(Cn, Cc, 20.0, idxs[i], 1e-3)
    assert np.max(np.abs(m2.get_params() - after)) <= 1e-5 * np.max(np.abs(after))
    assert not np.allclose(after, saved)
    b2 = Bank((32, 32), 1, (0,), device=0)
    m3 = MLP(b2)
    with pytest.raises(ShearletError):
        m3.load(ck)
    with pytest.raises(ShearletError):
        m3.load(str(tmp_path / "missing.ckpt"))
