"""Mixed-radix sizes (384 = 3 * 2^7) and batched runs of images of uneven shapes.

384-sided grids are compared with the FP64 oracle like every other size (1e-5
relative). A batch computes, per image, exactly what the single-image calls compute
(the same kernels and launch shapes, only a different scratch buffer), so batch
results are compared with single-image results bit for bit, and at full size with
the oracle on one image of every distinct shape.
"""
import numpy as np
import pytest

from oracle import shearlet_oracle as O
from paper_1402_5670_b300 import synth
from tests.conftest import oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5670_b300.build import build
    build()


_BANKS = {}


def bank(dims, J, sl):
    from paper_1402_5670_b300.shearlet import Bank
    key = (tuple(dims), J, tuple(sl))
    if key not in _BANKS:
        _BANKS[key] = Bank(dims, J, sl, device=0)
    return _BANKS[key]


def image(dims, seed):
    return synth.add_noise(synth.piecewise_smooth_image(dims, seed), 20.0, seed + 1000)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


# ------------------------------------------------------------- 384 grids ---

CASES_384 = [((384, 64), 2, (1, 1)), ((64, 384), 2, (1, 1)), ((384, 128), 3, (1, 1, 2)),
             ((384, 384), 4, (1, 1, 2, 2))]


@pytest.mark.parametrize("case", CASES_384, ids=str)
def test_384_matches_oracle(case):
    """Mixed radix (radix-3 step in the register DFTs) along either axis."""
    dims, J, sl = case
    b = bank(dims, J, sl)
    s = oracle_system(dims, J, sl)
    x = image(dims, 1)
    C = b.forward(cuda(x))
    assert rel(C.cpu().numpy(), O.forward(x.astype(np.float64), s)) < TOL
    Cf = C.cpu().numpy().astype(np.float64)
    xi = b.inverse(C).cpu().numpy()
    assert rel(xi, O.inverse(Cf, s)) < TOL
    assert rel(xi, x) < TOL
    Cr = synth.gaussian_field((b.R,) + tuple(dims), 2)
    assert rel(b.adjoint(cuda(Cr)).cpu().numpy(), O.adjoint(Cr.astype(np.float64), s)) < TOL


def test_384_denoise_matches_oracle():
    dims, J, sl = (384, 384), 4, (1, 1, 2, 2)
    b = bank(dims, J, sl)
    s = oracle_system(dims, J, sl)
    K = [2.5, 2.5, 2.5, 3.8]
    clean = synth.piecewise_smooth_image(dims, 3)
    noisy = synth.add_noise(clean, 20.0, 4)
    xg = cuda(noisy)
    den = b.denoise(xg, 20.0, K).cpu().numpy()
    Cg = b.forward(xg)
    b.threshold_(Cg, 20.0, K)
    assert rel(den, O.inverse(Cg.cpu().numpy().astype(np.float64), s)) < TOL
    assert O.psnr(clean, den) > O.psnr(clean, noisy) + 5


# --------------------------------------------------------------- batches ---

SMALL_SHAPES = [(64, 64), (384, 64), (128, 128), (64, 384), (64, 64), (128, 128), (32, 32),
                (64, 64)]


def small_batch():
    banks = [bank(d, 2, (1, 1)) for d in SMALL_SHAPES]
    xs = [cuda(image(d, 10 + i)) for i, d in enumerate(SMALL_SHAPES)]
    return banks, xs


def singles(banks, xs):
    cs = [b.forward(x) for b, x in zip(banks, xs)]
    ys = [b.inverse(c) for b, c in zip(banks, cs)]
    return cs, ys


@pytest.mark.parametrize("branches,graph", [(1, True), (3, True), (3, False), (8, True)])
def test_batch_equals_single_calls(branches, graph):
    from paper_1402_5670_b300.shearlet import Batch
    banks, xs = small_batch()
    ref_c, ref_y = singles(banks, xs)
    B = Batch(banks, branches=branches, graph=graph)
    info = B.info()
    assert info["branches"] == min(branches, len(xs))
    assert sorted(set(info["branch_of"])) == list(range(info["branches"]))
    cs = [torch.full_like(c, np.nan) for c in ref_c]
    ys = [torch.full_like(x, np.nan) for x in xs]
    B.forward(xs, cs)
    B.inverse(cs, ys)
    torch.cuda.synchronize()
    for i in range(len(xs)):
        assert torch.equal(cs[i], ref_c[i]), i
        assert torch.equal(ys[i], ref_y[i]), i
    # fused form, twice with the same pointers (graph replay), then new pointers
    ys2 = [torch.full_like(x, np.nan) for x in xs]
    for _ in range(2):
        B.fwdinv(xs, cs, ys2)
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(ys2, ref_y))
    ys3 = [torch.full_like(x, np.nan) for x in xs]
    B.fwdinv(xs, cs, ys3)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(ys3, ref_y))
    B.close()


def test_batch_denoise_equals_single_calls():
    from paper_1402_5670_b300.shearlet import Batch
    banks, xs = small_batch()
    K = [2.5, 3.8]
    ref = [b.denoise(x, 20.0, K) for b, x in zip(banks, xs)]
    B = Batch(banks, branches=4)
    out = [torch.full_like(x, np.nan) for x in xs]
    B.denoise(xs, out, 20.0, K)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(out, ref))
    # new thresholds with the same pointers: the graph is captured again
    ref2 = [b.denoise(x, 30.0, K) for b, x in zip(banks, xs)]
    B.denoise(xs, out, 30.0, K)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(out, ref2))
    B.close()


def test_one_shot_batch_calls():
    from paper_1402_5670_b300.shearlet import sl_forward_batch, sl_inverse_batch
    banks, xs = small_batch()
    ref_c, ref_y = singles(banks, xs)
    cs = [torch.empty_like(c) for c in ref_c]
    ys = [torch.empty_like(x) for x in xs]
    sl_forward_batch(banks, xs, cs)
    sl_inverse_batch(banks, cs, ys)
    assert all(torch.equal(a, b) for a, b in zip(cs, ref_c))
    assert all(torch.equal(a, b) for a, b in zip(ys, ref_y))


def test_autotune_keeps_results():
    from paper_1402_5670_b300.shearlet import Batch
    banks, xs = small_batch()
    _, ref_y = singles(banks, xs)
    B = Batch(banks)
    cs = [torch.empty((b.R,) + b.dims, device="cuda") for b in banks]
    ys = [torch.empty_like(x) for x in xs]
    ms = B.autotune(xs, cs, ys, reps=3)
    assert ms > 0
    info = B.info()
    assert 1 <= info["branches"] <= len(xs)
    B.fwdinv(xs, cs, ys)
    torch.cuda.synchronize()
    # a different group cap changes the order of the partial sums: compare to 1e-5
    for a, b in zip(ys, ref_y):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < TOL
    B.close()


def test_batch_rejects_bad_arguments():
    from paper_1402_5670_b300 import shearlet as S
    banks, xs = small_batch()
    B = S.Batch(banks)
    with pytest.raises(TypeError):
        B.forward(xs[:-1] + [xs[-1].cpu()], [torch.empty(1, device="cuda")] * len(xs))
    with pytest.raises(ValueError):
        B.forward(xs, [torch.empty(1, device="cuda")] * len(xs))
    n = len(banks)
    null = (S._vp * n)()
    st = S.lib().sl_batch_forward(B.handle, null, null, None)
    assert S.STATUS[st] == "SL_EINVAL"
    B.close()


# ------------------------------------------------- the full uneven batch ---

def test_full_uneven_batch_64():
    """64 images, sides drawn from {256, 384, 512, 1024}, four scales, levels
    (1,1,2,2): every image reconstructs to 1e-5 and equals its single-image call;
    one image of each distinct shape is compared with the oracle (sampled subbands)."""
    from paper_1402_5670_b300.shearlet import Batch
    shapes = synth.uneven_batch_shapes(64, (256, 384, 512, 1024), 2024)
    banks = [bank(d, 4, (1, 1, 2, 2)) for d in shapes]
    assert len({b.dims for b in banks}) <= 16
    xs = [cuda(image(d, 100 + i)) for i, d in enumerate(shapes)]
    cs = [torch.empty((b.R,) + b.dims, device="cuda") for b in banks]
    ys = [torch.empty_like(x) for x in xs]
    B = Batch(banks)
    B.fwdinv(xs, cs, ys)
    torch.cuda.synchronize()
    seen = set()
    for i, (b, x) in enumerate(zip(banks, xs)):
        assert rel(ys[i].cpu().numpy(), x.cpu().numpy()) < TOL, i
        if b.dims in seen:
            continue
        seen.add(b.dims)
        assert torch.equal(cs[i], b.forward(x)), i
        s = oracle_system(b.dims, 4, (1, 1, 2, 2))
        ref = O.forward_subset(x.cpu().numpy().astype(np.float64), s, (0, 9, 24, 48))
        for j, r in ref.items():
            assert rel(cs[i][j].cpu().numpy(), r) < TOL, (i, j)  # against its own size
    B.close()
