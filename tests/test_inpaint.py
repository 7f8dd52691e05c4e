"""Image inpainting by iterative thresholding (Sec. 5.4) through sl_inpaint.

Every step is one elementwise pass and one fused denoise, so the GPU result is
compared bit for bit with the same steps issued one by one through sl_denoise, and
with the FP64 oracle by image quality and to 1e-3 after a few iterations (threshold
decisions near delta are taken in FP32 on the GPU and in FP64 by the oracle, so single
coefficients may be kept on one side and zeroed on the other; that bounds the
agreement, not the transform's 1e-5).
"""
import numpy as np
import pytest

from oracle import shearlet_oracle as O
from paper_1402_5670_b300 import synth
from tests.conftest import oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5670_b300.build import build
    build()


def setup(dims, J, sl, missing, seed):
    from paper_1402_5670_b300.shearlet import Bank
    b = Bank(dims, J, sl, device=0)
    f = synth.piecewise_smooth_image(dims, seed)
    M = synth.random_mask(dims, missing, seed + 1)
    fm = torch.from_numpy(f * M).cuda()
    Mg = torch.from_numpy(M).cuda()
    return b, f, M, fm, Mg


def manual(b, fm, Mg, d0, d1, iters):
    """The algorithm's steps issued one by one (the mix in torch, the step's
    transform-threshold-synthesis through sl_denoise)."""
    lam = (d1 / d0) ** (1.0 / (iters - 1)) if iters > 1 else 1.0
    out = torch.zeros_like(fm)
    delta = d0
    ones = [1.0] * b.n_scales
    for _ in range(iters):
        u = torch.where(Mg > 0, fm, out)
        out = b.denoise(u, float(np.float32(delta)), ones)
        delta *= lam
    return out


def test_inpaint_equals_its_steps():
    b, f, M, fm, Mg = setup((128, 128), 3, (1, 1, 2), 0.5, 3)
    for iters in (1, 5):
        got = b.inpaint(fm, Mg, 150.0, 5.0, iters)
        want = manual(b, fm, Mg, 150.0, 5.0, iters)
        torch.cuda.synchronize()
        assert torch.equal(got, want), iters


def test_inpaint_matches_oracle():
    dims, J, sl = (64, 64), 3, (0, 1, 1)
    b, f, M, fm, Mg = setup(dims, J, sl, 0.6, 7)
    s = oracle_system(dims, J, sl)
    ref = O.inpaint((f * M).astype(np.float64), M, s, 200.0, 2.0, 4)
    got = b.inpaint(fm, Mg, 200.0, 2.0, 4).cpu().numpy()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-3
    ref30 = O.inpaint((f * M).astype(np.float64), M, s, 200.0, 2.0, 30)
    got30 = b.inpaint(fm, Mg, 200.0, 2.0, 30).cpu().numpy()
    assert abs(O.psnr(f, got30) - O.psnr(f, ref30)) < 0.1
    assert O.psnr(f, got30) > O.psnr(f, f * M) + 10.0


def test_inpaint_full_size_random80():
    """512^2, 49 filters, 80% of the pixels occluded at random (the paper's Random
    mask), 60 iterations: the holes are filled."""
    b, f, M, fm, Mg = setup((512, 512), 4, (1, 1, 2, 2), 0.8, 11)
    out = b.inpaint(fm, Mg, 300.0, 3.0, 60).cpu().numpy()
    mean_fill = np.where(M > 0, f, np.mean(f[M > 0]))
    assert O.psnr(f, out) > O.psnr(f, mean_fill) + 3.0
    assert np.all(np.isfinite(out))


def test_inpaint_rejects_bad_arguments():
    from paper_1402_5670_b300 import shearlet as S
    b, f, M, fm, Mg = setup((64, 64), 2, (1, 1), 0.5, 1)
    out = torch.empty_like(fm)
    L = S.lib()
    assert S.STATUS[L.sl_inpaint(b.handle, fm.data_ptr(), Mg.data_ptr(), out.data_ptr(),
                                 10.0, 1.0, 0, None)] == "SL_EINVAL"
    assert S.STATUS[L.sl_inpaint(b.handle, fm.data_ptr(), Mg.data_ptr(), out.data_ptr(),
                                 0.0, 1.0, 3, None)] == "SL_EINVAL"
    assert S.STATUS[L.sl_inpaint(b.handle, fm.data_ptr(), Mg.data_ptr(), fm.data_ptr(),
                                 10.0, 1.0, 3, None)] == "SL_EINVAL"
    mbuf = torch.zeros(b.N + 16, dtype=torch.uint8, device="cuda")
    assert S.STATUS[L.sl_inpaint(b.handle, fm.data_ptr(), mbuf.data_ptr() + 1, out.data_ptr(),
                                 10.0, 1.0, 3, None)] == "SL_EINVAL"
    torch.cuda.synchronize()


def test_inpaint_3d_volume():
    """The same iteration on a 3D bank (Sec. 5.7 uses it for videos): equal to its
    steps, close to the oracle after a few iterations, and it fills the holes."""
    from paper_1402_5670_b300.shearlet import Bank
    dims, J, sl = (16, 16, 16), 2, (0, 1)
    b = Bank(dims, J, sl, device=0)
    f = synth.moving_ellipses_volume(dims, 21)
    M = synth.random_mask(dims, 0.5, 22)
    fm = torch.from_numpy(f * M).cuda()
    Mg = torch.from_numpy(M).cuda()
    got = b.inpaint(fm, Mg, 100.0, 2.0, 4)
    torch.cuda.synchronize()
    assert torch.equal(got, manual(b, fm, Mg, 100.0, 2.0, 4))
    s = oracle_system(dims, J, sl)
    ref = O.inpaint((f * M).astype(np.float64), M, s, 100.0, 2.0, 4)
    g = got.cpu().numpy()
    assert np.max(np.abs(g - ref)) / np.max(np.abs(ref)) < 1e-3
    g20 = b.inpaint(fm, Mg, 100.0, 2.0, 20).cpu().numpy()
    assert O.psnr(f, g20) > O.psnr(f, f * M) + 10.0
