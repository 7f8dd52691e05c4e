"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: 1e-5 relative (max-abs error over max-abs reference, per output array),
the FP32 target of the transform. Threshold decisions are taken in FP32 on both sides
(bit-exact); denoising is compared both against the oracle's inverse of the GPU's own
FP32-thresholded coefficients and, by PSNR, against the oracle's full denoiser.
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


def bank(dims, J, sl, full=False, path="general"):
    from paper_1402_5670_b300.shearlet import Bank
    key = (tuple(dims), J, tuple(sl), full, path)
    if key not in _BANKS:
        _BANKS[key] = Bank(dims, J, sl, full, device=0, path=path)
        assert _BANKS[key].kernel_path == path
    return _BANKS[key]


def signal(dims, seed):
    if len(dims) == 2:
        x = synth.piecewise_smooth_image(dims, seed)
    else:
        x = synth.moving_ellipses_volume(dims, seed)
    return synth.add_noise(x, 20.0, seed + 100)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


CASES_2D = [((16, 16), 1, (1,)), ((32, 32), 2, (0, 1)), ((64, 32), 2, (1, 1)),
            ((32, 128), 2, (1, 2)), ((128, 256), 3, (1, 1, 2)), ((256, 256), 2, (1, 1)),
            ((8, 8), 1, (0,)), ((1024, 64), 2, (1, 1)), ((64, 64), 2, (2, 3))]
CASES_3D = [((8, 8, 8), 1, (0,)), ((16, 16, 16), 2, (0, 1)), ((32, 16, 8), 2, (1, 1)),
            ((16, 32, 64), 2, (1, 1)), ((64, 64, 64), 3, (0, 0, 1)),
            ((16, 192, 192), 2, (0, 1)), ((192, 32, 16), 2, (1, 1)), ((32, 32, 32), 2, (1, 2))]
CASES = CASES_2D + CASES_3D


@pytest.mark.parametrize("case", CASES, ids=str)
def test_forward_matches_oracle(case):
    dims, J, sl = case
    b = bank(dims, J, sl)
    s = oracle_system(dims, J, sl)
    x = signal(dims, 1)
    C = b.forward(cuda(x)).cpu().numpy()
    ref = O.forward(x.astype(np.float64), s)
    assert rel(C, ref) < TOL
    for j in range(b.R):
        assert rel(C[j], ref[j]) < TOL, j  # every subband against its own size


@pytest.mark.parametrize("case", CASES, ids=str)
def test_inverse_and_adjoint_match_oracle(case):
    dims, J, sl = case
    b = bank(dims, J, sl)
    s = oracle_system(dims, J, sl)
    x = signal(dims, 2)
    C = O.forward(x.astype(np.float64), s).astype(np.float32)
    Cg = cuda(C)
    xi = b.inverse(Cg).cpu().numpy()
    assert rel(xi, O.inverse(C.astype(np.float64), s)) < TOL
    assert rel(xi, x) < TOL  # perfect reconstruction from FP32 coefficients
    Cr = synth.gaussian_field((b.R,) + tuple(dims), 3)
    xa = b.adjoint(cuda(Cr)).cpu().numpy()
    assert rel(xa, O.adjoint(Cr.astype(np.float64), s)) < TOL


@pytest.mark.parametrize("case", [CASES_2D[2], CASES_2D[5], CASES_3D[1]], ids=str)
def test_threshold_bit_exact(case):
    dims, J, sl = case
    b = bank(dims, J, sl)
    s = oracle_system(dims, J, sl)
    K = [2.5] * (J - 1) + [3.8]
    x = signal(dims, 4)
    C = O.forward(x.astype(np.float64), s).astype(np.float32)
    Cg = cuda(C)
    b.threshold_(Cg, 20.0, K)
    ref = O.threshold(C, s, 20.0, K, dtype=np.float32)
    assert np.array_equal(Cg.cpu().numpy(), ref.astype(np.float32))


@pytest.mark.parametrize("case", [CASES_2D[2], CASES_2D[5], CASES_3D[1], CASES_3D[2],
                                  CASES_3D[5]], ids=str)
def test_denoise_fused_matches_oracle(case):
    dims, J, sl = case
    b = bank(dims, J, sl)
    s = oracle_system(dims, J, sl)
    K = [2.5] * (J - 1) + [3.8]
    clean = (synth.piecewise_smooth_image(dims, 5) if len(dims) == 2
             else synth.moving_ellipses_volume(dims, 5))
    noisy = synth.add_noise(clean, 20.0, 6)
    xg = cuda(noisy)
    den = b.denoise(xg, 20.0, K).cpu().numpy()
    # same FP32 decisions as the GPU: threshold the GPU's own coefficients
    Cg = b.forward(xg)
    b.threshold_(Cg, 20.0, K)
    ref = O.inverse(Cg.cpu().numpy().astype(np.float64), s)
    assert rel(den, ref) < TOL
    # against the oracle's own FP64 denoiser: the same image quality
    full = O.denoise(noisy.astype(np.float64), s, 20.0, K)
    assert abs(O.psnr(clean, den) - O.psnr(clean, full)) < 0.01
    assert O.psnr(clean, den) > O.psnr(clean, noisy)


@pytest.mark.parametrize("path", ["general", "cluster"])
def test_fwdinv_host_round_trip(path):
    dims = (256, 256)
    b = bank(dims, 2, (1, 1), path=path)
    x = signal(dims, 7)
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    b.fwdinv_host(xh, yh)
    torch.cuda.synchronize()
    dev = b.inverse(b.forward(cuda(x))).cpu().numpy()
    assert np.array_equal(yh.numpy(), dev)
    assert rel(yh.numpy(), x) < TOL


def test_zero_and_constant_inputs():
    dims = (64, 64)
    b = bank(dims, 3, (0, 1, 1))
    z = torch.zeros(dims, device="cuda")
    assert float(b.forward(z).abs().max()) == 0.0
    c = torch.full(dims, 7.0, device="cuda")
    C = b.forward(c)
    s = oracle_system(dims, 3, (0, 1, 1))
    assert rel(C.cpu().numpy(), O.forward(np.full(dims, 7.0), s)) < TOL
    assert rel(b.inverse(C).cpu().numpy(), np.full(dims, 7.0)) < TOL


def test_full_system_variant():
    dims, J, sl = (64, 64), 2, (1, 2)
    b = bank(dims, J, sl, True)
    s = oracle_system(dims, J, sl, True)
    x = signal(dims, 8)
    C = b.forward(cuda(x)).cpu().numpy()
    assert rel(C, O.forward(x.astype(np.float64), s)) < TOL
    assert rel(b.inverse(cuda(C)).cpu().numpy(), x) < TOL


def test_repeated_calls_are_deterministic():
    dims = (128, 256)
    b = bank(dims, 3, (1, 1, 2))
    xg = cuda(signal(dims, 9))
    C1 = b.forward(xg).clone()
    C2 = b.forward(xg)
    assert torch.equal(C1, C2)
    assert torch.equal(b.inverse(C1), b.inverse(C2))


# ----------------------------------------------- cluster-fused 2D path ---

CLUSTER_CASES = [((64, 64), 2, (1, 1)), ((128, 256), 3, (1, 1, 2)), ((256, 128), 3, (0, 1, 1)),
                 ((512, 64), 2, (1, 1)), ((64, 512), 2, (1, 2)), ((256, 512), 4, (1, 1, 2, 2))]


@pytest.mark.parametrize("case", CLUSTER_CASES, ids=str)
def test_cluster_path_matches_oracle(case):
    """The cluster-fused kernels (8 CTAs share one spectrum through distributed shared
    memory) against the oracle: forward, inverse and adjoint."""
    dims, J, sl = case
    b = bank(dims, J, sl, path="cluster")
    s = oracle_system(dims, J, sl)
    x = signal(dims, 12)
    C = b.forward(cuda(x)).cpu().numpy()
    assert rel(C, O.forward(x.astype(np.float64), s)) < TOL
    Cf = C.astype(np.float64)
    assert rel(b.inverse(cuda(C)).cpu().numpy(), O.inverse(Cf, s)) < TOL
    Cr = synth.gaussian_field((b.R,) + tuple(dims), 13)
    assert rel(b.adjoint(cuda(Cr)).cpu().numpy(), O.adjoint(Cr.astype(np.float64), s)) < TOL


def test_cluster_path_is_deterministic_and_agrees_with_general():
    dims, J, sl = (256, 256), 2, (1, 1)
    bc = bank(dims, J, sl, path="cluster")
    bg = bank(dims, J, sl, path="general")
    xg = cuda(signal(dims, 14))
    C1, C2 = bc.forward(xg).clone(), bc.forward(xg)
    assert torch.equal(C1, C2)
    assert torch.equal(bc.inverse(C1), bc.inverse(C2))
    assert rel(C1.cpu().numpy(), bg.forward(xg).cpu().numpy()) < TOL


# ------------------------------------------------ full-size configurations ---


@pytest.mark.parametrize("path", ["general", "cluster"])
def test_full_size_2d_512(path):
    """512^2, four scales, levels (1,1,2,2): R = 49 — the benchmark configuration,
    compared element by element (forward, inverse), on both kernel paths."""
    dims, J, sl = (512, 512), 4, (1, 1, 2, 2)
    b = bank(dims, J, sl, path=path)
    s = oracle_system(dims, J, sl)
    assert b.R == 49
    x = signal(dims, 10)
    C = b.forward(cuda(x))
    ref = O.forward(x.astype(np.float64), s)
    Cn = C.cpu().numpy()
    assert rel(Cn, ref) < TOL
    for j in range(b.R):
        assert rel(Cn[j], ref[j]) < TOL, j
    xi = b.inverse(C).cpu().numpy()
    assert rel(xi, O.inverse(C.cpu().numpy().astype(np.float64), s)) < TOL
    assert rel(xi, x) < TOL


def _oracle_inverse_worker(args):
    """Partial sum of eq. reconstruction over filters js, in a spawned process."""
    path, dims, J, sl, js = args
    import numpy as np_
    from oracle import shearlet_oracle as Orc
    C = np_.load(path, mmap_mode="r")
    s = Orc.build_system(dims, J, sl)
    return Orc.inverse_partial(lambda j: np_.asarray(C[j], dtype=np_.float64), s, js)


def _oracle_inverse_parallel(C, dims, J, sl, s, tmp_path, workers=None):
    """O.inverse of the coefficient stack C, its sum over filters split over spawned
    worker processes (the oracle's own inverse_partial / inverse_finish)."""
    import multiprocessing as mp
    import os
    path = str(tmp_path / "coeffs.npy")
    np.save(path, C)
    R = C.shape[0]
    workers = workers or max(1, min(16, (os.cpu_count() or 1)))
    chunks = [list(range(R))[i::workers] for i in range(workers)]
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = pool.map(_oracle_inverse_worker, [(path, dims, J, sl, c) for c in chunks if c])
    return O.inverse_finish(sum(parts), s, dual=True)


def test_full_size_3d_128(tmp_path):
    """128^3, three scales, levels (1,1,2): R = 292. Sampled subbands (every 17th and
    the last) against the oracle, each against its own size; the inverse of the GPU's
    own 292 coefficient volumes against the oracle's inverse; perfect reconstruction."""
    dims, J, sl = (128, 128, 128), 3, (1, 1, 2)
    b = bank(dims, J, sl)
    s = oracle_system(dims, J, sl)
    assert b.R == 292
    x = signal(dims, 11)
    xg = cuda(x)
    C = b.forward(xg)
    js = list(range(0, b.R, 17)) + [b.R - 1]
    ref = O.forward_subset(x.astype(np.float64), s, js)
    for j in js:
        assert rel(C[j].cpu().numpy(), ref[j]) < TOL, j
    xi = b.inverse(C).cpu().numpy()
    assert rel(xi, x) < TOL
    Cn = C.cpu().numpy()
    del C
    torch.cuda.empty_cache()
    assert rel(xi, _oracle_inverse_parallel(Cn, dims, J, sl, s, tmp_path)) < TOL


def test_full_size_3d_192():
    """192^3, the paper's video grid (Sec. 5.6), three scales, levels (1,1,2): R = 292.
    Its 192 x 192 planes take the one-plane-per-CTA kernel and its pencils the 16 x 12
    split with a radix-3 step. Sampled subbands against the oracle, each against its
    own size, and perfect reconstruction."""
    dims, J, sl = (192, 192, 192), 3, (1, 1, 2)
    b = bank(dims, J, sl)
    s = oracle_system(dims, J, sl)
    assert b.R == 292
    x = signal(dims, 16)
    C = b.forward(cuda(x))
    js = (0, 1, 70, 150, 291)
    ref = O.forward_subset(x.astype(np.float64), s, js)
    for j in js:
        assert rel(C[j].cpu().numpy(), ref[j]) < TOL, j
    xi = b.inverse(C).cpu().numpy()
    assert rel(xi, x) < TOL
    del C
    torch.cuda.empty_cache()


def test_full_size_2d_1024():
    """1024^2 (the largest 2D grid), four scales, levels (1,1,2,2): R = 49. Sampled
    subbands against the oracle, each against its own size, plus perfect
    reconstruction."""
    dims, J, sl = (1024, 1024), 4, (1, 1, 2, 2)
    b = bank(dims, J, sl)
    s = oracle_system(dims, J, sl)
    assert b.R == 49
    x = signal(dims, 15)
    C = b.forward(cuda(x))
    js = (0, 1, 12, 25, 33, 37, 48)
    ref = O.forward_subset(x.astype(np.float64), s, js)
    for j in js:
        assert rel(C[j].cpu().numpy(), ref[j]) < TOL, j
    xi = b.inverse(C).cpu().numpy()
    assert rel(xi, x) < TOL
    del C


def test_error_stats_kernel_matches_numpy():
    """The FP64-accumulating GPU reduction (max and L2 errors, PSNR of eq. PSNR)."""
    from paper_1402_5670_b300.shearlet import sl_error_stats
    x = synth.piecewise_smooth_image((512, 512), 3)
    y = synth.add_noise(x, 25.0, 4)
    st = sl_error_stats(cuda(y), cuda(x))
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    assert st["max_abs_err"] == np.max(np.abs(yd - xd))
    assert st["max_abs_ref"] == np.max(np.abs(xd))
    assert abs(st["sum_sq_err"] - np.sum((yd - xd) ** 2)) <= 1e-12 * np.sum((yd - xd) ** 2)
    assert abs(st["psnr"] - O.psnr(xd, yd)) < 1e-9


def test_misaligned_arrays_are_rejected_on_the_host():
    """Device arrays are accessed with 16-byte vector and asynchronous copies; a
    misaligned pointer is refused with SL_EINVAL before any kernel runs."""
    from paper_1402_5670_b300 import shearlet as S
    dims = (64, 64)
    b = bank(dims, 2, (1, 1))
    buf = torch.zeros(b.N + 4, device="cuda")
    C = torch.zeros((b.R,) + dims, device="cuda")
    st = S.lib().sl_forward(b.handle, buf.data_ptr() + 4, C.data_ptr(), None)
    assert S.STATUS[st] == "SL_EINVAL"
    assert "aligned" in S.lib().sl_last_error().decode()
    cbuf = torch.zeros(b.R * b.N + 4, device="cuda")
    st = S.lib().sl_inverse(b.handle, cbuf.data_ptr() + 8, buf.data_ptr(), None)
    assert S.STATUS[st] == "SL_EINVAL"
    torch.cuda.synchronize()


@pytest.mark.gpu
def test_shear_level_4_transform_matches_stored_oracle_spectra():
    """The maximum shear level on the GPU (64 x 64, R = 65): the forward transform of a
    unit impulse at the origin has DFT(C_j) = psi_hat_j, so the GPU coefficients,
    taken to frequency on the host, must hit the oracle's stored spectrum samples
    (tests/golden/shear4_bank_64x64.json) to 1e-5; the dual-frame inverse of those
    coefficients returns the impulse to 1e-5."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "shear4_bank_64x64.json")) as f:
        g = json.load(f)
    dims = tuple(g["dims"])
    b = bank(dims, g["nScales"], tuple(g["shearLevels"]))
    assert b.R == g["R"]
    x = np.zeros(dims, dtype=np.float32)
    x[0, 0] = 1.0
    C = b.forward(cuda(x))
    Cn = C.cpu().numpy().astype(np.float64)
    for j, fl in enumerate(g["filters"]):
        spec = np.fft.fft2(Cn[j])
        for k0, k1, v in fl["samples"]:
            assert abs(spec[k0, k1].real - v) <= 1e-5 and abs(spec[k0, k1].imag) <= 1e-5, (j, k0, k1)
    y = b.inverse(C).cpu().numpy()
    assert np.max(np.abs(y - x)) <= 1e-5
