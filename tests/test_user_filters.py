"""User-supplied filters (Sec. 4.1: the quadrature mirror filter's lowpass and the 2D
directional filter are inputs of the construction).

The library evaluates each filter from the DTFT of the given taps; the oracle builds
the same system in space from the same taps. They must agree to 1e-12 (FP64), and
the built-in designs passed as taps must reproduce the default bank.
"""
import numpy as np
import pytest

from oracle import shearlet_oracle as O
from paper_1402_5670_b300 import shearlet as S
from paper_1402_5670_b300 import synth


def binomial_qmf():
    """h = (1, 4, 6, 4, 1) / 16: H(w) = cos^4(w / 2), a lowpass with H(pi) = 0."""
    return np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0


def cubic_fan():
    """A lower-order maximally flat fan: P = 1/2 + 3/4 t - 1/4 t^3 with t the 3 x 3
    kernel of (cos w2 - cos w1) / 2 (built here as test data, 7 x 7 taps)."""
    t = np.zeros((3, 3))
    t[0, 1] = t[2, 1] = -0.25
    t[1, 0] = t[1, 2] = 0.25
    t2 = O.conv2d_full(t, t)
    t3 = O.conv2d_full(t2, t)
    P = 0.75 * np.pad(t, 2) - 0.25 * t3
    P[3, 3] += 0.5
    return P


def max_diff_vs_oracle(dims, J, sl, qmf, fan, full=False):
    b = S.Bank(dims, J, sl, full, device=-1, qmf=qmf, fan=fan)
    s = O.build_system(dims, J, sl, full, h=qmf, P=fan)
    assert b.R == s.R
    nh = dims[-1] // 2 + 1
    err = max(np.max(np.abs(b.eval_f64(j) - s.psi_hat(j)[..., :nh])) for j in range(b.R))
    err = max(err, np.max(np.abs(b.eval_f64(-1) - s.Psi[..., :nh])))
    err = max(err, np.max(np.abs(b.norms - s.norms)), abs(b.A - s.A))
    b.close()
    return err


def test_builtin_designs_passed_as_taps_reproduce_the_default_bank():
    dims, J, sl = (64, 64), 3, (0, 1, 1)
    d = S.Bank(dims, J, sl, device=-1)
    u = S.Bank(dims, J, sl, device=-1, qmf=O.qmf_lowpass(), fan=O.fan_filter())
    for j in range(d.R):
        assert np.max(np.abs(d.eval_f64(j) - u.eval_f64(j))) <= 1e-13
    d.close()
    u.close()


@pytest.mark.parametrize("case", [((64, 64), 2, (1, 1)), ((32, 64), 3, (0, 1, 2)),
                                  ((16, 16, 16), 2, (0, 1))], ids=str)
def test_user_filters_match_oracle(case):
    dims, J, sl = case
    assert max_diff_vs_oracle(dims, J, sl, binomial_qmf(), cubic_fan()) <= 1e-12
    assert max_diff_vs_oracle(dims, J, sl, binomial_qmf(), None) <= 1e-12
    assert max_diff_vs_oracle(dims, J, sl, None, cubic_fan()) <= 1e-12


@pytest.mark.parametrize("kw", [
    {"qmf": np.array([0.2, 0.5, 0.3])},                 # not symmetric
    {"qmf": np.array([0.25, 0.25, 0.25, 0.25])},        # even length
    {"fan": np.ones((4, 3))},                           # even size
    {"fan": np.arange(9.0).reshape(3, 3)},              # not point-symmetric
])
def test_invalid_taps_are_rejected(kw):
    with pytest.raises(S.ShearletError) as ei:
        S.Bank((32, 32), 1, (1,), device=-1, **kw)
    assert "SL_EINVAL" in str(ei.value)


torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_user_filter_bank_transforms_match_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5670_b300.build import build
    build()
    dims, J, sl = (128, 128), 3, (1, 1, 2)
    qmf, fan = binomial_qmf(), cubic_fan()
    b = S.Bank(dims, J, sl, device=0, qmf=qmf, fan=fan)
    s = O.build_system(dims, J, sl, False, h=qmf, P=fan)
    x = synth.add_noise(synth.piecewise_smooth_image(dims, 31), 20.0, 32)
    C = b.forward(torch.from_numpy(x).cuda())
    ref = O.forward(x.astype(np.float64), s)
    assert np.max(np.abs(C.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 1e-5
    y = b.inverse(C).cpu().numpy()
    assert np.max(np.abs(y - x)) / np.max(np.abs(x)) < 1e-5
    b.close()
