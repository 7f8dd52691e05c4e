"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

Each test states what it pins. None of them re-types the oracle's own formula: the
checks are values printed in the paper (tests/golden/, cited there), closed-form
properties, exact identities of the transform, brute-force sums on tiny grids,
special cases that reduce to textbook constructions, and mutation checks that plant
a plausible mistake in the oracle and require some pin to catch it.
"""
import math

import numpy as np
import pytest

from oracle import dft_oracle as D
from oracle import shearlet_oracle as O
from paper_1402_5670_b300 import synth
from tests.conftest import oracle_system, read_golden


def dtft1(taps, w):
    """DTFT of an origin-centred 1D filter at frequencies w (direct sum)."""
    n = np.arange(taps.size) - (taps.size - 1) // 2
    return np.exp(-1j * np.outer(np.atleast_1d(w), n)) @ taps


def dtft2(taps, w1, w2):
    n1 = np.arange(taps.shape[0]) - (taps.shape[0] - 1) // 2
    n2 = np.arange(taps.shape[1]) - (taps.shape[1] - 1) // 2
    E1 = np.exp(-1j * np.outer(np.atleast_1d(w1), n1))
    E2 = np.exp(-1j * np.outer(np.atleast_1d(w2), n2))
    return np.einsum("pi,ij,pj->p", E1, taps, E2)


# ------------------------------------------------------------------ 1D filters ---


def test_h_matches_printed_taps():
    """Sec. 5.1 footnote: printed taps to 5 decimals, and sum h = 1."""
    h = O.qmf_lowpass()
    rows = [r for r in read_golden("h_shearlab_taps.txt") if r[0].isdigit()]
    printed = np.array([float(v) for _, v in rows])
    assert h.size == 9
    assert np.max(np.abs(h[:5] - printed)) <= 5e-6
    assert np.allclose(h, h[::-1], atol=0, rtol=0)
    assert abs(h.sum() - 1.0) <= 1e-15


def test_h_orthonormality_bound():
    """Sec. 5.1: |2 sum h(n)h(n+2l) - delta_l0| <= 0.0018 (printed to 2 significant
    digits; the maximum, at l = 0, rounds to it)."""
    h = O.qmf_lowpass()
    bound = float([r for r in read_golden("h_shearlab_taps.txt")
                   if r[0] == "orthonormality_bound"][0][1])
    ac = np.correlate(h, h, mode="full")  # lags -8..8
    lags = np.arange(-8, 9)
    dev = np.abs(2 * ac[lags % 2 == 0] - (lags[lags % 2 == 0] == 0))
    assert dev.max() == pytest.approx(bound, abs=5e-5)
    assert np.argmax(dev) == 4  # l = 0


def test_h_is_maximally_flat_halfband_design():
    """Maximally flat lowpass of order 8 with half power at half band (Sec. 5.1
    footnote): H(0)=1, H(pi)=0, H(pi/2)=1/sqrt2, and the response is flat at 0 to
    5th order (vanishing 2nd and 4th moments). Checked by direct DTFT sums."""
    h = O.qmf_lowpass()
    n = np.arange(9) - 4
    H = dtft1(h, np.array([0.0, np.pi, np.pi / 2]))
    assert abs(H[0] - 1) < 1e-15 and abs(H[1]) < 1e-15
    assert abs(H[2] - 1 / math.sqrt(2)) < 1e-15
    assert abs(np.sum(n ** 2 * h)) < 1e-14
    assert abs(np.sum(n ** 4 * h)) < 1e-13
    assert abs(np.sum(n ** 6 * h)) > 1e-3  # and no flatter than that


def test_g_is_mirror_filter():
    """g(n) = (-1)^n h(n) (Sec. 5.1) means g_hat(w) = h_hat(w + pi)."""
    h = O.qmf_lowpass()
    g = O.qmf_highpass(h)
    w = np.linspace(-np.pi, np.pi, 37)
    assert np.allclose(dtft1(g, w), dtft1(h, w + np.pi), atol=1e-14)


@pytest.mark.parametrize("j", [1, 2, 3, 4, 5])
def test_lowhigh_frequency_products(j):
    """eq. lowhigh (Sec. 3.1): the spatial h_j, g_j have the DTFTs
    prod_{k<j} h_hat(2^k w) and g_hat(2^{j-1} w) h_hat_{j-1}(w)."""
    h = O.qmf_lowpass()
    g = O.qmf_highpass(h)
    w = np.random.default_rng(j).uniform(-np.pi, np.pi, 25)
    want_h = np.prod([dtft1(h, 2 ** k * w) for k in range(j)], axis=0)
    assert np.allclose(dtft1(O.lowpass_j(h, j), w), want_h, atol=1e-13)
    want_g = dtft1(g, 2 ** (j - 1) * w) * (np.prod([dtft1(h, 2 ** k * w) for k in range(j - 1)],
                                                  axis=0) if j > 1 else 1.0)
    assert np.allclose(dtft1(O.highpass_j(h, g, j), w), want_g, atol=1e-13)


# ------------------------------------------------------------------ fan filter ---


def test_fan_filter_properties():
    """The fan filter P of eq. nonsep: real and point-symmetric, complementary to its
    transpose (the two cones of Sec. 2.2.1 split the plane), half-band
    P(w) + P(w + (pi, pi)) = 1, full pass at (pi, 0), full stop at (0, pi), passes the
    cone |w2| < |w1| and stops |w2| > |w1| (Sec. 3.2.1), values in [0, 1]."""
    P = O.fan_filter()
    assert np.allclose(P, P[::-1, ::-1], atol=0)
    comp = -P.T
    comp[7, 7] += 1.0
    assert np.allclose(P, comp, atol=1e-16)  # P(w2, w1) = 1 - P(w1, w2): the two cones
    r = np.random.default_rng(7)
    w1, w2 = r.uniform(-np.pi, np.pi, 200), r.uniform(-np.pi, np.pi, 200)
    V = dtft2(P, w1, w2)
    assert np.max(np.abs(V.imag)) < 1e-14
    V2 = dtft2(P, w1 + np.pi, w2 + np.pi)
    assert np.max(np.abs(V.real + V2.real - 1)) < 1e-14
    assert abs(dtft2(P, np.pi, 0.0)[0] - 1) < 1e-14
    assert abs(dtft2(P, 0.0, np.pi)[0]) < 1e-14
    assert np.all(V.real > -1e-12) and np.all(V.real < 1 + 1e-12)
    inner = (np.abs(w2) < 0.5 * np.abs(w1)) & (np.abs(w1) > 2.0)
    outer = (np.abs(w1) < 0.5 * np.abs(w2)) & (np.abs(w2) > 2.0)
    assert np.all(V.real[inner] > 0.9) and np.all(V.real[outer] < 0.1)


def test_fan_filter_maximally_flat_at_passband_centre():
    """'maximally flat' (Sec. 5.1): 1 - P(pi - e, 0) falls off like e^8 (the order-4
    flatness of M), checked by the ratio at e and e/2 (expected 2^8)."""
    P = O.fan_filter()
    e = 0.2
    a = 1 - dtft2(P, np.pi - e, 0.0)[0].real
    b = 1 - dtft2(P, np.pi - e / 2, 0.0)[0].real
    assert 200 < a / b < 300


# -------------------------------------------------------------------- shearing ---


def test_integer_shear_is_index_map():
    """With d = 0 the digital shear is S_k itself: out(n1, n2) = f(n1 + k n2, n2)."""
    r = np.random.default_rng(3)
    f = r.standard_normal((5, 7))
    for k in (-2, -1, 1, 2):
        out = O.dshear(f, k, 0, O.qmf_lowpass())
        cM, cN = 2, 3
        cO = (out.shape[0] - 1) // 2
        for i in range(out.shape[0]):
            for i2 in range(7):
                n1, n2 = i - cO, i2 - cN
                src = n1 + k * n2
                want = f[src + cM, i2] if -cM <= src <= cM else 0.0
                assert out[i, i2] == want


def test_zero_shear_is_identity_up_to_orthonormality_defect():
    """S^1_0 applied to a delta is 2 (h * h)(2 l): by Sec. 5.1's orthonormality bound it
    differs from the delta by at most 0.0018 at every tap."""
    h = O.qmf_lowpass()
    delta = np.zeros((1, 1))
    delta[0, 0] = 1.0
    out = O.dshear(delta, 0, 1, h)
    ref = np.zeros_like(out)
    ref[(out.shape[0] - 1) // 2, 0] = 1.0
    assert np.max(np.abs(out - ref)) <= 0.0018 + 5e-5
    assert np.max(np.abs(out - ref)) > 1e-3  # it is not exact: h is not orthonormal


def test_shear_direction_follows_k():
    """Sec. 3.2.2: filter psi_{j,k} covers directions of slope about k / 2^d (cone 1:
    xi2/xi1; cone 2: xi1/xi2). The energy-weighted slope must have the sign of k,
    increase with k, and lie within 0.2 of k/2^d."""
    s = oracle_system((128, 128), 3, (1, 1, 2))
    w = 2 * np.pi * np.fft.fftfreq(128)
    W1, W2 = np.meshgrid(w, w, indexing="ij")
    for cone in (1, 2):
        rows = [(m.k[0], j) for j, m in enumerate(s.meta) if m.scale == 2 and m.cone == cone]
        cents = []
        for k, j in sorted(rows):
            F = s.psi_hat(j) ** 2
            if cone == 1:
                mask = np.abs(W1) > np.pi / 4
                slope = W2[mask] / W1[mask]
            else:
                mask = np.abs(W2) > np.pi / 4
                slope = W1[mask] / W2[mask]
            c = float((F[mask] * slope).sum() / F[mask].sum())
            cents.append(c)
            assert abs(c - k / 4) < 0.2
            assert np.sign(round(c, 6)) == np.sign(k)
        assert np.all(np.diff(cents) > 0)


def test_separable_special_case():
    """Sec. 3.2.1 after eq. noshear: with p_j = delta (P = 1), the scale-j filter is the
    separable wavelet g_{J-j} (x) h_{J-j}; with d = 0 and k = 0 the shear is the
    identity. The oracle's pipeline must return exactly that outer product."""
    h = O.qmf_lowpass()
    g = O.qmf_highpass(h)
    one = np.ones((1, 1))
    J = 3
    for j in range(J):
        u = O._unsheared_2d(h, g, one, J, j, 0)
        sep = np.outer(O.highpass_j(h, g, J - j), O.lowpass_j(h, J - j))
        assert u.shape == sep.shape and np.array_equal(u, sep)
        assert np.array_equal(O.dshear(u, 0, 0, h), u)


# ----------------------------------------------------------------- the systems ---


@pytest.mark.parametrize("row", read_golden("systems_table.txt"), ids=lambda r: r[0])
def test_filter_counts_match_table(row):
    """Sec. 5.1 table: directions per scale and redundancy of SL2D_1/2, SL3D_1/2."""
    name, ndim, scales, dirs, sl, R = row[:6]
    ndim, scales, R = int(ndim), int(scales), int(R)
    dirs = [int(v) for v in dirs.split(",")]
    sl = [int(v) for v in sl.split(",")]
    assert O.redundancy_formula(ndim, sl, False) == R
    dims = (16, 16) if ndim == 2 else (8, 8, 8)
    s = oracle_system(dims, scales, sl)
    assert s.R == R
    per_scale = [sum(1 for m in s.meta if m.scale == j) for j in range(scales)]
    assert per_scale == dirs


@pytest.mark.parametrize("row", read_golden("redundancy_examples.txt"))
def test_redundancy_examples(row):
    """Secs. 4.1 and 4.4: per-scale counts with and without boundary omission."""
    ndim, full, sl, counts, R = row
    sl = [int(v) for v in sl.split(",")]
    counts = [int(v) for v in counts.split(",")]
    dims = (16, 16) if int(ndim) == 2 else (8, 8, 8)
    s = oracle_system(dims, len(sl), sl, bool(int(full)))
    assert s.R == int(R) == O.redundancy_formula(int(ndim), sl, bool(int(full)))
    assert [sum(1 for m in s.meta if m.scale == j) for j in range(len(sl))] == counts


def test_frame_bounds_hard_and_soft():
    """eq. frame_filter: Psi > 0 everywhere (else the dual filters of eq. dual_filter do
    not exist) and B = max Psi = 1 after normalisation (the table's B = 1.0000).
    Soft (reported, not gated): A of SL2D_2 on 512^2 against the table's 0.0669."""
    s = oracle_system((512, 512), 4, (1, 1, 2, 2))
    assert s.A > 0.0 and abs(s.B - 1.0) < 1e-14
    print(f"SL2D_2 on 512^2: A = {s.A:.4f} (paper 0.0669), B/A = {1 / s.A:.2f} (paper 14.94)")
    assert 0.03 < s.A < 0.2


def test_filters_are_point_symmetric():
    """All ingredients are odd-length and symmetric, so psi(-n) = psi(n) on the grid
    and psi_hat is real (Sec. 3.4 uses |psi_hat|^2 = psi_hat^2)."""
    s = oracle_system((32, 32), 2, (1, 2))
    for j in range(s.R):
        f = s.psi_spatial(j)
        fm = np.roll(f[::-1, ::-1], 1, axis=(0, 1))  # f(-n)
        assert np.allclose(f, fm, atol=1e-15)


# --------------------------------------------------------------- the transform ---


CASES_2D = [((64, 64), 3, (0, 1, 1)), ((48, 32), 2, (1, 1)), ((256, 256), 2, (1, 1))]
CASES_3D = [((16, 16, 16), 2, (0, 1)), ((32, 16, 24), 2, (1, 1))]


@pytest.mark.parametrize("case", CASES_2D + CASES_3D, ids=str)
def test_perfect_reconstruction(case):
    """eq. reconstruction: inverse(forward(x)) = x exactly, to 1e-12 in FP64."""
    dims, J, sl = case
    s = oracle_system(dims, J, sl)
    x = synth.gaussian_field(dims, 11, 50.0).astype(np.float64) + 100.0
    y = O.inverse(O.forward(x, s), s)
    assert np.max(np.abs(y - x)) / np.max(np.abs(x)) < 1e-12


@pytest.mark.parametrize("case", CASES_2D[:2] + CASES_3D[:1], ids=str)
def test_adjoint_identity(case):
    """<SH x, C> = <x, SH* C> for random x and C, to 1e-12 relative."""
    dims, J, sl = case
    s = oracle_system(dims, J, sl)
    x = synth.gaussian_field(dims, 5).astype(np.float64)
    C = synth.gaussian_field((s.R,) + tuple(dims), 6).astype(np.float64)
    lhs = float(np.sum(O.forward(x, s) * C))
    rhs = float(np.sum(x * O.adjoint(C, s)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0) * 10


@pytest.mark.parametrize("case", [((16, 16), 2, (0, 1)), ((16, 16), 1, (1,)),
                                  ((24, 16), 1, (1,)), ((12, 24), 1, (0,)),
                                  ((8, 8, 8), 1, (0,)), ((8, 8, 8), 1, (1,))], ids=str)
def test_forward_equals_bruteforce_correlation(case):
    """eq. convolution: C_j(m) = (x * conj(psi_j))(m) = sum_n x(n) psi_j(n - m), summed
    directly over the grid with the spatial, folded filter (3D: the filter built in
    space as the circular convolution of its three factors)."""
    dims, J, sl = case
    s = oracle_system(dims, J, sl)
    x = synth.gaussian_field(dims, 21).astype(np.float64)
    C = O.forward(x, s)
    js = range(s.R) if len(dims) == 2 else [0, 1, s.R // 2, s.R - 1]
    for j in js:
        want = O.circular_correlate_direct(x, s.psi_spatial(j))
        assert np.max(np.abs(C[j] - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))


def test_threshold_semantics():
    """eq. hard_tresholding: keep x(n) iff |x(n)| >= delta (ties kept); the lowpass is
    never thresholded (reading)."""
    s = oracle_system((16, 16), 2, (0, 1))
    C = np.zeros((s.R, 16, 16))
    dl = O.thresholds(s, 10.0, [2.0, 3.0])
    for j in range(s.R):
        C[j, 0, 0] = dl[j]            # tie: kept
        C[j, 0, 1] = np.nextafter(dl[j], 0) if dl[j] > 0 else 0.0  # just below
        C[j, 0, 2] = -2 * dl[j] - 1   # kept
    T = O.threshold(C, s, 10.0, [2.0, 3.0])
    assert dl[0] == 0.0
    assert np.array_equal(T[0], C[0])
    for j in range(1, s.R):
        assert T[j, 0, 0] == C[j, 0, 0] and T[j, 0, 1] == 0.0 and T[j, 0, 2] == C[j, 0, 2]


def test_noisy_psnr_matches_paper():
    """eq. PSNR: an unclipped N(0, 40^2) perturbation of a 512^2 image has PSNR
    20 log10(255/40) = 16.09; the paper prints 16.06 for its (clipped) noisy images."""
    rows = dict((r[0], float(r[1])) for r in read_golden("psnr_noisy.txt"))
    x = synth.piecewise_smooth_image((512, 512), 1).astype(np.float64)
    y = synth.add_noise(x, rows["sigma"], 2)
    p = O.psnr(x, y)
    assert abs(p - 20 * math.log10(255 / rows["sigma"])) < 0.02
    assert abs(p - rows["psnr_printed"]) < 0.06


def test_denoising_improves_psnr():
    """Sec. 5.3: hard thresholding of the coefficients removes noise; on a synthetic
    piecewise-smooth 256^2 image at sigma = 20 the PSNR must rise by several dB."""
    s = oracle_system((256, 256), 2, (1, 1))
    x = synth.piecewise_smooth_image((256, 256), 3).astype(np.float64)
    y = synth.add_noise(x, 20.0, 4).astype(np.float64)
    z = O.denoise(y, s, 20.0, [2.5, 3.8])
    assert O.psnr(x, z) > O.psnr(x, y) + 4.0


# ------------------------------------------------------- the oracle's own DFT ---


@pytest.mark.parametrize("n", [1, 2, 3, 8, 12, 16])
def test_direct_dft_closed_forms(n):
    """The defining sum on closed forms: the DFT of the unit impulse at a is
    exp(-2 pi i a k / n), the DFT of exp(+2 pi i m t / n) is n at k = m and 0 elsewhere
    (fixes the sign convention), and the inverse sum brings the impulse back."""
    k = np.arange(n)
    for a in range(n):
        e = np.zeros(n)
        e[a] = 1.0
        want = np.exp(-2j * np.pi * a * k / n)
        assert np.max(np.abs(D.dft_direct(e) - want)) <= 1e-14 * n
        assert np.max(np.abs(D.dft_direct(want, sign=+1) / n - e)) <= 1e-14 * n
    for m in range(n):
        x = np.exp(2j * np.pi * m * k / n)
        want = np.zeros(n)
        want[m] = n
        assert np.max(np.abs(D.dft_direct(x) - want)) <= 1e-13 * n


@pytest.mark.parametrize("n", [9, 16, 24, 64, 96, 128, 192, 256, 384, 512, 1024])
def test_fft_equals_direct_dft(n):
    """The recursive FFT (radix 2, one radix-3 step for 3 * 2^k) equals the direct sum
    to 1e-13 relative, both directions, on seeded complex data."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, 1):
        want = D.dft_direct(x, sign=sign)
        assert np.max(np.abs(D.fft(x, sign=sign) - want)) <= 1e-13 * np.max(np.abs(want))


def test_fftn_is_separable_and_inverts():
    """fftn applies the 1D DFT along each axis (checked axis by axis against the direct
    sum on a 12 x 8 x 6 grid), and ifftn(fftn(x)) = x to 1e-14."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal((12, 8, 6))
    want = D.dft_direct(D.dft_direct(D.dft_direct(x, 0), 1), 2)
    got = D.fftn(x)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))
    assert np.max(np.abs(D.ifftn(got) - x)) <= 1e-14 * np.max(np.abs(x)) * 10


def test_pin_catches_wrong_fft_twiddle(monkeypatch):
    """Planted mistake: the inter-stage twiddle of the FFT with the wrong sign. The
    FFT-versus-direct-sum pin must fail."""
    orig = D._twiddle
    monkeypatch.setattr(D, "_twiddle", lambda r, k1, n_len, sign: orig(r, k1, n_len, -sign))
    rng = np.random.default_rng(3)
    x = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    want = D.dft_direct(x)
    assert np.max(np.abs(D.fft(x) - want)) > 1e-3 * np.max(np.abs(want))


# ------------------------------------------------ filter norms and thresholds ---


def _parseval_deviation(dims, J, sl):
    """max_j | ||psi_j||_2^2 (the oracle's norm) / sum_n psi_j(n)^2 - 1 |, the sum taken
    over the filter folded onto the grid in SPACE (Parseval's identity on Z_N): the
    norm the thresholds use must be the l2 norm of the spatial filter."""
    s = O.build_system(dims, J, sl)
    dev = 0.0
    for j in range(s.R):
        e = float(np.sum(s.psi_spatial(j) ** 2))
        dev = max(dev, abs(float(s.norms[j]) ** 2 / e - 1.0))
    return dev


def _white_noise_stats(sigma=3.0, draws=400, K=1.0):
    """Monte Carlo over seeded Gaussian noise of std sigma on a 32x32 grid (J = 2,
    levels (0, 1)). Returns (max_j |std(C_j) / (sigma ||psi_j||) - 1|, max_j>=1 |P(|C_j|
    >= delta_j) - 2 (1 - Phi(K))|) with delta_j from the oracle's thresholds at K.
    For white noise C_j(m) ~ N(0, sigma^2 sum_n psi_j(n)^2) exactly, so the threshold
    K sigma ||psi_j||_2 of the hard-thresholding rule (Sec. 5.3) is exceeded with
    the two-sided Gaussian tail probability."""
    s = O.build_system((32, 32), 2, (0, 1))
    rng = np.random.default_rng(np.random.PCG64(77))
    dl = O.thresholds(s, sigma, [K, K])
    var = np.zeros(s.R)
    hit = np.zeros(s.R)
    for _ in range(draws):
        C = O.forward(sigma * rng.standard_normal((32, 32)), s)
        var += (C ** 2).reshape(s.R, -1).mean(axis=1)
        hit += (np.abs(C) >= dl[:, None, None]).reshape(s.R, -1).mean(axis=1)
    std_dev = float(np.max(np.abs(np.sqrt(var / draws) / (sigma * s.norms) - 1.0)))
    tail = math.erfc(K / math.sqrt(2.0))          # 2 (1 - Phi(K))
    tail_dev = float(np.max(np.abs(hit[1:] / draws - tail)))
    return std_dev, tail_dev


@pytest.mark.parametrize("case", [((16, 16), 2, (0, 1)), ((24, 16), 1, (1,)),
                                  ((8, 8, 8), 1, (1,))], ids=str)
def test_norms_equal_spatial_l2_norm(case):
    """||psi_j||_2 (the factor of the threshold delta_j = K sigma ||psi_j||_2) equals
    the l2 norm of the filter in space, computed from the folded spatial filter
    rather than from its spectrum (Parseval on Z_N)."""
    assert _parseval_deviation(*case) <= 1e-12


@pytest.mark.slow
def test_norms_are_subband_noise_std_and_thresholds_hit_gaussian_tail():
    """Sec. 5.3 thresholds subband j at K sigma ||psi_j||_2: the standard deviation of
    the subband's response to white noise of std sigma. Monte Carlo (400 seeded
    draws): the sample std matches sigma ||psi_j|| to 2% and |C_j| >= delta_j (K = 1)
    occurs with probability erfc(1/sqrt 2) = 0.3173 to 0.015."""
    std_dev, tail_dev = _white_noise_stats()
    assert std_dev < 0.02, std_dev
    assert tail_dev < 0.015, tail_dev


def test_pin_catches_norm_without_grid_size(monkeypatch):
    """Planted mistake: ||psi_j||^2 = sum_xi psi_hat^2 (no 1/N). Parseval must fail."""
    orig = O._finish_system

    def bad(sysm):
        sysm = orig(sysm)
        sysm.norms = sysm.norms * math.sqrt(sysm.N)
        return sysm
    monkeypatch.setattr(O, "_finish_system", bad)
    assert _parseval_deviation((16, 16), 2, (0, 1)) > 0.5


def test_pin_catches_norm_without_sqrt(monkeypatch):
    """Planted mistake: the squared norm used as the norm. Parseval must fail."""
    orig = O._finish_system

    def bad(sysm):
        sysm = orig(sysm)
        sysm.norms = sysm.norms ** 2
        return sysm
    monkeypatch.setattr(O, "_finish_system", bad)
    assert _parseval_deviation((16, 16), 2, (0, 1)) > 0.5


@pytest.mark.slow
def test_pin_catches_threshold_without_sigma(monkeypatch):
    """Planted mistake: delta_j = K ||psi_j|| (sigma dropped). The tail pin must fail."""
    def bad_thresholds(sysm, sigma, K):
        d = np.zeros(sysm.R)
        for j, m in enumerate(sysm.meta):
            if m.scale >= 0:
                d[j] = float(K[m.scale]) * float(sysm.norms[j])
        return d
    monkeypatch.setattr(O, "thresholds", bad_thresholds)
    _, tail_dev = _white_noise_stats(draws=50)
    assert tail_dev > 0.1


# ------------------------------------------------- planted mistakes are caught ---


def test_pin_catches_conjugated_signal(monkeypatch):
    """Planted mistake: Algorithm 1's literal IFFT(psi_hat .* conj(FFT f)) instead of
    the definition's f * conj(psi). The brute-force correlation pin must fail."""
    s = oracle_system((16, 16), 1, (1,))
    x = synth.gaussian_field((16, 16), 21).astype(np.float64)

    def bad_forward_iter(x, sysm):
        X = np.fft.fftn(x)
        for j in range(sysm.R):
            yield j, np.real(np.fft.ifftn(sysm.psi_hat(j) * np.conj(X)))
    monkeypatch.setattr(O, "forward_iter", bad_forward_iter)
    C = O.forward(x, s)
    errs = [np.max(np.abs(C[j] - O.circular_correlate_direct(x, s.psi_spatial(j))))
            for j in range(s.R)]
    assert max(errs) > 1e-3


def test_pin_catches_flipped_shear_sign(monkeypatch):
    """Planted mistake: shear x1 <- x1 - k x2. The direction pin must fail."""
    orig = O.shear_integer
    monkeypatch.setattr(O, "shear_integer", lambda f, k: orig(f, -k))
    _SYS = O.build_system((128, 128), 3, (1, 1, 2))
    w = 2 * np.pi * np.fft.fftfreq(128)
    W1, W2 = np.meshgrid(w, w, indexing="ij")
    j = [i for i, m in enumerate(_SYS.meta) if m.scale == 2 and m.cone == 1 and m.k == (2,)][0]
    F = _SYS.psi_hat(j) ** 2
    mask = np.abs(W1) > np.pi / 4
    c = float((F[mask] * W2[mask] / W1[mask]).sum() / F[mask].sum())
    assert abs(c - 0.5) > 0.2


def test_pin_catches_missing_interpolation_gain(monkeypatch):
    """Planted mistake: refine with h_d instead of 2^d h_d. The zero-shear pin fails."""
    h = O.qmf_lowpass()

    def bad_dshear(f, k, d, h):
        s = 2 ** d
        hd = O.lowpass_j(h, d)
        ft = O.conv_axis(O.upsample_axis(f, s, 0), hd, 0)
        ft = O.shear_integer(ft, k)
        return O.downsample_axis(O.conv_axis(ft, hd, 0), s, 0)
    delta = np.ones((1, 1))
    out = bad_dshear(delta, 0, 1, h)
    assert abs(out[(out.shape[0] - 1) // 2, 0] - 1.0) > 0.4


def test_pin_catches_dropped_filter(monkeypatch):
    """Planted mistake: a filter missing from the frame weight. Perfect reconstruction
    must fail."""
    s = O.build_system((32, 32), 2, (1, 1))
    Psi_bad = s.Psi - s.psi_hat(5) ** 2
    x = synth.gaussian_field((32, 32), 1).astype(np.float64)
    C = O.forward(x, s)
    acc = sum(np.fft.fftn(C[j]) * s.psi_hat(j) / Psi_bad for j in range(s.R))
    y = np.real(np.fft.ifftn(acc))
    assert np.max(np.abs(y - x)) > 1e-3 * np.max(np.abs(x))


def test_pin_catches_swapped_wavelet_axes(monkeypatch):
    """Planted mistake: W_j = h (x) g instead of g (x) h (wavelet on the wrong axis). The
    shear-direction pin (cone 1 concentrates around the xi_1 axis) must fail."""
    def bad_unsheared(h, g, P, J, j, d):
        p = O.upsample_axis(O.upsample_axis(P, 2 ** (J - j - 1), 0), 2 ** (J - j + d), 1)
        W = np.outer(O.lowpass_j(h, J - j + d), O.highpass_j(h, g, J - j))
        return O.conv2d_full(p, W)
    w = 2 * np.pi * np.fft.fftfreq(64)
    W1, W2 = np.meshgrid(w, w, indexing="ij")

    def frac_in_cone1():
        s = O.build_system((64, 64), 2, (1, 1))
        j = [i for i, m in enumerate(s.meta) if m.scale == 1 and m.cone == 1 and m.k == (0,)][0]
        F = s.psi_hat(j) ** 2
        return F[np.abs(W2) < np.abs(W1)].sum() / F.sum()
    assert frac_in_cone1() > 0.9
    monkeypatch.setattr(O, "_unsheared_2d", bad_unsheared)
    assert frac_in_cone1() < 0.5


# ------------------------------------------------------------------ inpainting ---

def test_inpaint_schedule_ends_at_delta_min():
    """Sec. 5.4: delta shrinks geometrically from delta_init to delta_min."""
    lam = O.inpaint_ratio(50.0, 2.0, 11)
    assert abs(50.0 * lam ** 10 - 2.0) < 1e-12
    assert O.inpaint_ratio(5.0, 1.0, 1) == 1.0


def test_inpaint_without_occlusion_is_perfect_reconstruction():
    """Mask of ones and a threshold far below every coefficient: one iteration is
    T^-1 T f = f (eq. reconstruction)."""
    dims = (32, 32)
    s = oracle_system(dims, 2, (1, 1))
    f = synth.piecewise_smooth_image(dims, 3).astype(np.float64)
    out = O.inpaint(f, np.ones(dims, np.uint8), s, 1e-12, 1e-12, 1)
    assert np.max(np.abs(out - f)) <= 1e-10 * np.max(np.abs(f))


def test_inpaint_without_thresholding_keeps_the_known_pixels_only():
    """With no coefficient thresholded the iteration is f_k+1 = M f_masked + (1 - M) f_k
    (M^2 = M), whose fixed point reached at once from 0 is M f_masked: the unknown
    pixels stay 0. A sign slip in the residual breaks this."""
    dims = (32, 32)
    s = oracle_system(dims, 2, (1, 1))
    f = synth.piecewise_smooth_image(dims, 4).astype(np.float64)
    M = synth.random_mask(dims, 0.5, 5)
    out = O.inpaint(f * M, M, s, 1e-12, 1e-12, 3)
    assert np.max(np.abs(out - f * M)) <= 1e-9 * np.max(np.abs(f))


def test_inpainting_fills_the_holes():
    """Iterative thresholding recovers most of a randomly 60%-occluded cartoon image:
    far better PSNR than the masked image, and better than the mean fill."""
    dims = (64, 64)
    s = oracle_system(dims, 3, (0, 1, 1))
    f = synth.piecewise_smooth_image(dims, 6).astype(np.float64)
    M = synth.random_mask(dims, 0.6, 7)
    out = O.inpaint(f * M, M, s, 200.0, 2.0, 30)
    mean_fill = np.where(M > 0, f, np.mean(f[M > 0]))
    assert O.psnr(f, out) > O.psnr(f, mean_fill) + 3.0
    assert O.psnr(f, out) > O.psnr(f, f * M) + 10.0


def test_pin_catches_residual_sign_slip():
    """Planted mistake (a copy of the iteration with f_res = M (f_inpainted - f_masked)):
    the fixed-point pin above must fail for it."""
    dims = (32, 32)
    s = oracle_system(dims, 2, (1, 1))
    f = synth.piecewise_smooth_image(dims, 4).astype(np.float64)
    M = synth.random_mask(dims, 0.5, 5).astype(np.float64)
    out = np.zeros_like(f)
    for _ in range(3):
        out = O.denoise(M * (out - f * M) + out, s, 1e-12, [1.0, 1.0])
    assert np.max(np.abs(out - f * M)) > 1e-3 * np.max(np.abs(f))
