"""FP64 CPU oracle of the non-subsampled digital shearlet transform (ShearLab 3D,
Kutyniok, Lim, Reisenhofer, arXiv 1402.5670).

TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module. The product path (the CUDA library and its
Python binding) never does, and this module imports nothing from it.

What it computes, step by step in the paper's order and notation:

* 1D filters h, g and the multiscale filters h_j, g_j        (Sec. 3.1, eq. lowhigh;
                                                               Sec. 5.1)
* the 2D fan filter P                                         (Sec. 3.2.1, eq. nonsep;
                                                               Sec. 5.1)
* the unsheared scale-j filter p_j * W_j                      (Sec. 3.2, eqs. noshear,
                                                               ext_noshear_alpha)
* the digital shear S^d_{k/2^d}                               (Sec. 3.2.2, eqs.
                                                               dshear1_alpha, dshear2_alpha)
* the 2D filters psi^d_{j,k} and the axis-swapped second cone (Def. digitSH_alpha,
                                                               Sec. 3.4 eq. convolution01)
* the 3D filters as products of a 1D and two 2D factors, in
  three pyramids                                              (Def. 3DdigitSH(_alpha),
                                                               eqs. 3Dfilters1/2_alpha)
* omission of boundary shearlets                              (Sec. 4.4)
* lowpass, frame weight Psi, dual filters                     (Sec. 3.4, eqs.
                                                               frame_filter, dual_filter)
* forward (Algorithm 1 with the conjugation of eq. convolution), adjoint, dual-frame
  inverse (Algorithm 2, eq. reconstruction), the same inverse split into partial sums
  over filter subsets, hard thresholding (eq. hard_tresholding) and PSNR (eq. PSNR)
                                                              (Secs. 4.1, 4.2, 5.3)

Every filter is built in the SPATIAL domain with explicit upsampling, convolution,
shearing and downsampling of finite arrays, then folded periodically onto the
N-grid and transformed with the oracle's own DFT (oracle/dft_oracle.py: the direct
sum on tiny lengths, decimation in time by 2 (and once by 3) beyond). Readings taken where
the paper is silent or ambiguous are marked "Reading:" below; each is listed in the
design notes.

Parity status: every function here is pinned by a test in tests/test_oracle_pins.py
except the exact numerical values of ShearLab's own fan filter (the paper names it,
'dmaxflat4', but does not print its taps), so the bank's absolute values are
"parity unpinned" against ShearLab itself; the bank is pinned against the paper's
invariants (real spectra, frame identities, filter counts, special cases) instead.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Iterator, List, Optional, Sequence, Tuple, Union

import numpy as np

from oracle import dft_oracle as _dft

# --------------------------------------------------------------------------------
# Finite arrays. Every filter here has odd extent on every axis with the origin
# n = 0 at the centre index, so "center" is always (size - 1) // 2.
# --------------------------------------------------------------------------------


def _center(a: np.ndarray, axis: int) -> int:
    return (a.shape[axis] - 1) // 2


def conv_axis(a: np.ndarray, k: np.ndarray, axis: int) -> np.ndarray:
    """Full linear convolution of array ``a`` with the 1D filter ``k`` along ``axis``.

    Written as a sum of shifted, scaled copies of ``a`` (one per tap), so the
    result of every output sample is the textbook sum  sum_i k(i) a(n - i).
    Odd lengths in, odd length out; centres stay aligned.
    """
    a = np.moveaxis(np.asarray(a, dtype=np.float64), axis, 0)
    k = np.asarray(k, dtype=np.float64)
    out = np.zeros((a.shape[0] + k.size - 1,) + a.shape[1:])
    for i, c in enumerate(k):
        if c != 0.0:
            out[i:i + a.shape[0]] += c * a
    return np.moveaxis(out, 0, axis)


def conv1d(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Full linear convolution of two 1D filters."""
    return conv_axis(np.asarray(a, dtype=np.float64), b, 0)


def conv2d_full(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Full 2D linear convolution, as a sum over the nonzero taps of ``a``."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    out = np.zeros((a.shape[0] + b.shape[0] - 1, a.shape[1] + b.shape[1] - 1))
    for (i0, i1) in zip(*np.nonzero(a)):
        out[i0:i0 + b.shape[0], i1:i1 + b.shape[1]] += a[i0, i1] * b
    return out


def upsample_axis(a: np.ndarray, m: int, axis: int) -> np.ndarray:
    """Insert m-1 zeros between samples along ``axis`` (the operator 'up m')."""
    a = np.moveaxis(np.asarray(a, dtype=np.float64), axis, 0)
    out = np.zeros(((a.shape[0] - 1) * m + 1,) + a.shape[1:])
    out[::m] = a
    return np.moveaxis(out, 0, axis)


def downsample_axis(a: np.ndarray, m: int, axis: int) -> np.ndarray:
    """Keep the samples n = 0 (mod m) along ``axis`` (the operator 'down m')."""
    a = np.moveaxis(np.asarray(a, dtype=np.float64), axis, 0)
    c = (a.shape[0] - 1) // 2
    first = c % m
    out = a[first::m]
    assert (out.shape[0] - 1) // 2 * m + first == c, "origin must stay a kept sample"
    return np.moveaxis(out, 0, axis)


# --------------------------------------------------------------------------------
# 1D wavelet filters (Sec. 5.1 and Sec. 3.1)
# --------------------------------------------------------------------------------


def qmf_lowpass() -> np.ndarray:
    """h_ShearLab: symmetric, maximally flat 9-tap lowpass with sum 1 (Sec. 5.1).

    The paper gives it as MATLAB's maxflat design of order 8 with its half-power
    point at half the band and prints its approximate taps. Its frequency response is
    the degree-4 polynomial in s = sin^2(w/2)
        H(w) = 1 + (8 sqrt2 - 15) s^3 + (14 - 8 sqrt2) s^4,
    the one with H(0)=1, H'(0)=H''(0)=0 (flat at 0), H(pi)=0 and H(pi/2)=1/sqrt2.
    s is the 3-tap filter (-1/4, 1/2, -1/4), so the taps are
        h = delta + a (s*s*s) + b (s*s*s*s),  n = -4..4.
    """
    a = 8.0 * math.sqrt(2.0) - 15.0
    b = 14.0 - 8.0 * math.sqrt(2.0)
    s = np.array([-0.25, 0.5, -0.25])
    s3 = conv1d(conv1d(s, s), s)
    s4 = conv1d(s3, s)
    h = b * s4
    h[1:8] += a * s3
    h[4] += 1.0
    return h


def qmf_highpass(h: np.ndarray) -> np.ndarray:
    """g(n) = (-1)^n h(n) with n counted from the centre tap (Sec. 5.1)."""
    c = (h.size - 1) // 2
    n = np.arange(h.size) - c
    return ((-1.0) ** n) * h


def lowpass_j(h: np.ndarray, j: int) -> np.ndarray:
    """h_j of eq. lowhigh (Sec. 3.1): hat h_j(xi) = prod_{k<j} hat h(2^k xi), h_0 = delta.

    In space: h_j = h * (h up 2) * ... * (h up 2^{j-1}).
    """
    out = np.array([1.0])
    for k in range(j):
        out = conv1d(out, upsample_axis(h, 2 ** k, 0))
    return out


def highpass_j(h: np.ndarray, g: np.ndarray, j: int) -> np.ndarray:
    """g_j of eq. lowhigh (Sec. 3.1): hat g_j(xi) = hat g(2^{j-1} xi) hat h_{j-1}(xi), j >= 1."""
    assert j >= 1
    return conv1d(upsample_axis(g, 2 ** (j - 1), 0), lowpass_j(h, j - 1))


# --------------------------------------------------------------------------------
# 2D fan filter P (Sec. 3.2.1 eq. nonsep; Sec. 5.1)
# --------------------------------------------------------------------------------

#: Coefficients of M(t) = 1/2 + c1 t + c3 t^3 + c5 t^5 + c7 t^7, the maximally flat
#: odd-symmetric polynomial with M(1)=1 and M'(1)=M''(1)=M'''(1)=0.
FAN_POLY = {1: 35.0 / 32.0, 3: -35.0 / 32.0, 5: 21.0 / 32.0, 7: -5.0 / 32.0}


def fan_filter() -> np.ndarray:
    """The 2D fan filter P as 15x15 taps (axis 0 <-> xi_1, axis 1 <-> xi_2).

    Reading: the paper uses the 4th-order maximally flat diamond filter of the
    nonsubsampled contourlet toolbox, divided by sqrt2 and modulated into a fan, but
    prints no taps. Here the diamond filter is D(w) = M((cos w1 + cos w2)/2) with M as
    in FAN_POLY; modulating by (-1)^{n1} gives the fan
        P(w) = M((cos w2 - cos w1)/2),
    which passes |w2| < |w1| (the cone around the xi_1 axis that eq. nonsep needs),
    is real, point-symmetric and half-band: P(w) + P(w + (pi, pi)) = 1.
    In space t = (cos w2 - cos w1)/2 is the 3x3 kernel with -1/4 at (+-1, 0) and
    +1/4 at (0, +-1), and P = delta/2 + sum_m c_m t^{*m}.
    """
    t = np.zeros((3, 3))
    t[0, 1] = t[2, 1] = -0.25
    t[1, 0] = t[1, 2] = 0.25
    P = np.zeros((15, 15))
    P[7, 7] = 0.5
    tp = np.array([[1.0]])
    for m in range(1, 8):
        tp = conv2d_full(tp, t)
        if m in FAN_POLY:
            c = (tp.shape[0] - 1) // 2
            P[7 - c:8 + c, 7 - c:8 + c] += FAN_POLY[m] * tp
    return P


# --------------------------------------------------------------------------------
# Digital shear (Sec. 3.2.2, eqs. dshear1_alpha and dshear2_alpha)
# --------------------------------------------------------------------------------


def shear_integer(f: np.ndarray, k: int) -> np.ndarray:
    """f(S_k n) with S_k = [[1, k], [0, 1]]: out(n1, n2) = f(n1 + k n2, n2).

    Axis 0 carries n1 (the sheared axis), axis 1 carries n2. The support grows along
    axis 0 by |k| * (extent of n2) on each side.
    """
    M, N = f.shape
    cM, cN = (M - 1) // 2, (N - 1) // 2
    cMo = cM + abs(k) * cN
    out = np.zeros((2 * cMo + 1, N))
    for i2 in range(N):
        n2 = i2 - cN
        # out(n1, n2) = f(n1 + k n2, n2): f row i (n1' = i - cM) lands at n1 = n1' - k n2
        start = (0 - cM) - k * n2 + cMo
        out[start:start + M, i2] = f[:, i2]
    return out


def dshear(f: np.ndarray, k: int, d: int, h: np.ndarray) -> np.ndarray:
    """S^d_{k/2^d}(f) along axis 0 (eqs. dshear1_alpha, dshear2_alpha).

    1. refine axis 0 by 2^d:  f~ = (f up 2^d) *_1 (2^d h_d)
       Reading: the paper writes h_d; the factor 2^d restores the amplitude lost to
       the inserted zeros (sum h_d = 1), so that S^d_0 is close to the identity.
    2. shear on the refined grid:  f~(S_k .)
    3. *_1 conj(h_d) (= h_d, h_d is symmetric), then 'down 2^d' on axis 0.
    Reading: the shear sign is x1 <- x1 + k x2 (S_k as in Sec. 2.2.1).
    """
    if d == 0:
        return shear_integer(f, k)
    s = 2 ** d
    hd = lowpass_j(h, d)
    ft = conv_axis(upsample_axis(f, s, 0), s * hd, 0)
    ft = shear_integer(ft, k)
    ft = conv_axis(ft, hd[::-1], 0)
    return downsample_axis(ft, s, 0)


# --------------------------------------------------------------------------------
# Folding onto the N-grid and the DFT
# --------------------------------------------------------------------------------


def fold(a: np.ndarray, dims: Sequence[int]) -> np.ndarray:
    """Periodic fold of a finite, origin-centred array onto Z_{n0} x ... (origin -> 0).

    Reading: filters larger than the grid wrap around (the paper is silent).
    """
    out = np.asarray(a, dtype=np.float64)
    for ax in range(out.ndim):
        N = int(dims[ax])
        c = (out.shape[ax] - 1) // 2
        left = (-c) % N                      # origin moves to index c + left = 0 (mod N)
        right = (-(out.shape[ax] + left)) % N
        pad = [(0, 0)] * out.ndim
        pad[ax] = (left, right)
        o = np.moveaxis(np.pad(out, pad), ax, 0)
        o = o.reshape((-1, N) + o.shape[1:]).sum(axis=0)  # index i -> n = i - c' -> n mod N
        out = np.moveaxis(o, 0, ax)
    return np.ascontiguousarray(out)


def dft_real(a_folded: np.ndarray, l1: Optional[float] = None) -> np.ndarray:
    """DFT of a folded filter. Every filter here is real and point-symmetric, so its
    DFT is real; the (rounding-level) imaginary part is checked and dropped.
    ``l1`` is the l1 norm of the unfolded filter (it bounds |F| and the rounding
    error of the fold); by default that of the folded array."""
    F = _dft.fftn(a_folded)
    scale = float(np.sum(np.abs(a_folded))) if l1 is None else float(l1)
    assert float(np.max(np.abs(F.imag))) <= 1e-12 * scale, "filter spectrum not real"
    return np.ascontiguousarray(F.real)


# --------------------------------------------------------------------------------
# Filter systems
# --------------------------------------------------------------------------------


@dataclass
class FilterMeta:
    scale: int          # j in 0..J-1 coarse -> fine; -1 for the lowpass
    cone: int           # 2D: 1 or 2; 3D: pyramid 1..3; 0 for the lowpass
    k: Tuple[int, ...]  # 2D: (k,); 3D: (k1, k2); () for the lowpass


@dataclass
class ShearletSystem:
    """A digital shearlet system on an N-grid (the oracle's filter bank)."""
    ndim: int
    dims: Tuple[int, ...]
    n_scales: int
    shear_levels: Tuple[int, ...]
    full_system: bool
    meta: List[FilterMeta]
    _filter_fn: Callable[[int], np.ndarray]           # unnormalised psi_hat_j, full grid
    _spatial_fn: Callable[[int], np.ndarray]          # unnormalised folded psi_j
    scale_factor: float = 1.0                         # 1/sqrt(max Psi)
    Psi: Optional[np.ndarray] = None                  # normalised frame weight
    norms: Optional[np.ndarray] = None                # ||psi_j||_2 (normalised)
    _cache: dict = field(default_factory=dict)
    cache_filters: bool = True

    @property
    def R(self) -> int:
        return len(self.meta)

    @property
    def N(self) -> int:
        return int(np.prod(self.dims))

    def psi_hat(self, j: int) -> np.ndarray:
        """Normalised, real DFT of filter j on the full grid."""
        if j in self._cache:
            return self._cache[j]
        F = self._filter_fn(j) * self.scale_factor
        if self.cache_filters:
            self._cache[j] = F
        return F

    def psi_spatial(self, j: int) -> np.ndarray:
        """Normalised filter j folded onto the grid, in space (origin at index 0)."""
        return self._spatial_fn(j) * self.scale_factor

    @property
    def A(self) -> float:
        return float(self.Psi.min())

    @property
    def B(self) -> float:
        return float(self.Psi.max())


def _finish_system(sysm: ShearletSystem) -> ShearletSystem:
    """Frame weight (eq. frame_filter), normalisation and filter norms.

    Reading: the paper's table of frame bounds has B = 1.0000 for every system, so
    all filters are scaled by 1/sqrt(max Psi): then B = 1 and A = min Psi.
    ||psi_j||_2^2 = sum_xi psi_hat_j(xi)^2 / N (Parseval on the grid).
    """
    cache = sysm.cache_filters
    sysm.cache_filters = False
    Psi = np.zeros(sysm.dims)
    sq = np.zeros(sysm.R)
    for j in range(sysm.R):
        F = sysm._filter_fn(j)
        F2 = F * F
        Psi += F2
        sq[j] = float(F2.sum())
    sysm.cache_filters = cache
    m = float(Psi.max())
    sysm.scale_factor = 1.0 / math.sqrt(m)
    sysm.Psi = Psi / m
    sysm.norms = np.sqrt(sq / m / sysm.N)
    return sysm


def _unsheared_2d(h, g, P, J, j, d):
    """p_j * W_j (eq. ext_noshear_alpha), axis 0 = x1, axis 1 = x2.

    p_j: taps of P(2^{J-j-1} xi1, 2^{J-j+d} xi2), i.e. P upsampled by those factors;
    W_j = g_{J-j} (x) h_{J-j+d}  (Sec. 3.2.2, with j - d_j in place of j/2).
    """
    p = upsample_axis(upsample_axis(P, 2 ** (J - j - 1), 0), 2 ** (J - j + d), 1)
    W = np.outer(highpass_j(h, g, J - j), lowpass_j(h, J - j + d))
    return conv2d_full(p, W)


def shear_range(d: int) -> range:
    return range(-(2 ** d), 2 ** d + 1)


def build_system_2d(dims: Sequence[int], n_scales: int, shear_levels: Sequence[int],
                    full_system: bool = False, P: Optional[np.ndarray] = None,
                    h: Optional[np.ndarray] = None) -> ShearletSystem:
    """The 2D digital shearlet system (Def. digitSH_alpha; Sec. 3.4; Sec. 4.4).

    Order (reading, the paper fixes none): index 0 is the lowpass
    phi_hat = h_J(xi1) h_J(xi2) (Sec. 3.4); then scales j = 0..J-1 coarse to fine;
    within a scale cone 1 (psi_{j,k}, k = -2^d..2^d ascending) then cone 2
    (psi~_{j,k}(x1, x2) = psi_{j,k}(x2, x1), eq. convolution01), whose boundary
    filters k = +-2^d are omitted unless full_system (Sec. 4.4).
    Reading of the scale index: J = nScales, d_j = shearLevels[j].
    """
    dims = tuple(int(n) for n in dims)
    J = int(n_scales)
    sl = tuple(int(s) for s in shear_levels)
    assert len(dims) == 2 and len(sl) == J
    h = qmf_lowpass() if h is None else np.asarray(h, dtype=np.float64)
    g = qmf_highpass(h)
    P = fan_filter() if P is None else np.asarray(P, dtype=np.float64)

    spatial: List[np.ndarray] = []
    meta: List[FilterMeta] = []
    spatial.append(np.outer(lowpass_j(h, J), lowpass_j(h, J)))
    meta.append(FilterMeta(-1, 0, ()))
    for j in range(J):
        d = sl[j]
        u = _unsheared_2d(h, g, P, J, j, d)
        for k in shear_range(d):
            spatial.append(dshear(u, k, d, h))
            meta.append(FilterMeta(j, 1, (k,)))
        for k in shear_range(d):
            if not full_system and abs(k) == 2 ** d:
                continue
            spatial.append(dshear(u, k, d, h).T)
            meta.append(FilterMeta(j, 2, (k,)))

    def spatial_fn(i):
        return fold(spatial[i], dims)

    def filter_fn(i):
        return dft_real(spatial_fn(i), float(np.sum(np.abs(spatial[i]))))

    sysm = ShearletSystem(2, dims, J, sl, bool(full_system), meta, filter_fn, spatial_fn)
    return _finish_system(sysm)


def _expand(F2: np.ndarray, ax_a: int, ax_b: int, ndim: int) -> np.ndarray:
    """Place a 2D array whose axis 0 is grid axis ax_a and axis 1 is grid axis ax_b
    into an ndim-dimensional broadcastable array."""
    if ax_a > ax_b:
        F2 = F2.T
        ax_a, ax_b = ax_b, ax_a
    shape = [1] * ndim
    shape[ax_a] = F2.shape[0]
    shape[ax_b] = F2.shape[1]
    return F2.reshape(shape)


def _expand1(F1: np.ndarray, ax: int, ndim: int) -> np.ndarray:
    shape = [1] * ndim
    shape[ax] = F1.size
    return F1.reshape(shape)


# (principal axis, axis sheared by k1, axis sheared by k2) for pyramids 1, 2, 3:
# psi~(x1,x2,x3) = psi(x2,x1,x3) and psi_breve(x1,x2,x3) = psi(x3,x1,x2) (Sec. 3.3.1).
PYRAMID_AXES = {1: (0, 1, 2), 2: (1, 0, 2), 3: (2, 0, 1)}


def _kept_3d(pyr: int, k1: int, k2: int, d: int, full_system: bool) -> bool:
    """Omission of boundary shearlets in 3D (Sec. 4.4).

    Reading: a filter with |k1| = 2^d or |k2| = 2^d lies on the seam between two
    pyramids. Pyramid 1 keeps all (2 2^d + 1)^2 filters, pyramid 2 drops those with
    |k1| = 2^d (its seam with pyramid 1), pyramid 3 drops those with |k1| = 2^d or
    |k2| = 2^d (its seams with pyramids 1 and 2). This leaves 3n^2 - 6n + 4 filters
    per scale (n = 2 2^d + 1), the count the paper gives.
    """
    if full_system:
        return True
    e = 2 ** d
    if pyr == 1:
        return True
    if pyr == 2:
        return abs(k1) != e
    return abs(k1) != e and abs(k2) != e


def build_system_3d(dims: Sequence[int], n_scales: int, shear_levels: Sequence[int],
                    full_system: bool = False, P: Optional[np.ndarray] = None,
                    h: Optional[np.ndarray] = None,
                    cache_filters: Optional[bool] = None) -> ShearletSystem:
    """The 3D digital shearlet system (Defs. 3DdigitSH, 3DdigitSH_alpha; Sec. 4.4).

    psi_hat_{j,k}(xi) = g_hat_{J-j}(xi1) Phi_hat_{j,k1}(xi1, xi2) Phi_hat_{j,k2}(xi1, xi3)
    with Phi_{j,k}(n1, n2) = S^d_{k 2^-d}(h_{J-j+d} *_{x2} p_j)  (eqs. 3Dfilters1/2_alpha).
    Reading: the paper writes *_{x2} in the parabolic case and *_1 in the general
    case; the lowpass acts on the non-principal axis (x2), as in the parabolic case.
    The product is taken on the grid: each factor is folded onto its own 1D or 2D
    grid and transformed, which is the DFT of the 3D filter by the convolution theorem.
    Order (reading): lowpass h_J (x) h_J (x) h_J; scales coarse to fine; within a scale
    pyramid 1, 2, 3, each with k1 outer and k2 inner, ascending.
    """
    dims = tuple(int(n) for n in dims)
    J = int(n_scales)
    sl = tuple(int(s) for s in shear_levels)
    assert len(dims) == 3 and len(sl) == J
    h = qmf_lowpass() if h is None else np.asarray(h, dtype=np.float64)
    g = qmf_highpass(h)
    P = fan_filter() if P is None else np.asarray(P, dtype=np.float64)

    # Spatial factors per scale.
    gj = {}
    Phi = {}
    for j in range(J):
        d = sl[j]
        gj[j] = highpass_j(h, g, J - j)
        p = upsample_axis(upsample_axis(P, 2 ** (J - j - 1), 0), 2 ** (J - j + d), 1)
        v = conv_axis(p, lowpass_j(h, J - j + d), 1)
        for k in shear_range(d):
            Phi[(j, k)] = dshear(v, k, d, h)
    hJ = lowpass_j(h, J)

    meta: List[FilterMeta] = [FilterMeta(-1, 0, ())]
    for j in range(J):
        d = sl[j]
        for pyr in (1, 2, 3):
            for k1 in shear_range(d):
                for k2 in shear_range(d):
                    if _kept_3d(pyr, k1, k2, d, full_system):
                        meta.append(FilterMeta(j, pyr, (k1, k2)))

    dft1 = {}
    dft2 = {}

    def g_hat(j, ax):
        key = (j, ax)
        if key not in dft1:
            dft1[key] = dft_real(fold(gj[j], (dims[ax],)), float(np.sum(np.abs(gj[j]))))
        return dft1[key]

    def phi_hat(j, k, ax_a, ax_b):
        key = (j, k, ax_a, ax_b)
        if key not in dft2:
            dft2[key] = dft_real(fold(Phi[(j, k)], (dims[ax_a], dims[ax_b])),
                                 float(np.sum(np.abs(Phi[(j, k)]))))
        return dft2[key]

    lp_hat = [dft_real(fold(hJ, (dims[ax],))) for ax in range(3)]

    def filter_fn(i):
        m = meta[i]
        if m.scale < 0:
            return (_expand1(lp_hat[0], 0, 3) * _expand1(lp_hat[1], 1, 3)
                    * _expand1(lp_hat[2], 2, 3))
        a, b, c = PYRAMID_AXES[m.cone]
        k1, k2 = m.k
        return (_expand1(g_hat(m.scale, a), a, 3)
                * _expand(phi_hat(m.scale, k1, a, b), a, b, 3)
                * _expand(phi_hat(m.scale, k2, a, c), a, c, 3))

    def spatial_fn(i):
        """Folded 3D filter in space, by brute-force circular convolution of its three
        folded factors (each a function of one or two axes). Tiny grids only."""
        m = meta[i]
        assert int(np.prod(dims)) <= 4096, "spatial 3D filters are for tiny grids"
        if m.scale < 0:
            f = [fold(hJ, (dims[ax],)) for ax in range(3)]
            return np.einsum('i,j,k->ijk', f[0], f[1], f[2])
        a, b, c = PYRAMID_AXES[m.cone]
        k1, k2 = m.k
        f1 = np.zeros(dims)
        f1[tuple(slice(None) if ax == a else 0 for ax in range(3))] = \
            fold(gj[m.scale], (dims[a],))
        F2 = fold(Phi[(m.scale, k1)], (dims[a], dims[b]))
        f2 = np.zeros(dims)
        sl2 = [0, 0, 0]
        sl2[a] = slice(None)
        sl2[b] = slice(None)
        f2[tuple(sl2)] = F2 if a < b else F2.T
        F3 = fold(Phi[(m.scale, k2)], (dims[a], dims[c]))
        f3 = np.zeros(dims)
        sl3 = [0, 0, 0]
        sl3[a] = slice(None)
        sl3[c] = slice(None)
        f3[tuple(sl3)] = F3 if a < c else F3.T
        return circular_convolve(circular_convolve(f1, f2), f3)

    if cache_filters is None:
        cache_filters = int(np.prod(dims)) * len(meta) <= 40_000_000
    sysm = ShearletSystem(3, dims, J, sl, bool(full_system), meta, filter_fn, spatial_fn,
                          cache_filters=cache_filters)
    return _finish_system(sysm)


def build_system_wavelet_2d(dims: Sequence[int], n_scales: int,
                            h: Optional[np.ndarray] = None) -> ShearletSystem:
    """The separable stationary wavelet system (the isotropic dictionary of the image
    decomposition, Sec. 5.5), on the same QMF: the undecimated ("a trous") 2D wavelet
    filters built from h_a and g_a of eq. lowhigh, a = J - j.

    Order: lowpass h_J (x) h_J (the shearlet system's lowpass), then per scale
    j = 0..J-1 coarse to fine: g_a (x) h_a (cone 1), h_a (x) g_a (cone 2), g_a (x) g_a
    (cone 3); axis 0 of each outer product is x1. Built in space, folded onto the grid
    and transformed like the shearlet filters; normalised the same way (max Psi = 1).
    """
    dims = tuple(int(n) for n in dims)
    J = int(n_scales)
    assert len(dims) == 2
    h = qmf_lowpass() if h is None else np.asarray(h, dtype=np.float64)
    g = qmf_highpass(h)
    spatial: List[np.ndarray] = [np.outer(lowpass_j(h, J), lowpass_j(h, J))]
    meta: List[FilterMeta] = [FilterMeta(-1, 0, ())]
    for j in range(J):
        a = J - j
        ha, ga = lowpass_j(h, a), highpass_j(h, g, a)
        for cone, (f1, f2) in enumerate(((ga, ha), (ha, ga), (ga, ga)), start=1):
            spatial.append(np.outer(f1, f2))
            meta.append(FilterMeta(j, cone, ()))

    def spatial_fn(i):
        return fold(spatial[i], dims)

    def filter_fn(i):
        return dft_real(spatial_fn(i), float(np.sum(np.abs(spatial[i]))))

    sysm = ShearletSystem(2, dims, J, (0,) * J, False, meta, filter_fn, spatial_fn)
    return _finish_system(sysm)


def build_system(dims: Sequence[int], n_scales: int, shear_levels: Sequence[int],
                 full_system: bool = False, **kw) -> ShearletSystem:
    if len(dims) == 2:
        return build_system_2d(dims, n_scales, shear_levels, full_system, **kw)
    if len(dims) == 3:
        return build_system_3d(dims, n_scales, shear_levels, full_system, **kw)
    raise ValueError("dims must have 2 or 3 entries")


def redundancy_formula(ndim: int, shear_levels: Sequence[int], full_system: bool) -> int:
    """R as the paper counts it (Secs. 4.1 and 4.4): 1 + sum over scales of
    2(2 2^d + 1) (2D) or 3(2 2^d + 1)^2 (3D), minus the omitted boundary filters
    (2 per scale in 2D, 6n - 4 per scale in 3D, n = 2 2^d + 1)."""
    R = 1
    for d in shear_levels:
        n = 2 * 2 ** d + 1
        if ndim == 2:
            R += 2 * n if full_system else 2 ** (d + 2)
        else:
            R += 3 * n * n if full_system else 3 * n * n - 6 * n + 4
    return R


# --------------------------------------------------------------------------------
# Brute-force helpers (tiny grids)
# --------------------------------------------------------------------------------


def circular_convolve(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """(a * b)(m) = sum_n a(n) b(m - n) on Z_N, by direct summation."""
    dims = a.shape
    out = np.zeros(dims)
    for n in np.ndindex(*dims):
        if a[n] != 0.0:
            out += a[n] * np.roll(b, shift=n, axis=tuple(range(a.ndim)))
    return out


def circular_correlate_direct(x: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(x * conj(psi))(m) = sum_n x(n) psi(n - m) on Z_N, by direct summation
    (eq. convolution with psi-bar(n) = psi(-n))."""
    dims = x.shape
    out = np.zeros(dims)
    for m in np.ndindex(*dims):
        shifted = np.roll(psi, shift=m, axis=tuple(range(x.ndim)))  # psi(n - m)
        out[m] = float(np.sum(x * shifted))
    return out


# --------------------------------------------------------------------------------
# Transforms (Secs. 3.4, 4.1, 4.2, 5.3)
# --------------------------------------------------------------------------------

CoeffSource = Union[np.ndarray, Callable[[int], np.ndarray]]


def forward_iter(x: np.ndarray, sysm: ShearletSystem) -> Iterator[Tuple[int, np.ndarray]]:
    """Yield (j, C_j) with C_j = Re IFFT( FFT(x) * conj(psi_hat_j) ).

    This is Algorithm 1 with the conjugation of the definition, f * conj(psi)
    (eq. convolution, Def. digitSH_alpha); the algorithm box conjugates the signal
    spectrum instead, which for the real filters here would reverse the coefficient
    index (reading: follow the definition)."""
    X = _dft.fftn(np.asarray(x, dtype=np.float64))
    for j in range(sysm.R):
        yield j, np.real(_dft.ifftn(X * np.conj(sysm.psi_hat(j))))


def forward(x: np.ndarray, sysm: ShearletSystem) -> np.ndarray:
    """All coefficients as one array [R][dims]."""
    out = np.empty((sysm.R,) + tuple(sysm.dims))
    for j, C in forward_iter(x, sysm):
        out[j] = C
    return out


def forward_subset(x: np.ndarray, sysm: ShearletSystem, js: Sequence[int]) -> dict:
    """{j: C_j} for the filters in js only: the forward transform's definition
    restricted to a subset of subbands (for sampled checks on large grids)."""
    X = _dft.fftn(np.asarray(x, dtype=np.float64))
    return {j: np.real(_dft.ifftn(X * np.conj(sysm.psi_hat(j)))) for j in js}


def _coeff(C: CoeffSource, j: int) -> np.ndarray:
    return np.asarray(C(j) if callable(C) else C[j], dtype=np.float64)


def adjoint(C: CoeffSource, sysm: ShearletSystem) -> np.ndarray:
    """SH* C = Re IFFT( sum_j FFT(C_j) psi_hat_j ): the adjoint of forward."""
    acc = np.zeros(sysm.dims, dtype=np.complex128)
    for j in range(sysm.R):
        acc += _dft.fftn(_coeff(C, j)) * sysm.psi_hat(j)
    return np.real(_dft.ifftn(acc))


def inverse(C: CoeffSource, sysm: ShearletSystem) -> np.ndarray:
    """Dual-frame reconstruction (eq. reconstruction, Algorithm 2):
    x = Re IFFT( sum_j FFT(C_j) gamma_hat_j ), gamma_hat_j = psi_hat_j / Psi (eq. dual_filter)."""
    acc = np.zeros(sysm.dims, dtype=np.complex128)
    for j in range(sysm.R):
        acc += _dft.fftn(_coeff(C, j)) * (sysm.psi_hat(j) / sysm.Psi)
    return np.real(_dft.ifftn(acc))


def inverse_partial(C: CoeffSource, sysm: ShearletSystem, js: Sequence[int]) -> np.ndarray:
    """The part of the sum in eq. reconstruction that a subset of filters contributes:
    sum_{j in js} FFT(C_j) psi_hat_j (a full complex spectrum). ``C(j)`` or ``C[j]``
    must give C_j for every j in js. Summing the parts of disjoint subsets that cover
    all filters and passing the result to inverse_finish gives inverse (or adjoint)."""
    acc = np.zeros(sysm.dims, dtype=np.complex128)
    for j in js:
        acc += _dft.fftn(_coeff(C, j)) * sysm.psi_hat(j)
    return acc


def inverse_finish(acc: np.ndarray, sysm: ShearletSystem, dual: bool = True) -> np.ndarray:
    """Re IFFT(acc / Psi) (dual frame, eq. reconstruction) or Re IFFT(acc) (adjoint)."""
    return np.real(_dft.ifftn(acc / sysm.Psi if dual else acc))


# --------------------------------------------------------------------------------
# Subsampled transform and its inversion by conjugate gradients (Defs. digitSH,
# digitSH_alpha with sampling; Sec. 3.4; the frame algorithms of Sec. 2.1)
# --------------------------------------------------------------------------------


def sub_steps(sysm: ShearletSystem) -> List[int]:
    """Lattice step of every subband. Reading: the sampling matrix of scale j keeps
    (2^(J-1-j) Z)^2, the finest scale every point, the lowpass (2^(J-1) Z)^2: each
    subband at the rate its passband allows."""
    J = sysm.n_scales
    return [2 ** (J - 1) if m.scale < 0 else 2 ** max(0, J - 1 - m.scale) for m in sysm.meta]


def forward_sub(x: np.ndarray, sysm: ShearletSystem, steps: Optional[Sequence[int]] = None
                ) -> List[np.ndarray]:
    """C_j sampled on its lattice: [C_j[::s_j, ::s_j] for every j] (2D)."""
    steps = sub_steps(sysm) if steps is None else steps
    C = forward(x, sysm)
    return [C[j][::steps[j], ::steps[j]].copy() for j in range(sysm.R)]


def adjoint_sub(c: Sequence[np.ndarray], sysm: ShearletSystem,
                steps: Optional[Sequence[int]] = None) -> np.ndarray:
    """Adjoint of forward_sub: each subband's lattice values put back on the grid
    (zeros elsewhere), then the adjoint of the full transform."""
    steps = sub_steps(sysm) if steps is None else steps
    full = np.zeros((sysm.R,) + tuple(sysm.dims))
    for j in range(sysm.R):
        full[j][::steps[j], ::steps[j]] = c[j]
    return adjoint(full, sysm)


def sub_frame_weight(sysm: ShearletSystem, steps: Optional[Sequence[int]] = None) -> np.ndarray:
    """Psi_sub = sum_j |psi_hat_j|^2 / s_j^2: the frame weight (eq. frame_filter) with
    each subband's sampling density; the preconditioner's symbol."""
    steps = sub_steps(sysm) if steps is None else steps
    return sum(sysm.psi_hat(j) ** 2 / float(steps[j]) ** 2 for j in range(sysm.R))


def cg_inverse_sub(c: Sequence[np.ndarray], sysm: ShearletSystem, iterations: int,
                   precondition: bool = True, steps: Optional[Sequence[int]] = None
                   ) -> Tuple[np.ndarray, List[float]]:
    """Solve S x = T_sub* c, S = T_sub* T_sub, by (preconditioned) conjugate gradients
    from x = 0 for `iterations` steps; returns x and the relative residual after each
    step. The preconditioner (our addition) is the diagonal-in-frequency operator
    v -> IFFT(FFT(v) / Psi_sub)."""
    steps = sub_steps(sysm) if steps is None else steps

    def S(v):
        return adjoint_sub(forward_sub(v, sysm, steps), sysm, steps)
    W = sub_frame_weight(sysm, steps)

    def Pinv(v):
        return np.real(_dft.ifftn(_dft.fftn(v) / W)) if precondition else v
    b = adjoint_sub(c, sysm, steps)
    nb = float(np.sqrt(np.sum(b * b)))
    x = np.zeros(sysm.dims)
    r = b.copy()
    z = Pinv(r)
    p = z.copy()
    rz = float(np.sum(r * z))
    hist = []
    for _ in range(int(iterations)):
        q = S(p)
        alpha = rz / float(np.sum(p * q))
        x = x + alpha * p
        r = r - alpha * q
        z = Pinv(r)
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
        hist.append(float(np.sqrt(np.sum(r * r))) / nb)
    return x, hist


def thresholds(sysm: ShearletSystem, sigma: float, K: Sequence[float]) -> np.ndarray:
    """delta_j = K_{s(j)} sigma ||psi_j||_2 (Sec. 5.3 uses delta_j = K_j sigma; the
    factor ||psi_j||_2, the noise standard deviation in subband j, is the reading).
    The lowpass (index 0) gets delta = 0: it is never thresholded (reading)."""
    d = np.zeros(sysm.R)
    for j, m in enumerate(sysm.meta):
        if m.scale >= 0:
            d[j] = float(K[m.scale]) * float(sigma) * float(sysm.norms[j])
    return d


def hard_threshold(C: np.ndarray, delta: float, dtype=np.float64) -> np.ndarray:
    """T_delta of eq. hard_tresholding: keep x(n) where |x(n)| >= delta, else 0.
    ``dtype`` is the precision in which the comparison is made."""
    C = np.asarray(C)
    keep = np.abs(C.astype(dtype)) >= dtype(delta)
    return np.where(keep, C, 0.0)


def threshold(C: np.ndarray, sysm: ShearletSystem, sigma: float, K: Sequence[float],
              dtype=np.float64) -> np.ndarray:
    """Apply T_{delta_j} to every subband j >= 1 of the coefficient stack."""
    out = np.array(C, dtype=np.float64, copy=True)
    dl = thresholds(sysm, sigma, K)
    for j in range(1, sysm.R):
        if sysm.meta[j].scale >= 0:
            out[j] = hard_threshold(C[j], dl[j], dtype)
    return out


def denoise(x: np.ndarray, sysm: ShearletSystem, sigma: float, K: Sequence[float],
            dtype=np.float64, keep_lowpass: bool = True) -> np.ndarray:
    """f_denoised = T^-1 T_delta T f_noisy (Sec. 5.3), streaming over filters.
    keep_lowpass=False drops the lowpass subband instead of keeping it whole."""
    dl = thresholds(sysm, sigma, K)
    X = _dft.fftn(np.asarray(x, dtype=np.float64))
    acc = np.zeros(sysm.dims, dtype=np.complex128)
    for j in range(sysm.R):
        F = sysm.psi_hat(j)
        if sysm.meta[j].scale < 0 and not keep_lowpass:
            continue
        C = np.real(_dft.ifftn(X * np.conj(F)))
        if sysm.meta[j].scale >= 0:
            C = hard_threshold(C, dl[j], dtype)
        acc += _dft.fftn(C) * (F / sysm.Psi)
    return np.real(_dft.ifftn(acc))


def inpaint_ratio(delta_init: float, delta_min: float, iterations: int) -> float:
    """The factor lambda of the threshold schedule delta_{k+1} = lambda delta_k of the
    inpainting algorithm (Sec. 5.4). Reading: the paper writes lambda = delta_min^(1 /
    (iterations - 1)), i.e. delta_min relative to delta_init; here lambda is chosen so
    that the last iteration thresholds at delta_min itself:
    delta_init lambda^(iterations - 1) = delta_min."""
    if iterations <= 1:
        return 1.0
    return (float(delta_min) / float(delta_init)) ** (1.0 / (iterations - 1))


def inpaint(f_masked: np.ndarray, mask: np.ndarray, sysm: ShearletSystem, delta_init: float,
            delta_min: float, iterations: int, dtype=np.float64) -> np.ndarray:
    """Image inpainting by iterative thresholding (Sec. 5.4, algorithm
    image_inpainting): starting from 0, each iteration adds the residual on the known
    pixels, f_res = M (f_masked - f_inpainted), and replaces f_inpainted by
    T^-1 T_delta T (f_res + f_inpainted); delta then shrinks by inpaint_ratio.
    Reading: T_delta thresholds subband j >= 1 at delta ||psi_j||_2 (the denoising
    convention with K = 1 and sigma = delta) and keeps the lowpass."""
    M = (np.asarray(mask) != 0).astype(np.float64)
    f = np.asarray(f_masked, dtype=np.float64)
    out = np.zeros_like(f)
    lam = inpaint_ratio(delta_init, delta_min, iterations)
    ones = [1.0] * sysm.n_scales
    delta = float(delta_init)
    for _ in range(int(iterations)):
        res = M * (f - out)
        out = denoise(res + out, sysm, delta, ones, dtype)
        delta *= lam
    return out


def decompose(f: np.ndarray, curv: ShearletSystem, iso: ShearletSystem, delta_init: float,
              delta_min: float, iterations: int, dtype=np.float64,
              refresh_residual: bool = True) -> Tuple[np.ndarray, np.ndarray]:
    """Image decomposition by iterative thresholding (Sec. 5.5, algorithm
    image_decomposition): f = f0 + f1, f0 sparse in the shearlet system `curv`
    (curvilinear part), f1 sparse in the wavelet system `iso` (isotropic part).

    Each iteration updates f0 from the residual f - f0 - f1 added to f0, i.e. from
    f - f1, then f1 from f - f0; delta then shrinks by inpaint_ratio's factor.
    Readings (the paper is silent or ambiguous):
    * the residual is recomputed between the two updates, the block-coordinate order
      of the morphological component analysis the paper cites; the printed loop
      computes it once per iteration (refresh_residual=False reproduces that);
    * T_delta thresholds subband j >= 1 at delta ||psi_j||_2, as in inpainting;
    * the curvilinear part has no lowpass (its lowpass subband is dropped), the
      isotropic part keeps its lowpass whole, so smooth content goes to f1.
    """
    f = np.asarray(f, dtype=np.float64)
    f0 = np.zeros_like(f)
    f1 = np.zeros_like(f)
    lam = inpaint_ratio(delta_init, delta_min, iterations)
    delta = float(delta_init)
    for _ in range(int(iterations)):
        f0_old = f0
        f0 = denoise(f - f1, curv, delta, [1.0] * curv.n_scales, dtype, keep_lowpass=False)
        f1 = denoise(f - (f0 if refresh_residual else f0_old), iso, delta,
                     [1.0] * iso.n_scales, dtype)
        delta *= lam
    return f0, f1


def gaussian_kernel(sigma: float = 1.0, radius: int = 3) -> np.ndarray:
    """The discrete 2D Gaussian g of the separation measure (Sec. 5.5): exp(-|n|^2 /
    (2 sigma^2)) on |n_i| <= radius, normalised to sum 1. Reading: sigma = 1 pixel, the
    paper gives no width."""
    n = np.arange(-radius, radius + 1, dtype=np.float64)
    g1 = np.exp(-n * n / (2.0 * sigma * sigma))
    g = np.outer(g1, g1)
    return g / g.sum()


def separation_q(f_true: np.ndarray, f_est: np.ndarray, delta: float,
                 g: Optional[np.ndarray] = None, peak: float = 255.0) -> float:
    """Q(f_est, delta) = ||g * f_true - g * (peak B_delta f_est)|| / ||g * f_true||
    (Sec. 5.5), with B_delta the binarisation |.| >= delta and * circular convolution.
    Reading: the binary images take the values 0 and peak = 255, so the binarised
    estimate is scaled by the peak before the comparison."""
    g = gaussian_kernel() if g is None else g
    gk = np.zeros(np.shape(f_true))
    r = (g.shape[0] - 1) // 2
    gk[:g.shape[0], :g.shape[1]] = g
    gk = np.roll(gk, (-r, -r), axis=(0, 1))                  # centre at the origin
    G = _dft.fftn(gk)
    a = np.real(_dft.ifftn(G * _dft.fftn(np.asarray(f_true, dtype=np.float64))))
    B = peak * (np.abs(np.asarray(f_est, dtype=np.float64)) >= delta)
    b = np.real(_dft.ifftn(G * _dft.fftn(B)))
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(a.ravel()))


def separation_q_opt(f_true: np.ndarray, f_est: np.ndarray) -> Tuple[float, int]:
    """Q_opt = min over delta in {0, ..., 255} of Q (Sec. 5.5), and the minimising delta."""
    qs = [separation_q(f_true, f_est, d) for d in range(256)]
    k = int(np.argmin(qs))
    return float(qs[k]), k


def psnr(f: np.ndarray, g: np.ndarray, peak: float = 255.0) -> float:
    """PSNR = 20 log10( peak sqrt(N) / ||f - g||_F )  (eq. PSNR)."""
    f = np.asarray(f, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    err = float(np.linalg.norm((f - g).ravel()))
    return 20.0 * math.log10(peak * math.sqrt(f.size) / err)
