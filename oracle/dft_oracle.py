"""The oracle's own discrete Fourier transforms, FP64.

TEST INFRASTRUCTURE, like the rest of this package: only the tests, the smoke check
and the CPU-baseline leg of the benchmark use it. It shares nothing with the CUDA
library.

Convention (the one Algorithm 1 of the paper uses through MATLAB's fft/ifft):
    DFT:  X[k] = sum_n x[n] exp(-2 pi i n k / n_len)
    IDFT: x[n] = (1 / n_len) sum_k X[k] exp(+2 pi i n k / n_len)
applied along every axis for the multidimensional transforms.

Two routes that share no code beyond the angle reduction:

* ``dft_direct``: the defining sum as a product with the n_len x n_len matrix of
  exponentials (tiny lengths, and the reference the FFT is checked against);
* ``fft``: decimation in time by the smallest prime factor p of the length
  (radix 2 for the power-of-two grids, one radix-3 step for 192 = 3 * 64 and
  384 = 3 * 128), recursing on the p interleaved subsequences, down to the direct
  sum at length <= 8. With n = p i + r and k = k1 + (n_len / p) k2,
      X[k] = sum_r exp(-2 pi i r k2 / p) * exp(-2 pi i r k1 / n_len) * Y_r[k1],
  Y_r the length-(n_len / p) DFT of x[p i + r].
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def _expo(num: np.ndarray, n_len: int, sign: int) -> np.ndarray:
    """exp(sign 2 pi i num / n_len) for integer num, with num reduced mod n_len first
    so that the angle stays in [0, 2 pi) and keeps full FP64 accuracy."""
    m = np.mod(num, n_len).astype(np.float64)
    return np.exp(sign * 2j * np.pi * m / n_len)


def _twiddle(r: np.ndarray, k1: np.ndarray, n_len: int, sign: int) -> np.ndarray:
    """The inter-stage factors exp(sign 2 pi i r k1 / n_len), indexed [r, k1]."""
    return _expo(np.outer(r, k1), n_len, sign)


def dft_direct(x: np.ndarray, axis: int = -1, sign: int = -1) -> np.ndarray:
    """The defining sum along ``axis`` (unnormalised; sign -1 forward, +1 inverse)."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n_len = x.shape[-1]
    idx = np.arange(n_len)
    W = _expo(np.outer(idx, idx), n_len, sign)      # W[n, k]
    return np.moveaxis(x @ W, -1, axis)


def _smallest_factor(n_len: int) -> int:
    p = 2
    while n_len % p:
        p += 1
    return p


def _fft_last(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised DFT along the last axis by recursive decimation in time."""
    n_len = x.shape[-1]
    if n_len <= 8:
        return dft_direct(x, -1, sign)
    p = _smallest_factor(n_len)
    q = n_len // p
    # subsequence r holds x[p i + r], i = 0..q-1: shape (..., p, q)
    sub = np.swapaxes(x.reshape(x.shape[:-1] + (q, p)), -1, -2)
    Y = _fft_last(sub, sign)                                   # (..., p[r], q[k1])
    r = np.arange(p)
    k1 = np.arange(q)
    T = Y * _twiddle(r, k1, n_len, sign)                        # W_n^{r k1}
    if p == 2:                                                  # X = T0 +- T1
        X = np.concatenate((T[..., 0, :] + T[..., 1, :], T[..., 0, :] - T[..., 1, :]), axis=-1)
        return X
    Wp = _expo(np.outer(r, r), p, sign)                         # Wp[r, k2]
    X = np.einsum("...rk,rs->...sk", T, Wp)                     # (..., p[k2], q[k1])
    return X.reshape(x.shape[:-1] + (n_len,))


def fft(x: np.ndarray, axis: int = -1, sign: int = -1) -> np.ndarray:
    """Unnormalised DFT along ``axis`` (sign -1 forward, +1 inverse)."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    return np.moveaxis(_fft_last(np.ascontiguousarray(x), sign), -1, axis)


def fftn(x: np.ndarray, axes: Sequence[int] = None) -> np.ndarray:
    """Forward DFT along every axis (or ``axes``)."""
    out = np.asarray(x, dtype=np.complex128)
    for ax in (range(out.ndim) if axes is None else axes):
        out = fft(out, ax, -1)
    return out


def ifftn(X: np.ndarray, axes: Sequence[int] = None) -> np.ndarray:
    """Inverse DFT along every axis (or ``axes``), normalised by the grid size."""
    out = np.asarray(X, dtype=np.complex128)
    axes = range(out.ndim) if axes is None else axes
    n_tot = 1
    for ax in axes:
        out = fft(out, ax, +1)
        n_tot *= out.shape[ax]
    return out / n_tot
