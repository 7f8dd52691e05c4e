"""FP64 CPU oracle of the learned shrinkage stage (a small MLP that replaces hard
thresholding). TEST INFRASTRUCTURE: only the tests, the smoke check and the
benchmark's CPU-baseline leg use it; it imports nothing from the CUDA path.

The paper denoises with the hard threshold T_delta of eq. hard_tresholding
(Sec. 5.3), delta_j = K_j sigma. The learned stage keeps that setting (coefficients
of the same digital shearlet transform, the same noise level sigma, the same subband
noise scale s_j = sigma ||psi_j||_2) and replaces the keep-or-kill rule by a gain
g in [0, 1] predicted per coefficient:

  features of coefficient c = C_j(m), with s = sigma ||psi_j||_2:
      x_0            = c / s
      x_1 .. x_nb    = |C_j(m + d)| / s   for the 3x3 (2D) or 3x3x3 (3D) neighbourhood
                       d in {-1, 0, 1}^ndim in row-major order, periodic boundary
      x_nb+1 ..      = E_j, a learned 8-dimensional embedding of subband j
  MLP:  h1 = relu(W1 x + b1)  (64),  h2 = relu(W2 h1 + b2)  (64),
        g  = sigmoid(w3 . h2 + b3),  output  c_hat = g c.
  Training loss over a sample of coefficients: mean ((g c - c_clean) / s)^2.

Parity status: the forward, loss and analytic gradients are pinned by finite
differences in tests/test_mlp.py; the network's values themselves have no
counterpart in the paper.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, Sequence, Tuple

import numpy as np

HIDDEN = 64
EMBED = 8
ORDER = ("W1", "b1", "W2", "b2", "w3", "b3", "E")


def n_features(ndim: int) -> int:
    return 1 + 3 ** ndim + EMBED


def param_shapes(ndim: int, R: int) -> Dict[str, Tuple[int, ...]]:
    """Parameter tensors in the order of the flat parameter vector."""
    F = n_features(ndim)
    return {"W1": (HIDDEN, F), "b1": (HIDDEN,), "W2": (HIDDEN, HIDDEN), "b2": (HIDDEN,),
            "w3": (HIDDEN,), "b3": (1,), "E": (R, EMBED)}


def unflatten(flat: np.ndarray, ndim: int, R: int) -> Dict[str, np.ndarray]:
    out, o = {}, 0
    for k, sh in param_shapes(ndim, R).items():
        n = int(np.prod(sh))
        out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(sh)
        o += n
    assert o == flat.size
    return out


def flatten(p: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(v, dtype=np.float64).ravel() for v in p.values()])


def neighbour_offsets(ndim: int):
    r = (-1, 0, 1)
    if ndim == 2:
        return [(a, b) for a in r for b in r]
    return [(a, b, c) for a in r for b in r for c in r]


def features(C: np.ndarray, j: np.ndarray, m: np.ndarray, s: np.ndarray,
             E: np.ndarray) -> np.ndarray:
    """Feature rows for coefficients (j[i], m[i]) of the stack C[R][dims].

    s[j] = sigma ||psi_j||_2 is the noise scale of subband j."""
    dims = C.shape[1:]
    ndim = len(dims)
    j = np.asarray(j)
    m = np.asarray(m).reshape(len(j), ndim)
    sj = s[j]
    rows = [C[(j,) + tuple(m.T)] / sj]
    for d in neighbour_offsets(ndim):
        idx = tuple(((m[:, a] + d[a]) % dims[a]) for a in range(ndim))
        rows.append(np.abs(C[(j,) + idx]) / sj)
    X = np.stack(rows, axis=1)
    return np.concatenate([X, E[j]], axis=1)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (via float32, round to nearest even), returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _q(a, on):
    return bf16(a) if on else a


def forward(p: Dict[str, np.ndarray], X: np.ndarray, bf16_operands: bool = False):
    """Returns g and the intermediates needed by backward.

    bf16_operands: round the operands of the two matrix products (features, W1, h1,
    W2) to bfloat16 first, as the tensor-core kernels do; arithmetic stays FP64."""
    q = bf16_operands
    z1 = _q(X, q) @ _q(p["W1"], q).T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = _q(h1, q) @ _q(p["W2"], q).T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ p["w3"] + p["b3"][0]
    g = sigmoid(z3)
    return g, (X, z1, h1, z2, h2, z3)


def loss(p, X, c, c_clean, sj) -> float:
    g, _ = forward(p, X)
    r = (g * c - c_clean) / sj
    return float(np.mean(r * r))


def backward(p, X, c, c_clean, sj, j, bf16_operands: bool = False
             ) -> Tuple[float, Dict[str, np.ndarray]]:
    """Loss and its gradient with respect to every parameter (chain rule written out).

    bf16_operands: as in forward, and the operands of the backward products (dz2,
    dz1 and the weights they meet) are rounded to bfloat16 as well."""
    q = bf16_operands
    g, (X, z1, h1, z2, h2, z3) = forward(p, X, q)
    n = X.shape[0]
    r = (g * c - c_clean) / sj
    L = float(np.mean(r * r))
    dg = 2.0 * r * c / sj / n
    dz3 = dg * g * (1.0 - g)
    grads = {}
    grads["w3"] = h2.T @ dz3
    grads["b3"] = np.array([dz3.sum()])
    dz2 = np.outer(dz3, p["w3"]) * (z2 > 0)
    grads["W2"] = _q(dz2, q).T @ _q(h1, q)
    grads["b2"] = dz2.sum(axis=0)
    dz1 = (_q(dz2, q) @ _q(p["W2"], q)) * (z1 > 0)
    grads["W1"] = _q(dz1, q).T @ _q(X, q)
    grads["b1"] = dz1.sum(axis=0)
    dX = _q(dz1, q) @ _q(p["W1"], q)
    dE = np.zeros_like(p["E"])
    np.add.at(dE, j, dX[:, X.shape[1] - EMBED:])
    grads["E"] = dE
    return L, {k: grads[k] for k in ORDER}


def adam_step(flat: np.ndarray, grad: np.ndarray, m: np.ndarray, v: np.ndarray, t: int,
              lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba) of flat parameters, in place; t counts from 1."""
    m *= b1
    m += (1 - b1) * grad
    v *= b2
    v += (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    flat -= lr * mh / (np.sqrt(vh) + eps)


def apply(p, C: np.ndarray, s: np.ndarray, bf16_operands: bool = False) -> np.ndarray:
    """c_hat = g c for every coefficient of every subband j >= 1 (lowpass untouched)."""
    out = np.array(C, dtype=np.float64, copy=True)
    dims = C.shape[1:]
    grid = np.stack(np.meshgrid(*[np.arange(n) for n in dims], indexing="ij"), -1)
    m = grid.reshape(-1, len(dims))
    for jj in range(1, C.shape[0]):
        j = np.full(m.shape[0], jj)
        g, _ = forward(p, features(C, j, m, s, p["E"]), bf16_operands)
        out[jj] = (g * C[jj].ravel()).reshape(dims)
    return out
