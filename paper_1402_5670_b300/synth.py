"""Seeded synthetic inputs shaped like the paper's workloads.

The paper denoises 512x512 grayscale natural images with additive Gaussian noise
(Sec. 5.3) and 192x192x192 grayscale videos (Sec. 5.6). Those images and videos are
not available here; these generators stand in for them with cartoon-like content of
the same shape and value range: piecewise-smooth images (ellipses with smooth
intensity ramps and curved edges, values in [0, 255]) and volumes of moving
ellipses (one frame per index of axis 0).

This module holds no shearlet arithmetic. It is shared by the tests, the benchmark
and the oracle checks so that every side sees the same inputs.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(int(seed)))


def piecewise_smooth_image(shape: Sequence[int], seed: int) -> np.ndarray:
    """A cartoon-like image in [0, 255] (float32): a smooth background ramp, 12
    rotated ellipses drawn on top of each other, each with its own linear intensity
    ramp, and 3 curved edges y > a sin(w x + phi) + b that add a step."""
    n0, n1 = int(shape[0]), int(shape[1])
    r = _rng(seed)
    y, x = np.meshgrid(np.arange(n0, dtype=np.float64), np.arange(n1, dtype=np.float64),
                       indexing="ij")
    m = float(max(n0, n1))
    img = (r.uniform(60, 140) + r.uniform(-40, 40) * (y / n0 - 0.5)
           + r.uniform(-40, 40) * (x / n1 - 0.5))
    for _ in range(12):
        cy, cx = r.uniform(0, n0), r.uniform(0, n1)
        ay, ax = r.uniform(m / 16, m / 3), r.uniform(m / 16, m / 3)
        th = r.uniform(0, np.pi)
        c, s = np.cos(th), np.sin(th)
        u = ((y - cy) * c + (x - cx) * s) / ay
        v = (-(y - cy) * s + (x - cx) * c) / ax
        inside = (u * u + v * v) <= 1.0
        gy, gx = r.uniform(-1, 1, size=2)
        val = r.uniform(20, 235) + 30.0 * (gy * (y - cy) + gx * (x - cx)) / m
        img = np.where(inside, val, img)
    for _ in range(3):
        a = r.uniform(0.02, 0.15) * n0
        w = r.uniform(1.0, 6.0) * 2 * np.pi / n1
        phi = r.uniform(0, 2 * np.pi)
        b = r.uniform(0.1, 0.9) * n0
        step = r.uniform(-40, 40)
        img = np.where(y > a * np.sin(w * x + phi) + b, img + step, img)
    return np.clip(img, 0.0, 255.0).astype(np.float32)


def moving_ellipses_volume(shape: Sequence[int], seed: int) -> np.ndarray:
    """A video volume in [0, 255] (float32), frames along axis 0: a smooth background
    and 6 ellipses that move at constant velocity (at most 1.5 pixels per frame),
    each with a smooth intensity ramp that drifts slowly over time."""
    n0, n1, n2 = (int(s) for s in shape)
    r = _rng(seed)
    y, x = np.meshgrid(np.arange(n1, dtype=np.float64), np.arange(n2, dtype=np.float64),
                       indexing="ij")
    m = float(max(n1, n2))
    bg0 = r.uniform(60, 140)
    bgy, bgx = r.uniform(-30, 30, size=2)
    objs = []
    for _ in range(6):
        objs.append(dict(
            cy=r.uniform(0, n1), cx=r.uniform(0, n2),
            vy=r.uniform(-1.5, 1.5) / np.sqrt(2), vx=r.uniform(-1.5, 1.5) / np.sqrt(2),
            ay=r.uniform(m / 12, m / 4), ax=r.uniform(m / 12, m / 4),
            th=r.uniform(0, np.pi), val=r.uniform(20, 235),
            gy=r.uniform(-1, 1), gx=r.uniform(-1, 1), dval=r.uniform(-0.3, 0.3)))
    vol = np.empty((n0, n1, n2), dtype=np.float32)
    for t in range(n0):
        img = bg0 + bgy * (y / n1 - 0.5) + bgx * (x / n2 - 0.5)
        for o in objs:
            cy = (o["cy"] + o["vy"] * t) % n1
            cx = (o["cx"] + o["vx"] * t) % n2
            c, s = np.cos(o["th"]), np.sin(o["th"])
            u = ((y - cy) * c + (x - cx) * s) / o["ay"]
            v = (-(y - cy) * s + (x - cx) * c) / o["ax"]
            inside = (u * u + v * v) <= 1.0
            val = o["val"] + o["dval"] * t + 30.0 * (o["gy"] * (y - cy) + o["gx"] * (x - cx)) / m
            img = np.where(inside, val, img)
        vol[t] = np.clip(img, 0.0, 255.0)
    return vol


def points_and_curves(shape: Sequence[int], seed: int, n_curves: int = 4, n_points: int = 40,
                      peak: float = 255.0) -> Tuple[np.ndarray, np.ndarray]:
    """The two binary parts of a decomposition test image (Sec. 5.5 separates an image
    of curves and points): (curves, points), float32 with values 0 and ``peak``.
    curves: ``n_curves`` sine-shaped curves y = a sin(w x + phi) + b about 1.5 pixels
    thick, half of them drawn along the other axis; points: ``n_points`` disks of
    radius U[1.5, 3]. The image to decompose is their sum."""
    n0, n1 = int(shape[0]), int(shape[1])
    r = _rng(seed)
    y, x = np.meshgrid(np.arange(n0, dtype=np.float64), np.arange(n1, dtype=np.float64),
                       indexing="ij")
    curves = np.zeros((n0, n1), dtype=bool)
    for i in range(int(n_curves)):
        u, v, nu, nv = (y, x, n0, n1) if i % 2 == 0 else (x, y, n1, n0)
        a = r.uniform(0.05, 0.2) * nu
        w = r.uniform(0.5, 2.0) * 2 * np.pi / nv
        phi = r.uniform(0, 2 * np.pi)
        b = r.uniform(0.2, 0.8) * nu
        # distance to the curve along u, scaled by the local slope
        slope = a * w * np.cos(w * v + phi)
        dist = np.abs(u - (a * np.sin(w * v + phi) + b)) / np.sqrt(1.0 + slope * slope)
        curves |= dist <= 0.75
    points = np.zeros((n0, n1), dtype=bool)
    for _ in range(int(n_points)):
        cy, cx = r.uniform(0, n0), r.uniform(0, n1)
        rad = r.uniform(1.5, 3.0)
        points |= (y - cy) ** 2 + (x - cx) ** 2 <= rad * rad
    return (peak * curves).astype(np.float32), (peak * points).astype(np.float32)


def add_noise(x: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """x + e with e ~ N(0, sigma^2) i.i.d. (Sec. 5.3); not clipped (float32)."""
    r = _rng(seed)
    return (np.asarray(x, dtype=np.float64)
            + float(sigma) * r.standard_normal(np.shape(x))).astype(np.float32)


def gaussian_field(shape: Sequence[int], seed: int, scale: float = 1.0) -> np.ndarray:
    """i.i.d. N(0, scale^2) samples (float32), e.g. random coefficient stacks."""
    return (float(scale) * _rng(seed).standard_normal(tuple(shape))).astype(np.float32)


def random_mask(shape: Sequence[int], missing: float, seed: int) -> np.ndarray:
    """Binary mask (uint8, 1 = known pixel) with a fraction ``missing`` of the pixels
    occluded at random (the paper's "Random" mask occludes 80%)."""
    return (_rng(seed).random(tuple(shape)) >= float(missing)).astype(np.uint8)


def squares_mask(shape: Sequence[int], n_squares: int, side: int, seed: int) -> np.ndarray:
    """Binary mask (uint8, 1 = known pixel) with ``n_squares`` occluded squares of
    ``side`` pixels at random positions (the paper's "Squares" mask)."""
    r = _rng(seed)
    m = np.ones(tuple(shape), dtype=np.uint8)
    for _ in range(int(n_squares)):
        y = int(r.integers(0, max(1, shape[0] - side)))
        x = int(r.integers(0, max(1, shape[1] - side)))
        m[y:y + side, x:x + side] = 0
    return m


def uneven_batch_shapes(n: int, sides: Sequence[int], seed: int) -> List[Tuple[int, int]]:
    """n image shapes (n0, n1) with each side drawn independently from ``sides``."""
    r = _rng(seed)
    s = np.asarray(list(sides))
    return [(int(r.choice(s)), int(r.choice(s))) for _ in range(n)]


def mlp_init(ndim: int, R: int, seed: int) -> np.ndarray:
    """Seeded initial parameters of the learned-shrinkage MLP (flat float32 in the
    library's layout W1[64][F], b1[64], W2[64][64], b2[64], w3[64], b3, E[R][8] with
    F = 1 + 3^ndim + 8): uniform fan-in scaling for the weights, zero hidden biases,
    b3 = 2 (the initial gain sigmoid(2) ~ 0.88 keeps most of each coefficient) and a
    small random subband embedding."""
    r = _rng(seed)
    F = 1 + 3 ** ndim + 8
    parts = [r.uniform(-1, 1, (64, F)) / np.sqrt(F), np.zeros(64),
             r.uniform(-1, 1, (64, 64)) / 8.0, np.zeros(64),
             r.uniform(-1, 1, 64) / 8.0, np.array([2.0]),
             0.1 * r.standard_normal((R, 8))]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)
