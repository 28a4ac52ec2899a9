"""Seeded synthetic inputs: phantoms, measurement noise and the DIP input.

This module holds none of the operator arithmetic; it only draws and renders
images and random arrays.  It is the one module that both the CPU oracle's
tests and the GPU path's tests/benchmarks take inputs from.  The phantoms
stand in for the paper's simulated phantom and digital-twin data
(Sec. 2.4.1-2.4.2), which are not available here.

Conventions
-----------
* Images are N x N on [-1,1]^2, row iy <-> y = -1 + (iy + 1/2) h, column
  ix <-> x, h = 2/N; arrays are float64 ``[iy, ix]``.
* Gaussian blob: ``a * exp(-|x - c|^2 / sigma^2)`` (sigma^2, not 2 sigma^2).
* Vessel tube: polyline; a pixel gets ``a * coverage`` where coverage is the
  fraction of its 4 x 4 sub-samples within ``width_px * h / 2`` of the
  polyline; tubes combine by maximum, Gaussians add.
* Noise: i.i.d. normal, scaled either to ``level * max|g|`` (standard
  deviation) or to a relative L2 norm ``||delta|| = level * ||g||``
  (the convention of Sec. 2.4.1 and Sec. 3.1).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "pixel_centres", "gaussian_phantom", "vessel_phantom", "mixed_phantom",
    "add_noise", "dip_input", "random_image", "random_data",
]


def pixel_centres(n: int) -> np.ndarray:
    h = 2.0 / n
    return -1.0 + (np.arange(n) + 0.5) * h


def _uniform_in_disk(rng: np.random.Generator, radius: float) -> np.ndarray:
    r = radius * math.sqrt(rng.uniform())
    t = rng.uniform(0.0, 2.0 * math.pi)
    return np.array([r * math.cos(t), r * math.sin(t)])


def gaussian_phantom(n: int, count: int = 5, seed: int = 1, r_max: float = 0.8,
                     sigma=(0.03, 0.1), amp=(0.5, 1.0)) -> np.ndarray:
    """Sum of ``count`` isotropic Gaussians, centres uniform in the disk r < r_max."""
    rng = np.random.default_rng(seed)
    x = pixel_centres(n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    f = np.zeros((n, n))
    for _ in range(count):
        c = _uniform_in_disk(rng, r_max)
        s = rng.uniform(*sigma)
        a = rng.uniform(*amp)
        f += a * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2) / (s * s))
    return f


def _polyline(rng: np.random.Generator, r_max: float) -> np.ndarray:
    n_vert = int(rng.integers(3, 7))
    pts = [_uniform_in_disk(rng, r_max)]
    heading = rng.uniform(0.0, 2.0 * math.pi)
    while len(pts) < n_vert:
        for _ in range(64):
            turn = rng.uniform(-math.pi / 4, math.pi / 4)
            length = rng.uniform(0.1, 0.4)
            h2 = heading + turn
            p = pts[-1] + length * np.array([math.cos(h2), math.sin(h2)])
            if np.hypot(*p) < r_max:
                heading = h2
                pts.append(p)
                break
        else:  # boxed in: reverse direction and try again
            heading += math.pi
    return np.array(pts)


def _render_tube(n: int, poly: np.ndarray, half_width: float, amp: float, out: np.ndarray) -> None:
    h = 2.0 / n
    sub = (np.arange(4) + 0.5) / 4.0 - 0.5  # 4 x 4 supersampling offsets in pixels
    lo = poly.min(axis=0) - half_width - h
    hi = poly.max(axis=0) + half_width + h
    ix0 = max(int(math.floor((lo[0] + 1) / h)), 0)
    ix1 = min(int(math.ceil((hi[0] + 1) / h)), n)
    iy0 = max(int(math.floor((lo[1] + 1) / h)), 0)
    iy1 = min(int(math.ceil((hi[1] + 1) / h)), n)
    if ix0 >= ix1 or iy0 >= iy1:
        return
    xs = -1.0 + (np.arange(ix0, ix1)[:, None] + 0.5 + sub[None, :]) * h  # (nx, 4)
    ys = -1.0 + (np.arange(iy0, iy1)[:, None] + 0.5 + sub[None, :]) * h  # (ny, 4)
    PX = xs[None, None, :, :]  # (1, 1, nx, 4)
    PY = ys[:, :, None, None]  # (ny, 4, 1, 1)
    d2 = np.full((ys.shape[0], 4, xs.shape[0], 4), np.inf)
    for a, b in zip(poly[:-1], poly[1:]):
        # only the segment's own box (widened by the half width) can be within
        # half_width of it, so the coverage test below sees the same answer
        slo = np.minimum(a, b) - half_width - h
        shi = np.maximum(a, b) + half_width + h
        sx0 = max(int(math.floor((slo[0] + 1) / h)), ix0) - ix0
        sx1 = min(int(math.ceil((shi[0] + 1) / h)), ix1) - ix0
        sy0 = max(int(math.floor((slo[1] + 1) / h)), iy0) - iy0
        sy1 = min(int(math.ceil((shi[1] + 1) / h)), iy1) - iy0
        if sx0 >= sx1 or sy0 >= sy1:
            continue
        px, py = PX[:, :, sx0:sx1, :], PY[sy0:sy1]
        ab = b - a
        L2 = float(ab @ ab)
        t = ((px - a[0]) * ab[0] + (py - a[1]) * ab[1]) / L2
        t = np.clip(t, 0.0, 1.0)
        dx = px - (a[0] + t * ab[0])
        dy = py - (a[1] + t * ab[1])
        blk = d2[sy0:sy1, :, sx0:sx1, :]
        np.minimum(blk, dx * dx + dy * dy, out=blk)
    cover = (d2 <= half_width * half_width).mean(axis=(1, 3))
    np.maximum(out[iy0:iy1, ix0:ix1], amp * cover, out=out[iy0:iy1, ix0:ix1])


def vessel_phantom(n: int, count: int = 12, seed: int = 2, r_max: float = 0.9,
                   width_px=(2.0, 4.0), amp=(0.3, 1.0)) -> np.ndarray:
    """``count`` random piecewise-linear tubes inside the disk r < r_max."""
    rng = np.random.default_rng(seed)
    h = 2.0 / n
    f = np.zeros((n, n))
    for _ in range(count):
        poly = _polyline(rng, r_max)
        w = rng.uniform(*width_px)
        a = rng.uniform(*amp)
        _render_tube(n, poly, 0.5 * w * h, a, f)
    return f


def mixed_phantom(n: int, tubes: int, gaussians: int, seed: int,
                  width_px=(2.0, 4.0)) -> np.ndarray:
    """Vessel tubes plus Gaussian blobs (blobs add onto the tube image)."""
    return vessel_phantom(n, tubes, seed=seed, width_px=width_px) + gaussian_phantom(
        n, gaussians, seed=seed + 100_000)


def add_noise(g: np.ndarray, level: float, seed: int, mode: str = "max") -> np.ndarray:
    """Return ``g + delta`` with i.i.d. normal delta.

    mode "max": std = level * max|g|;  mode "rel_l2": ||delta|| = level * ||g||.
    """
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(g.shape)
    if mode == "max":
        return g + level * np.abs(g).max() * z
    if mode == "rel_l2":
        return g + level * np.linalg.norm(g) / max(np.linalg.norm(z), 1e-300) * z
    raise ValueError(mode)


def dip_input(channels: int, n: int, seed: int = 3, std: float = 0.1) -> np.ndarray:
    """Fixed DIP network input z ~ N(0, std^2), shape (1, channels, n, n)."""
    rng = np.random.default_rng(seed)
    return std * rng.standard_normal((1, channels, n, n))


def random_image(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal((n, n))


def random_data(n_det: int, n_t: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal((n_det, n_t))
