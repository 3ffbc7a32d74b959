"""Seeded synthetic inputs for the FoE despeckling solver.

This module only *draws* inputs: clean images, speckled observations and the
filter bank that stands in for the learned 48 x 7 x 7 FoE bank (Fig. 1 of the
paper, whose learned weights are not available).  It holds none of the
method's arithmetic (no convolution, potential, gradient, prox or iPiano
step), so both the CUDA path and the FP64 oracle can be fed from it without
sharing any of the computation they are compared on.

All generators use NumPy's PCG64 with an explicit seed and return C-contiguous
float32 arrays (row-major, pitch = width), the layout the C ABI takes.

Noise model (Sec. II-B): the observation is f = u * n with n ~ Gamma(shape L,
scale 1/L), i.e. intensity speckle of mean 1 with L looks.  For L = 1 this is
the unit exponential.  The paper's Nakagami amplitude model (f = u * sqrt(n))
is available with ``amplitude=True``; the solver takes f as given either way.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng_for",
    "piecewise_image",
    "textured_image",
    "speckle",
    "filter_bank",
    "uneven_sizes",
    "psnr",
]

LO, HI = 10.0, 250.0


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _voronoi_levels(rng, H, W, n_regions):
    cy = rng.uniform(0, H, n_regions)
    cx = rng.uniform(0, W, n_regions)
    levels = rng.uniform(LO, HI, n_regions)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    best = np.full((H, W), np.inf)
    lab = np.zeros((H, W), dtype=np.int64)
    for r in range(n_regions):
        d = (yy - cy[r]) ** 2 + (xx - cx[r]) ** 2
        m = d < best
        best[m] = d[m]
        lab[m] = r
    return levels[lab]


def _rectangles(rng, u, n_rect):
    H, W = u.shape
    for _ in range(n_rect):
        h = int(rng.integers(max(2, H // 8), max(3, H // 2)))
        w = int(rng.integers(max(2, W // 8), max(3, W // 2)))
        y0 = int(rng.integers(0, H - h + 1))
        x0 = int(rng.integers(0, W - w + 1))
        u[y0:y0 + h, x0:x0 + w] = rng.uniform(LO, HI)
    return u


def _ramps(rng, u, n_ramps):
    H, W = u.shape
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    for _ in range(n_ramps):
        h = int(rng.integers(max(2, H // 4), max(3, H // 2 + 1)))
        w = int(rng.integers(max(2, W // 4), max(3, W // 2 + 1)))
        y0 = int(rng.integers(0, H - h + 1))
        x0 = int(rng.integers(0, W - w + 1))
        ang = rng.uniform(0.0, 2.0 * np.pi)
        a, b = rng.uniform(LO, HI, 2)
        # linear ramp from level a to level b along direction ang over the box
        t = ((yy - y0) * np.sin(ang) + (xx - x0) * np.cos(ang))
        sl = (slice(y0, y0 + h), slice(x0, x0 + w))
        tt = t[sl]
        span = max(tt.max() - tt.min(), 1e-9)
        u[sl] = a + (b - a) * (tt - tt.min()) / span
    return u


def piecewise_image(H: int = 64, W: int = 64, seed: int = 0,
                    n_regions: int = 8, n_rect: int = 2, n_ramps: int = 2) -> np.ndarray:
    """Piecewise-constant regions (Voronoi cells + rectangles) with constant
    levels U[10, 250] plus linear ramps, clipped to [10, 250]."""
    rng = rng_for(seed)
    u = _voronoi_levels(rng, H, W, n_regions)
    u = _rectangles(rng, u, n_rect)
    u = _ramps(rng, u, n_ramps)
    return np.ascontiguousarray(np.clip(u, LO, HI), dtype=np.float32)


def textured_image(H: int = 256, W: int = 256, seed: int = 0,
                   n_regions: int = 12, n_tex: int = 4, max_amp: float = 20.0) -> np.ndarray:
    """Regions + smooth gradients + seeded sinusoidal textures (amplitude
    <= max_amp, random frequency and orientation), clipped to [10, 250]."""
    rng = rng_for(seed)
    u = _voronoi_levels(rng, H, W, n_regions)
    u = _rectangles(rng, u, 2)
    u = _ramps(rng, u, 2)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    # smooth global gradient
    gy, gx = rng.uniform(-30.0, 30.0, 2)
    u = u + gy * (yy / max(H - 1, 1) - 0.5) + gx * (xx / max(W - 1, 1) - 0.5)
    for _ in range(n_tex):
        h = int(rng.integers(max(2, H // 6), max(3, H // 2 + 1)))
        w = int(rng.integers(max(2, W // 6), max(3, W // 2 + 1)))
        y0 = int(rng.integers(0, H - h + 1))
        x0 = int(rng.integers(0, W - w + 1))
        amp = rng.uniform(0.25 * max_amp, max_amp)
        freq = rng.uniform(0.05, 0.6)   # radians per pixel
        ang = rng.uniform(0.0, np.pi)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        sl = (slice(y0, y0 + h), slice(x0, x0 + w))
        u[sl] = u[sl] + amp * np.sin(freq * (yy[sl] * np.sin(ang) + xx[sl] * np.cos(ang)) + ph)
    return np.ascontiguousarray(np.clip(u, LO, HI), dtype=np.float32)


def speckle(u: np.ndarray, L: float = 1.0, seed: int = 1, amplitude: bool = False) -> np.ndarray:
    """f = u * n, n ~ Gamma(L, 1/L) (mean 1).  ``amplitude`` draws the
    Nakagami amplitude observation f = u * sqrt(n) instead."""
    rng = rng_for(seed)
    n = rng.gamma(shape=float(L), scale=1.0 / float(L), size=u.shape)
    # Gamma draws are positive almost surely; guard the measure-zero case so
    # that every observation is strictly positive (the data term needs f > 0).
    n = np.maximum(n, np.finfo(np.float32).tiny * 1e6)
    if amplitude:
        n = np.sqrt(n)
    return np.ascontiguousarray(u.astype(np.float64) * n, dtype=np.float32)


def filter_bank(nf: int = 48, ks: int = 7, seed: int = 0, theta: float = 0.1):
    """Seeded stand-in for the learned FoE bank: N(0,1) draws, each filter
    projected to zero mean and then scaled to unit Frobenius norm (in FP64),
    stored as float32; every weight theta_i = ``theta``.

    Returns (filters[nf, ks, ks] float32, theta[nf] float32)."""
    rng = rng_for(seed)
    k = rng.standard_normal((nf, ks, ks))
    k = k - k.mean(axis=(1, 2), keepdims=True)
    k = k / np.sqrt((k * k).sum(axis=(1, 2), keepdims=True))
    return (np.ascontiguousarray(k, dtype=np.float32),
            np.full(nf, theta, dtype=np.float32))


def uneven_sizes(n: int = 64, lo: int = 128, hi: int = 1536, seed: int = 7):
    """n square side lengths drawn log-uniformly in [lo, hi] (integers)."""
    rng = rng_for(seed)
    s = np.exp(rng.uniform(np.log(lo), np.log(hi), n))
    return [int(round(v)) for v in s]


def psnr(u: np.ndarray, ref: np.ndarray, peak: float = 255.0) -> float:
    """10 log10(peak^2 / MSE) over all pixels, no clipping."""
    d = np.asarray(u, np.float64) - np.asarray(ref, np.float64)
    mse = float(np.mean(d * d))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(peak * peak / mse)
