"""Quality measures the paper reports (Sec. III), written out plainly in
NumPy for the tests.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* ``psnr``: 10 log10(peak^2 / MSE) over all pixels.
* ``ssim``: the SSIM index of Wang, Bovik, Sheikh and Simoncelli (2004), as
  the paper cites it: local statistics under an 11 x 11 circular Gaussian
  window (sigma 1.5, weights normalised to sum 1) at every position where
  the window fits, the index
      ((2 mx my + C1)(2 sxy + C2)) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2))
  with C1 = (0.01 peak)^2, C2 = (0.03 peak)^2, and its mean over the
  positions.  The windowed sums are plain loops over the 121 offsets
  (float64).
"""
from __future__ import annotations

import numpy as np


def gaussian_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    r = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-0.5 * (r[:, None] ** 2 + r[None, :] ** 2) / (sigma * sigma))
    return g / g.sum()


def _windowed(a: np.ndarray, w: np.ndarray) -> np.ndarray:
    """sum_{s,t} w[s,t] a[i+s, j+t] at every position (i, j) where the
    window fits ('valid')."""
    n = w.shape[0]
    H, W = a.shape
    out = np.zeros((H - n + 1, W - n + 1))
    for s in range(n):
        for t in range(n):
            out += w[s, t] * a[s:s + H - n + 1, t:t + W - n + 1]
    return out


def ssim_map(x, y, peak: float = 255.0, size: int = 11, sigma: float = 1.5) -> np.ndarray:
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = gaussian_window(size, sigma)
    mx, my = _windowed(x, w), _windowed(y, w)
    vx = _windowed(x * x, w) - mx * mx
    vy = _windowed(y * y, w) - my * my
    cxy = _windowed(x * y, w) - mx * my
    C1, C2 = (0.01 * peak) ** 2, (0.03 * peak) ** 2
    return ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))


def ssim(x, y, peak: float = 255.0) -> float:
    return float(np.mean(ssim_map(x, y, peak)))


def psnr(x, y, peak: float = 255.0) -> float:
    d = np.asarray(x, np.float64) - np.asarray(y, np.float64)
    mse = float(np.mean(d * d))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(peak * peak / mse)
