"""Pins for the quality measures of the oracle (oracle/quality.py): SSIM as
defined by Wang et al. (2004), cited in Sec. III, and PSNR."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def q():
    from oracle import quality
    return quality


def _pair(H=23, W=29, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(10, 250, (H, W))
    y = x * rng.gamma(4.0, 0.25, (H, W))
    return x, y


def test_gaussian_window(q):
    w = q.gaussian_window()
    assert w.shape == (11, 11) and w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.array_equal(w, w.T) and np.array_equal(w, w[::-1, ::-1])
    assert w[5, 5] == w.max()
    assert w[5, 5] / w[5, 6] == pytest.approx(np.exp(1.0 / (2 * 1.5 ** 2)), rel=1e-13)


def test_identity_symmetry_and_range(q):
    x, y = _pair()
    assert q.ssim(x, x) == 1.0
    assert q.ssim(x, y) == q.ssim(y, x)
    m = q.ssim_map(x, y)
    assert m.shape == (23 - 10, 29 - 10)
    assert np.all(np.abs(m) <= 1.0) and q.ssim(x, y) < 0.9


def test_constant_images_closed_form(q):
    a, b = 80.0, 130.0
    C1 = (0.01 * 255) ** 2
    ref = (2 * a * b + C1) / (a * a + b * b + C1)
    assert q.ssim(np.full((15, 16), a), np.full((15, 16), b)) == pytest.approx(ref, rel=1e-12)


def test_brute_force_per_window(q):
    """Per position: weighted mean, variance and covariance of the 11 x 11
    patch with np.sum, then the index - a separate code path."""
    x, y = _pair(15, 17, seed=3)
    w = q.gaussian_window()
    C1, C2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2
    m = np.empty((5, 7))
    for i in range(5):
        for j in range(7):
            px, py = x[i:i + 11, j:j + 11], y[i:i + 11, j:j + 11]
            mx, my = np.sum(w * px), np.sum(w * py)
            vx, vy = np.sum(w * (px - mx) ** 2), np.sum(w * (py - my) ** 2)
            cxy = np.sum(w * (px - mx) * (py - my))
            m[i, j] = ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx ** 2 + my ** 2 + C1) * (vx + vy + C2))
    np.testing.assert_allclose(q.ssim_map(x, y), m, rtol=1e-10)
    assert q.ssim(x, y) == pytest.approx(m.mean(), rel=1e-10)


def test_offset_leaves_only_the_luminance_term(q):
    """y = x + d: sy = sx and sxy = sx^2, so the contrast-structure factor is
    1 and the index is (2 mx (mx + d) + C1) / (mx^2 + (mx + d)^2 + C1)."""
    x, _ = _pair(20, 21, seed=5)
    d = 17.0
    mx = q._windowed(x, q.gaussian_window())
    C1 = (0.01 * 255) ** 2
    lum = (2 * mx * (mx + d) + C1) / (mx ** 2 + (mx + d) ** 2 + C1)
    np.testing.assert_allclose(q.ssim_map(x, x + d), lum, rtol=1e-9)


def test_psnr_closed_form(q):
    x, _ = _pair()
    assert q.psnr(x, x + 5.0) == pytest.approx(10 * np.log10(255.0 ** 2 / 25.0), rel=1e-13)
    assert q.psnr(x, x) == float("inf")
