"""Pins for the oracle's energy pieces: rho, rho' (Sec. II-A, II-C), the FoE
energy F (Eq. FOEmodel), the data term G (Eq. dataterm2) and
grad F = sum_i theta_i K_i^T rho'(K_i u) (Sec. II-C)."""
import json
import os

import numpy as np
import pytest
from scipy.signal import convolve2d

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _small_bank(nf=5, seed=2):
    rng = np.random.default_rng(seed)
    k = rng.standard_normal((nf, 7, 7))
    k -= k.mean(axis=(1, 2), keepdims=True)
    k /= np.sqrt((k ** 2).sum(axis=(1, 2), keepdims=True))
    th = rng.uniform(0.05, 0.3, nf)
    return k, th


def _image(H, W, seed=4):
    rng = np.random.default_rng(seed)
    return rng.uniform(10, 250, (H, W))


def test_rho_golden(orc):
    g = json.load(open(os.path.join(GOLD, "rho_values.json")))
    for c in g["cases"]:
        assert orc.rho(c["x"]) == pytest.approx(c["rho"], abs=1e-15)
        assert orc.drho(c["x"]) == pytest.approx(c["drho"], abs=1e-15)


def test_drho_is_derivative_of_rho(orc):
    for x in np.linspace(-7, 7, 29):
        h = 1e-6
        fd = (orc.rho(x + h) - orc.rho(x - h)) / (2 * h)
        assert orc.drho(x) == pytest.approx(fd, rel=1e-8, abs=1e-9)


def test_rho_is_nonconvex(orc):
    # rho'' = 2(1 - x^2)/(1 + x^2)^2 < 0 for |x| > 1 (Sec. II-A: non-convex prior)
    x, h = 2.0, 1e-4
    second = (orc.rho(x + h) - 2 * orc.rho(x) + orc.rho(x - h)) / h ** 2
    assert second < 0


def test_F_against_library_convolution(orc):
    k, th = _small_bank()
    u = _image(12, 15)
    ref = 0.0
    for i in range(len(th)):
        z = convolve2d(np.pad(u, 3, mode="symmetric"), k[i], mode="valid")
        ref += th[i] * np.log1p(z * z).sum()
    assert orc.F(u, k, th) == pytest.approx(ref, rel=1e-13)


def test_G_closed_form(orc):
    u = np.array([[1.0, 2.0], [3.0, 0.5]])
    f = np.array([[1.0, 1.0], [2.0, 0.25]])
    lam = 3.0
    ref = 0.5 * lam * sum(a * a - 2 * b * b * np.log(a) for a, b in zip(u.ravel(), f.ravel()))
    assert orc.G(u, f, lam) == pytest.approx(ref, rel=1e-15)
    # minimiser of G alone is u = f: d/du (u^2 - 2 f^2 log u) = 2u - 2f^2/u
    assert orc.G(f, f, lam) < orc.G(f * 1.01, f, lam)
    assert orc.G(f, f, lam) < orc.G(f * 0.99, f, lam)


def test_gradF_finite_differences(orc):
    k, th = _small_bank(4, seed=9)
    u = _image(9, 11, seed=5) * 0.05  # responses of order 1 so rho is curved
    g, Fv = orc.gradF(u, k, th)
    assert Fv == pytest.approx(orc.F(u, k, th), rel=1e-14)
    rng = np.random.default_rng(0)
    for _ in range(12):
        y, x = rng.integers(0, 9), rng.integers(0, 11)
        h = 1e-5
        up, um = u.copy(), u.copy()
        up[y, x] += h
        um[y, x] -= h
        fd = (orc.F(up, k, th) - orc.F(um, k, th)) / (2 * h)
        assert g[y, x] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_grad_H_directional_finite_difference(orc):
    k, th = _small_bank(6, seed=1)
    u = _image(10, 10, seed=8) * 0.1
    f = u * np.random.default_rng(3).uniform(0.5, 1.5, u.shape)
    lam = 2.0
    g, _ = orc.gradF(u, k, th)
    gH = g + lam * (u - f * f / u)
    d = np.random.default_rng(4).standard_normal(u.shape)
    h = 1e-4  # |G| ~ 1e5 here: a smaller step is dominated by round-off

    def Hf(v):
        return orc.F(v, k, th) + orc.G(v, f, lam)
    fd = (Hf(u + h * d) - Hf(u - h * d)) / (2 * h)
    assert float(np.sum(gH * d)) == pytest.approx(fd, rel=1e-7)


def test_gradF_dense_brute_force(orc):
    """grad F from dense library matrices: sum_i theta_i M_i^T rho'(M_i u)."""
    k, th = _small_bank(3, seed=6)
    H, W = 8, 8
    u = _image(H, W, seed=2) * 0.07
    ref = np.zeros(H * W)
    for i in range(len(th)):
        M = np.zeros((H * W, H * W))
        for j in range(H * W):
            e = np.zeros(H * W)
            e[j] = 1.0
            M[:, j] = convolve2d(np.pad(e.reshape(H, W), 3, mode="symmetric"), k[i],
                                 mode="valid").ravel()
        z = M @ u.ravel()
        ref += th[i] * (M.T @ (2 * z / (1 + z * z)))
    g, _ = orc.gradF(u, k, th)
    np.testing.assert_allclose(g.ravel(), ref, rtol=0, atol=1e-12)


def test_gradF_at_matches_full(orc):
    k, th = _small_bank(5, seed=3)
    u = _image(16, 13, seed=6) * 0.1
    g, _ = orc.gradF(u, k, th)
    pts = [(0, 0), (0, 12), (15, 0), (15, 12), (1, 2), (2, 1), (7, 6), (14, 11), (13, 3)]
    np.testing.assert_allclose(orc.gradF_at(u, k, th, pts), [g[p] for p in pts],
                               rtol=1e-12, atol=1e-12)


def test_special_cases(orc):
    # constant image + zero-mean filters: K_i u = 0 so F = 0 and grad F = 0
    k, th = _small_bank(4, seed=7)
    u = np.full((9, 10), 42.0)
    g, Fv = orc.gradF(u, k, th)
    assert abs(Fv) < 1e-20 and np.max(np.abs(g)) < 1e-12
    # theta = 0 switches the prior off
    u = _image(9, 10)
    g, Fv = orc.gradF(u, k, np.zeros(4))
    assert Fv == 0.0 and np.max(np.abs(g)) == 0.0
    # F is linear in theta
    assert orc.F(u, k, 2 * th) == pytest.approx(2 * orc.F(u, k, th), rel=1e-14)
