"""Pins for the oracle's iPiano iteration (Sec. II-C update rule) with the
Lipschitz backtracking step rule of the cited iPiano paper (a reading: the
paper names alpha and beta only)."""
import json
import os

import numpy as np
import pytest
from scipy.signal import convolve2d

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _bank(nf=6, seed=3, exact_zero_mean=True):
    rng = np.random.default_rng(seed)
    k = rng.standard_normal((nf, 7, 7))
    k -= k.mean(axis=(1, 2), keepdims=True)
    k /= np.sqrt((k ** 2).sum(axis=(1, 2), keepdims=True))
    return k, np.full(nf, 0.1)


def _problem(H=12, W=12, seed=0):
    rng = np.random.default_rng(seed)
    u = rng.uniform(10, 250, (H, W))
    f = u * rng.gamma(1.0, 1.0, (H, W))
    return u, np.maximum(f, 1e-3)


def test_golden_one_pixel_step(orc):
    g = json.load(open(os.path.join(GOLD, "ipiano_step_1px.json")))
    prm = orc.params(lam=g["lambda"], beta=g["beta"], L0=g["L"], c2=g["c2"], max_iter=1)
    f = np.array([[g["f"]]])
    out = orc.ipiano_step(f, np.zeros((1, 7, 7)), np.zeros(1), prm,
                          np.array([[g["u"]]]), np.array([[g["u_prev"]]]), g["L"])
    assert out["status"] == 0
    assert out["rec"][1] == pytest.approx(g["alpha"], rel=1e-15)
    assert out["u1"][0, 0] == pytest.approx(g["u_next"], rel=1e-14)


def _dense_ops(k, H, W):
    Ms = []
    for i in range(k.shape[0]):
        M = np.zeros((H * W, H * W))
        for j in range(H * W):
            e = np.zeros(H * W)
            e[j] = 1.0
            M[:, j] = convolve2d(np.pad(e.reshape(H, W), 3, mode="symmetric"), k[i],
                                 mode="valid").ravel()
        Ms.append(M)
    return Ms


def test_dense_step_8x8(orc):
    """One iPiano step computed with dense matrices in NumPy (a separate code
    path: library convolution, matrix products, quadratic formula) equals the
    oracle's step to 1e-12."""
    H = W = 8
    k, th = _bank(4, seed=5)
    u, f = _problem(H, W, seed=2)
    rng = np.random.default_rng(9)
    up = u + rng.normal(0, 2.0, u.shape)
    lam, beta, c2, L = 5.0, 0.8, 1e-6, 40.0
    prm = orc.params(lam=lam, beta=beta, L0=L, c2=c2, max_backtrack=0, max_iter=1)
    Ms = _dense_ops(k, H, W)
    x = u.ravel()
    g = sum(th[i] * (M.T @ (2 * (M @ x) / (1 + (M @ x) ** 2))) for i, M in enumerate(Ms))
    alpha = 2 * (1 - beta) / (L + 2 * c2)
    uhat = x - alpha * g + beta * (x - up.ravel())
    tl = alpha * lam
    ff = f.ravel() ** 2
    ref = (uhat + np.sqrt(uhat ** 2 + 4 * (1 + tl) * tl * ff)) / (2 * (1 + tl))
    out = orc.ipiano_step(f, k, th, prm, u, up, L)
    assert out["status"] == 0, "L large enough to be accepted without backtracking"
    np.testing.assert_allclose(out["u1"].ravel(), ref, rtol=1e-12, atol=1e-12)




@pytest.mark.parametrize("beta", [0.0, 0.5, 0.8])
def test_trajectory_inequalities(orc, beta):
    k, th = _bank(6, seed=1)
    u, f = _problem(16, 14, seed=4)
    lam = 5.0
    prm = orc.params(lam=lam, beta=beta, L0=1e-3, c2=1e-6, max_iter=40)
    out = orc.ipiano(f, k, th, prm)
    assert out["status"] == 0 and out["n"] == 40
    rec = out["rec"]
    H0 = out["F0"] + out["G0"]
    Hs = np.concatenate([[H0], rec[:, 4]])
    Ls = rec[:, 0]
    assert np.all(np.diff(Ls) >= 0), "L is never decreased"
    for n in range(len(rec)):
        L, a, F1, G1, H1, bt, gd, dd, dp = rec[n]
        assert a == pytest.approx(2 * (1 - beta) / (L + 2e-6), rel=1e-15)
        Fn = out["F0"] if n == 0 else rec[n - 1, 2]
        # the accepted trial passed the backtracking test
        assert F1 <= Fn + gd + 0.5 * L * dd
        tol = 1e-9 * abs(Hs[n])
        assert Hs[n + 1] <= Hs[n] - (1 / a - L / 2) * dd + (beta / a) * dp + tol
    if beta == 0.0:
        assert np.all(np.diff(Hs) <= 1e-9 * np.abs(Hs[1:])), "beta = 0: H is non-increasing"


def test_backtracking_triggers_and_is_bounded(orc):
    # intensities of order 1 put the responses in the convex part of rho, so a
    # tiny L0 fails the descent test until L has grown by enough factors of eta
    k, th = _bank(6, seed=1)
    u, f = _problem(16, 14, seed=4)
    f = f * 0.01
    prm = orc.params(lam=0.01, beta=0.5, L0=1e-4, eta=2.0, max_iter=10)
    out = orc.ipiano(f, k, th, prm)
    assert out["status"] == 0
    bt = out["rec"][:, 5]
    assert bt[0] > 0
    L0 = 1e-4
    assert out["rec"][0, 0] == pytest.approx(L0 * 2.0 ** bt[0], rel=1e-15)
    # the cap is honoured: with max_backtrack = 2 the same start fails
    prm2 = orc.params(lam=0.01, beta=0.5, L0=1e-4, eta=2.0, max_iter=10, max_backtrack=2)
    out2 = orc.ipiano(f, k, th, prm2)
    assert out2["status"] == 5 and out2["n"] == 0


def test_constant_image_is_fixed_point(orc):
    k, th = _bank(5, seed=2)
    c = 77.0
    f = np.full((10, 11), c)
    out = orc.ipiano(f, k, th, orc.params(lam=5.0, max_iter=5))
    assert out["status"] == 0
    np.testing.assert_allclose(out["u"], c, rtol=1e-12)


def test_theta_zero_converges_to_f(orc):
    k, _ = _bank(3, seed=2)
    u, f = _problem(9, 9, seed=5)
    out = orc.ipiano(f, k, np.zeros(3), orc.params(lam=5.0, beta=0.5, L0=1.0, max_iter=200),
                     u0=u)
    np.testing.assert_allclose(out["u"], f, rtol=1e-8)


def test_large_lambda_stays_at_f(orc):
    k, th = _bank(6, seed=4)
    _, f = _problem(10, 10, seed=6)
    out = orc.ipiano(f, k, th, orc.params(lam=1e8, max_iter=5))
    np.testing.assert_allclose(out["u"], f, rtol=1e-6)


def test_step_matches_solve(orc):
    """orc_ipiano_step from (u^n, u^{n-1}, L_{n-1}) reproduces iteration n+1
    of the full solve."""
    k, th = _bank(5, seed=8)
    _, f = _problem(11, 13, seed=7)
    prm = orc.params(lam=5.0, beta=0.8, L0=0.5, max_iter=6)
    a = orc.ipiano(f, k, th, prm)
    prm5 = orc.params(lam=5.0, beta=0.8, L0=0.5, max_iter=5)
    b = orc.ipiano(f, k, th, prm5)
    s = orc.ipiano_step(f, k, th, prm, b["u"], b["u_prev"], b["L"])
    np.testing.assert_allclose(s["u1"], a["u"], rtol=1e-13)
    np.testing.assert_allclose(s["rec"], a["rec"][5], rtol=1e-11)


def test_tolerance_stop(orc):
    """Stops at the first accepted step whose energy change, relative to the
    energy above the data-term floor G(f) = min_u G(u), is below tol."""
    k, th = _bank(6, seed=1)
    _, f = _problem(12, 12, seed=3)
    lam = 0.1  # a data weight at which the prior moves u away from f (lambda = 5 stops in 1-2 steps)
    out = orc.ipiano(f, k, th, orc.params(lam=lam, L0=1e-2, max_iter=3000, tol=1e-6))
    assert out["converged"] and 2 < out["n"] < 3000
    H = np.concatenate([[out["F0"] + out["G0"]], out["rec"][:, 4]])
    floor = orc.G(f, f, lam)
    assert np.all(H - floor >= 0)  # F >= 0 and G(u) >= G(f)
    rel = np.abs(np.diff(H)) / np.abs(H[1:] - floor)
    assert rel[-1] < 1e-6 and np.all(rel[:-1] >= 1e-6)


def test_fixed_sequence_matches_backtracking_run(orc):
    """Replaying the accepted L_n of a backtracking run with the prescribed-L
    iteration reproduces the run, and every replayed margin is >= 0."""
    k, th = _bank(6, seed=2)
    _, f = _problem(14, 15, seed=8)
    prm = orc.params(lam=0.05, beta=0.7, L0=1e-3, max_iter=25)
    a = orc.ipiano(f, k, th, prm)
    assert a["status"] == 0 and a["rec"][:, 5].sum() > 0
    b = orc.ipiano_fixed(f, k, th, prm, a["rec"][:, 0], f)
    np.testing.assert_allclose(b["u"], a["u"], rtol=1e-13)
    np.testing.assert_allclose(b["rec"][:, 4], a["rec"][:, 4], rtol=1e-13)
    assert np.all(b["rec"][:, 5] >= 0)
    # a rejected candidate (L / eta at a backtracked iteration) has margin < 0
    n = int(np.argmax(a["rec"][:, 5] > 0))
    start = orc.ipiano_fixed(f, k, th, prm, a["rec"][:n, 0], f) if n else dict(u=f, u_prev=f)
    c = orc.ipiano_fixed(f, k, th, prm, [a["rec"][n, 0] / 2.0], start["u"], start["u_prev"])
    assert c["rec"][0, 5] < 0
