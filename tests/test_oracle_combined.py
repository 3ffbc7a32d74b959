"""Pins for the oracle's combined model (Eq. newmodel, Sec. III-A) in
w = log u:

    F(w) = E_FoE(e^w),   grad_w F = e^w (.) sum_i theta_i K_i^T rho'(K_i e^w)
    G(w) = sum_p lambda1/2 (2w + f^2 e^{-2w}) + lambda2/2 (e^{2w} - 2 f^2 w)

with the prox of tau G solved by Newton's method (the paper's choice), and
its special case lambda2 = 0 (Eq. original).  Each pin is independent of the
oracle's arithmetic: finite differences, dense matrices built with library
convolutions, Lambert-W closed forms of the prox (the direct solver the
paper mentions), bounded 1-D minimisation, and the identities of the
iteration (descent inequality, fixed points)."""
import numpy as np
import pytest
from scipy.optimize import brentq, minimize_scalar
from scipy.signal import convolve2d
from scipy.special import lambertw

COMB = 1  # oracle.MODEL_COMBINED


def _bank(nf=5, seed=3):
    rng = np.random.default_rng(seed)
    k = rng.standard_normal((nf, 7, 7))
    k -= k.mean(axis=(1, 2), keepdims=True)
    k /= np.sqrt((k ** 2).sum(axis=(1, 2), keepdims=True))
    return k, np.full(nf, 0.1)


def _problem(H=12, W=12, seed=0):
    rng = np.random.default_rng(seed)
    u = rng.uniform(10, 250, (H, W))
    f = np.maximum(u * rng.gamma(1.0, 1.0, (H, W)), 1e-3)
    return u, f


def _dense_ops(k, H, W):
    Ms = []
    for i in range(k.shape[0]):
        M = np.zeros((H * W, H * W))
        for j in range(H * W):
            e = np.zeros(H * W)
            e[j] = 1.0
            M[:, j] = convolve2d(np.pad(e.reshape(H, W), 3, mode="symmetric"), k[i], mode="valid").ravel()
        Ms.append(M)
    return Ms


def _g1(w, f, l1, l2):
    return l1 * (1 - f * f * np.exp(-2 * w)) + l2 * (np.exp(2 * w) - f * f)


def test_gradFw_finite_differences(orc):
    k, th = _bank(4, seed=1)
    u, _ = _problem(9, 11, seed=2)
    w = np.log(u)
    g, F0 = orc.gradFw(w, k, th)
    assert F0 == pytest.approx(orc.F(u, k, th), rel=1e-14)
    h = 1e-6
    rng = np.random.default_rng(0)
    for (y, x) in [(0, 0), (8, 10), (4, 5)] + [tuple(p) for p in rng.integers(0, 9, (5, 2))]:
        wp, wm = w.copy(), w.copy()
        wp[y, x] += h
        wm[y, x] -= h
        fd = (orc.Fw(wp, k, th) - orc.Fw(wm, k, th)) / (2 * h)
        assert g[y, x] == pytest.approx(fd, rel=2e-6, abs=1e-9 * np.abs(g).max())


def test_gradFw_dense_matrices(orc):
    """e^w (.) sum_i theta_i M_i^T rho'(M_i e^w) with M_i built from numpy's
    symmetric padding and scipy's convolution."""
    H = W = 8
    k, th = _bank(3, seed=4)
    u, _ = _problem(H, W, seed=5)
    w = np.log(u)
    Ms = _dense_ops(k, H, W)
    x = np.exp(w).ravel()
    ref = x * sum(th[i] * (M.T @ (2 * (M @ x) / (1 + (M @ x) ** 2))) for i, M in enumerate(Ms))
    g, _ = orc.gradFw(w, k, th)
    np.testing.assert_allclose(g.ravel(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_Gc_closed_form_and_minimum_at_log_f(orc):
    rng = np.random.default_rng(1)
    f = rng.uniform(5, 200, (6, 7))
    w = rng.uniform(1, 6, f.shape)
    l1, l2 = 160.0, 0.004
    ref = np.sum(0.5 * l1 * (2 * w + f ** 2 * np.exp(-2 * w)) + 0.5 * l2 * (np.exp(2 * w) - 2 * f ** 2 * w))
    assert orc.Gc(w, f, l1, l2) == pytest.approx(ref, rel=1e-14)
    lf = np.log(f)
    g0 = orc.Gc(lf, f, l1, l2)
    floor = np.sum(0.5 * l1 * (2 * lf + 1) + 0.5 * l2 * (f ** 2 - 2 * f ** 2 * lf))
    assert g0 == pytest.approx(floor, rel=1e-14)
    for d in (-0.3, -1e-3, 1e-3, 0.3):
        assert orc.Gc(lf + d, f, l1, l2) > g0


@pytest.mark.parametrize("what,f,tau", [(4.0, 100.0, 0.05), (6.5, 30.0, 0.2), (-1.0, 12.0, 1e-3),
                                        (4.6, 100.0, 0.5)])
def test_proxc_lambert_w(orc, what, f, tau):
    """lambda2 = 0: w - c = A e^{-2w}, c = what - tau l1, A = tau l1 f^2, so
    w = c + W0(2 A e^{-2c}) / 2.  lambda1 = 0: c - w = tau l2 e^{2w},
    c = what + tau l2 f^2, so w = c - W0(2 tau l2 e^{2c}) / 2."""
    l1, l2 = 160.0, 0.004
    c = what - tau * l1
    A = tau * l1 * f * f
    w_ref = c + 0.5 * lambertw(2 * A * np.exp(-2 * c)).real
    assert orc.proxc(what, f, tau, l1, 0.0) == pytest.approx(w_ref, rel=1e-13, abs=1e-13)
    c2 = what + tau * l2 * f * f
    w_ref2 = c2 - 0.5 * lambertw(2 * tau * l2 * np.exp(2 * c2)).real
    assert orc.proxc(what, f, tau, 0.0, l2) == pytest.approx(w_ref2, rel=1e-13, abs=1e-13)


@pytest.mark.parametrize("what,f,tau,l1,l2", [(4.0, 100.0, 0.05, 160.0, 0.004), (2.0, 150.0, 0.5, 550.0, 0.02),
                                              (7.0, 40.0, 0.01, 310.0, 0.008), (4.2, 60.0, 1.0, 0.0, 0.02)])
def test_proxc_minimises_the_prox_objective(orc, what, f, tau, l1, l2):
    w = orc.proxc(what, f, tau, l1, l2)
    # optimality: w - what + tau g'(w) = 0
    assert abs(w - what + tau * _g1(w, f, l1, l2)) <= 1e-10 * (1 + abs(what) + tau * (l1 + l2 * f * f))

    def obj(v):
        return 0.5 * (v - what) ** 2 + tau * (0.5 * l1 * (2 * v + f * f * np.exp(-2 * v))
                                              + 0.5 * l2 * (np.exp(2 * v) - 2 * f * f * v))
    lo, hi = min(what, np.log(f)) - 1, max(what, np.log(f)) + 1
    res = minimize_scalar(obj, bounds=(lo, hi), method="bounded", options={"xatol": 1e-11})
    assert w == pytest.approx(res.x, abs=1e-7)
    # root of phi by bracketing (scipy) agrees to rounding
    root = brentq(lambda v: v - what + tau * _g1(v, f, l1, l2), lo, hi, xtol=1e-15, rtol=1e-15)
    assert w == pytest.approx(root, rel=1e-13, abs=1e-13)


def test_proxc_fixed_point_monotone_and_limits(orc):
    f, l1, l2 = 80.0, 160.0, 0.004
    lf = np.log(f)
    assert orc.proxc(lf, f, 0.3, l1, l2) == pytest.approx(lf, abs=1e-14)
    ws = [orc.proxc(a, f, 0.3, l1, l2) for a in np.linspace(0, 9, 19)]
    assert np.all(np.diff(ws) > 0)
    assert orc.proxc(3.0, f, 1e-12, l1, l2) == pytest.approx(3.0, abs=1e-8)   # tau -> 0: identity
    assert orc.proxc(3.0, f, 1e6, l1, l2) == pytest.approx(lf, abs=1e-5)       # tau -> inf: argmin G


def test_dense_step_8x8_combined(orc):
    """One iPiano step of the combined model computed with dense matrices and
    a bracketing root finder equals the oracle's step."""
    H = W = 8
    k, th = _bank(4, seed=5)
    u, f = _problem(H, W, seed=2)
    w = np.log(u)
    rng = np.random.default_rng(9)
    wp = w + rng.normal(0, 0.02, w.shape)
    l1, l2, beta, c2, L = 160.0, 0.004, 0.8, 1e-6, 400.0
    prm = orc.params(lam=l2, lam1=l1, model=COMB, beta=beta, L0=L, c2=c2, max_backtrack=0, max_iter=1)
    Ms = _dense_ops(k, H, W)
    x = np.exp(w).ravel()
    g = x * sum(th[i] * (M.T @ (2 * (M @ x) / (1 + (M @ x) ** 2))) for i, M in enumerate(Ms))
    alpha = 2 * (1 - beta) / (L + 2 * c2)
    what = w.ravel() - alpha * g + beta * (w.ravel() - wp.ravel())
    ref = np.array([brentq(lambda v: v - a + alpha * _g1(v, fv, l1, l2), min(a, np.log(fv)) - 1,
                           max(a, np.log(fv)) + 1, xtol=1e-15, rtol=1e-15)
                    for a, fv in zip(what, f.ravel())])
    out = orc.ipiano_step(f, k, th, prm, w, wp, L)
    assert out["status"] == 0, "L large enough to be accepted without backtracking"
    np.testing.assert_allclose(out["u1"].ravel(), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("beta,l1,l2,L0", [(0.0, 160.0, 0.004, 1e-3), (0.5, 550.0, 0.02, 1e-3),
                                           (0.8, 310.0, 0.008, 1e-3), (0.8, 160.0, 0.0, 1e-3)])
def test_trajectory_inequalities_combined(orc, beta, l1, l2, L0):
    """The accepted-step inequality (G is convex in w, so the derivation of
    the variant model carries over); l2 = 0 is Eq. original, where nothing
    bounds w from above: its first trials from L0 = 1e-3 overflow e^w
    (F not finite) and must be rejected by the step rule, not end the solve."""
    k, th = _bank(6, seed=1)
    u, f = _problem(16, 14, seed=4)
    prm = orc.params(lam=l2, lam1=l1, model=COMB, beta=beta, L0=L0, c2=1e-6, max_iter=40)
    out = orc.ipiano(f, k, th, prm)
    assert out["status"] == 0 and out["n"] == 40
    rec = out["rec"]
    Hs = np.concatenate([[out["F0"] + out["G0"]], rec[:, 4]])
    assert out["G0"] == pytest.approx(orc.Gc(np.log(f), f, l1, l2), rel=1e-14), "start w^0 = log f"
    for n in range(len(rec)):
        L, a, F1, G1, H1, bt, gd, dd, dp = rec[n]
        Fn = out["F0"] if n == 0 else rec[n - 1, 2]
        assert F1 <= Fn + gd + 0.5 * L * dd
        assert Hs[n + 1] <= Hs[n] - (1 / a - L / 2) * dd + (beta / a) * dp + 1e-9 * abs(Hs[n])
    if beta == 0.0:
        assert np.all(np.diff(Hs) <= 1e-9 * np.abs(Hs[1:]))
    if l2 == 0.0:
        assert rec[0, 5] > 0, "the overflowing first trials were rejected"
    w = out["u"]
    assert orc.Fw(w, k, th) == pytest.approx(rec[-1, 2], rel=1e-12)
    assert orc.Gc(w, f, l1, l2) == pytest.approx(rec[-1, 3], rel=1e-12)


def test_constant_image_is_fixed_point_combined(orc):
    k, th = _bank(5, seed=2)
    f = np.full((10, 12), 77.0)
    prm = orc.params(lam=0.004, lam1=160.0, model=COMB, max_iter=5)
    out = orc.ipiano(f, k, th, prm)
    assert out["status"] == 0
    np.testing.assert_allclose(out["u"], np.log(77.0), rtol=0, atol=1e-12)


def test_theta_zero_converges_to_log_f(orc):
    k, _ = _bank(3, seed=2)
    _, f = _problem(8, 9, seed=3)
    prm = orc.params(lam=0.02, lam1=550.0, model=COMB, beta=0.5, L0=1e-2, max_iter=200)
    out = orc.ipiano(f, k, np.zeros(3), prm, u0=np.log(f) + 0.5)
    np.testing.assert_allclose(out["u"], np.log(f), atol=1e-9)


def test_tolerance_stop_uses_the_data_term_floor(orc):
    """The solve stops at the first n with |H^n - H^{n-1}| / |H^n - G*| < tol,
    G* = sum_p lambda1/2 (2 log f + 1) + lambda2/2 (f^2 - 2 f^2 log f), the
    minimum of the data term (at w = log f), computed here independently."""
    k, th = _bank(6, seed=1)
    _, f = _problem(16, 14, seed=4)
    l1, l2, tol = 160.0, 0.004, 1e-4
    prm = orc.params(lam=l2, lam1=l1, model=COMB, beta=0.8, L0=1.0, max_iter=500, tol=tol)
    out = orc.ipiano(f, k, th, prm)
    assert out["status"] == 0 and out["converged"] and 1 < out["n"] < 500
    lf = np.log(f)
    floor = np.sum(0.5 * l1 * (2 * lf + 1) + 0.5 * l2 * (f ** 2 - 2 * f ** 2 * lf))
    Hs = np.concatenate([[out["F0"] + out["G0"]], out["rec"][:, 4]])
    rel = np.abs(np.diff(Hs)) / np.abs(Hs[1:] - floor)
    assert rel[-1] < tol and np.all(rel[:-1] >= tol)


@pytest.mark.parametrize("l1,l2", [(160.0, 0.004), (310.0, 0.008), (550.0, 0.02)])
def test_proxc_newton_converges_in_few_steps(orc, l1, l2):
    """Sec. III-A reports that Newton's method solves the prox in fewer than
    10 iterations.  On speckle-like inputs (u in [10, 250], f = u n with
    n ~ Gamma(1, 1), what = log u + N(0, 0.3^2)) at the paper's weights for
    L = 1, 3, 8 and step sizes tau from 1e-4 to 1, the oracle's safeguarded
    Newton iteration (to a step of 1e-15 (1 + |w|)) takes fewer than 10
    steps on average and at most 20, and its root zeroes phi(w) = w - what +
    tau g'(w) to rounding."""
    rng = np.random.default_rng(3)
    for tau in (1e-4, 1e-2, 1.0):
        its = []
        for _ in range(300):
            u = rng.uniform(10.0, 250.0)
            f = u * rng.gamma(1.0, 1.0)
            what = np.log(u) + rng.normal(0.0, 0.3)
            w, n = orc.proxc_iters(what, f, tau, l1, l2)
            its.append(n)
            a, b = l1 * f * f * np.exp(-2.0 * w), l2 * np.exp(2.0 * w)
            ph = w - what + tau * (l1 - a + b - l2 * f * f)
            scale = abs(w) + abs(what) + tau * (l1 + a + b + l2 * f * f)
            assert abs(ph) <= 1e-12 * scale, (tau, what, f, w, ph)
        assert np.mean(its) < 10 and max(its) <= 20, (tau, np.mean(its), max(its))
