"""Pins for the closed-form proximal map of tau*G (Sec. II-C, model with the
I-divergence data term, Eq. dataterm2)."""
import json
import os

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_roots(orc):
    g = json.load(open(os.path.join(GOLD, "prox_cases.json")))
    for c in g["cases"]:
        got = orc.prox(c["uhat"], c["f"], c["tau"], c["lambda"])
        assert got == pytest.approx(c["u"], rel=c.get("rel_tol", 1e-14))


def _objective(u, uhat, f, tau, lam):
    return 0.5 * (u - uhat) ** 2 + tau * 0.5 * lam * (u * u - 2 * f * f * np.log(u))


def test_optimality_and_brute_force(orc):
    rng = np.random.default_rng(0)
    for _ in range(200):
        uhat = rng.uniform(-300, 300)
        f = rng.uniform(0.1, 800)
        tau = 10 ** rng.uniform(-4, 1)
        lam = 10 ** rng.uniform(-2, 2)
        u = orc.prox(uhat, f, tau, lam)
        assert u > 0
        tl = tau * lam
        # root of the first-order condition (1+tl) u^2 - uhat u - tl f^2 = 0
        scale = (1 + tl) * u * u + abs(uhat * u) + tl * f * f
        assert abs((1 + tl) * u * u - uhat * u - tl * f * f) <= 1e-13 * scale
        # brute force: bounded scalar minimisation of the prox objective
        lo, hi = u * 0.5, u * 2.0 + 1e-12
        res = minimize_scalar(_objective, bounds=(lo, hi), args=(uhat, f, tau, lam),
                              method="bounded", options={"xatol": 1e-12 * u})
        assert res.x == pytest.approx(u, rel=1e-3)
        fu = _objective(u, uhat, f, tau, lam)
        assert fu <= res.fun + 1e-12 * abs(res.fun)
        # dense grid of neighbours: none is lower (beyond rounding)
        for s in np.linspace(0.9, 1.1, 41):
            assert fu <= _objective(u * s, uhat, f, tau, lam) + 1e-12 * abs(fu)


def test_literal_and_stable_forms_agree(orc):
    rng = np.random.default_rng(1)
    for _ in range(200):
        uhat = rng.uniform(0, 300)
        f, tau, lam = rng.uniform(1, 500), rng.uniform(0.01, 2), rng.uniform(0.1, 10)
        assert orc.prox(uhat, f, tau, lam) == orc.prox(uhat, f, tau, lam, literal=True)
    for _ in range(200):
        uhat = rng.uniform(-50, 0)
        f, tau, lam = rng.uniform(10, 500), rng.uniform(0.01, 2), rng.uniform(0.1, 10)
        assert orc.prox(uhat, f, tau, lam) == pytest.approx(
            orc.prox(uhat, f, tau, lam, literal=True), rel=1e-12)


def test_limits(orc):
    # tau*lambda -> 0: the prox is the identity on positive inputs
    assert orc.prox(7.0, 3.0, 1e-12, 1.0) == pytest.approx(7.0, rel=1e-10)
    # tau*lambda -> infinity: the prox returns the minimiser of G, u = f
    assert orc.prox(7.0, 3.0, 1e9, 1.0) == pytest.approx(3.0, rel=1e-8)
    # fixed point at uhat = f: (1+tl) f^2 - f^2 - tl f^2 = 0
    for f in (0.5, 10.0, 200.0):
        assert orc.prox(f, f, 0.3, 5.0) == pytest.approx(f, rel=1e-14)
