"""GPU parity of the combined model (Eq. newmodel, Sec. III-A; iterate
w = log u, FP32 form) against the FP64 oracle, through the C ABI.

Tolerances (FP32 against FP64):
  * v = K^T r is the variant model's gradient at u, held there to
    GRAD_TOL = 1e-5 of max|v_ref|.  Here the bank sees u_gpu = expf(w), which
    differs from e^w by up to 2 ulp; to first order that moves z_i by at most
    2 eps Z_i, Z_i = |k_i| * u, and v by at most
    4 eps A(p), A = sum_i theta_i |k_i|^T (|rho''(z_i)| Z_i)  (|rho''| from the
    oracle's z).  The product grad_w F = u (.) v adds one rounding.  So at
    every pixel |g - g_ref| <= u(p) (GRAD_TOL max|v_ref| + 4 eps A(p))
    + 2 eps |g_ref(p)|, A computed with the oracle's K and K^T applied to
    |k_i|.  (A bound of 1e-5 of max|g_ref| does not follow: u spans 10..2500
    on speckled inputs, so the largest errors sit at bright pixels.)
  * energies: per-pixel FP32 terms (expf, logf) summed in compensated FP32 and
    FP64: 2e-6 relative (F) and 5e-6 (G, whose two terms partly cancel).
  * one step: the per-pixel Newton prox in FP32 stops at a step below 2^-22
    relative, so w^{n+1} agrees to ~1e-6 of |w|; STEP_TOL = 1e-5 of max|w|.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-5
EF_TOL = 2e-6
EG_TOL = 5e-6
STEP_TOL = 1e-5
NOISE_REL = 4e-6
L1, L2 = 160.0, 0.004  # the paper's lambda1, lambda2 for L = 1 (Sec. III-B)


@pytest.fixture(scope="module")
def fe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_5344_gb300 import build
    build.build()
    from paper_1404_5344_gb300 import fe as fe_mod
    return fe_mod


@pytest.fixture(scope="module")
def bank():
    from paper_1404_5344_gb300 import synth
    return synth.filter_bank(48, 7, seed=0, theta=0.1)


def _problem(H, W, seed=0, L=1.0):
    from paper_1404_5344_gb300 import synth
    u = synth.textured_image(H, W, seed=seed)
    return u, synth.speckle(u, L=L, seed=seed + 1)


def _relmax(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / np.max(np.abs(b)))


def _solver(fe, f, k, th, **kw):
    kw.setdefault("lam", L2)
    kw.setdefault("lam1", L1)
    return fe.Solver([f], k, th, model="combined", **kw)


def _oprm(orc, **kw):
    kw.setdefault("lam", L2)
    kw.setdefault("lam1", L1)
    return orc.params(model=orc.MODEL_COMBINED, **kw)


@pytest.mark.parametrize("tile", [64, 32, 32 | 0x100, 64 | 0x100])
@pytest.mark.parametrize("shape", [(64, 64), (131, 77), (8, 9), (200, 13)])
def test_gradient_parity_combined(fe, orc, bank, shape, tile):
    k, th = bank
    H, W = shape
    _, f = _problem(H, W, seed=H + W)
    w = np.log(f).astype(np.float32)
    with _solver(fe, f, k, th, tile=tile) as s:
        g, Fg = s.gradient(0, w)
    g_ref, F_ref = orc.gradFw(w, k, th)
    u = np.exp(w.astype(np.float64))
    v_ref = g_ref / u
    eps = 2.0 ** -24
    A = np.zeros_like(u)
    for i in range(k.shape[0]):
        ka = np.abs(k[i])
        z = orc.K(u, k[i])
        rho2 = np.abs(2.0 * (1.0 - z * z) / (1.0 + z * z) ** 2)
        A += th[i] * orc.KT(rho2 * orc.K(u, ka), ka)
    bound = u * (GRAD_TOL * np.max(np.abs(v_ref)) + 4 * eps * A) + 2 * eps * np.abs(g_ref)
    err = np.abs(g.astype(np.float64) - g_ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert Fg == pytest.approx(F_ref, rel=EF_TOL)


@pytest.mark.parametrize("lam1,lam2", [(L1, L2), (550.0, 0.02), (310.0, 0.0)])
def test_energy_parity_combined(fe, orc, bank, lam1, lam2):
    k, th = bank
    _, f = _problem(96, 70, seed=5)
    rng = np.random.default_rng(2)
    w = (np.log(f) + rng.normal(0, 0.3, f.shape)).astype(np.float32)
    with _solver(fe, f, k, th, lam=lam2, lam1=lam1) as s:
        E, F, G = s.energy(0, w)
        info = s.info(0)
    assert F == pytest.approx(orc.Fw(w, k, th), rel=EF_TOL)
    assert G == pytest.approx(orc.Gc(w, f, lam1, lam2), rel=EG_TOL)
    # the state starts at w^0 = log f, and the floor is the data term there
    lf = np.log(f.astype(np.float64))
    floor = np.sum(0.5 * lam1 * (2 * lf + 1) + 0.5 * lam2 * (f.astype(np.float64) ** 2 * (1 - 2 * lf)))
    assert info["G_floor"] == pytest.approx(floor, rel=1e-7)  # the GPU reads f^2 rounded to FP32
    assert info["G"] == pytest.approx(orc.Gc(np.log(f.astype(np.float32)), f, lam1, lam2), rel=EG_TOL)


def _check_decisions(orc, f, k, th, prm, w, wp, L_start, L_acc, eta=2.0):
    """Same rule as for the variant model: the GPU's rejections and its
    acceptance agree with the oracle's FP64 test up to FP32 noise."""
    K = int(round(np.log(L_acc / L_start) / np.log(eta)))
    assert abs(L_start * eta ** K - L_acc) <= 1e-12 * L_acc
    out = None
    for j in range(K + 1):
        r = orc.ipiano_fixed(f, k, th, prm, [L_start * eta ** j], w, wp)
        assert r["status"] == 0
        F1, margin, gd = r["rec"][0, 2], r["rec"][0, 5], r["rec"][0, 6]
        if j < K:
            if not np.isfinite(F1):
                continue  # an overflowing trial fails the test on both sides
            noise = NOISE_REL * (abs(F1) + abs(gd))
            assert margin <= noise, ("GPU rejected a step the oracle accepts", j, margin, noise)
        else:
            assert np.isfinite(F1), "GPU accepted a trial whose F overflows"
            noise = NOISE_REL * (abs(F1) + abs(gd))
            assert margin >= -noise, ("GPU accepted a step the oracle rejects", margin, noise)
            out = r
    return out


@pytest.mark.parametrize("lam1,lam2,L0", [(L1, L2, 1.0), (550.0, 0.02, 1e-2), (310.0, 0.0, 1e2),
                                         (310.0, 0.0, 1.0)])
def test_single_step_parity_combined(fe, orc, bank, lam1, lam2, L0):
    """After k GPU steps, one more GPU step vs the FP64 oracle started from the
    GPU's own state (w^n, w^{n-1}) and L; lam2 = 0 is Eq. original, whose
    first trials from L0 = 1 overflow e^w and are rejected."""
    k, th = bank
    H, W = 96, 130
    _, f = _problem(H, W, seed=11)
    prm = _oprm(orc, lam=lam2, lam1=lam1, beta=0.8, L0=L0, eta=2.0, c2=1e-6, max_iter=1)
    with _solver(fe, f, k, th, lam=lam2, lam1=lam1, beta=0.8, L0=L0, eta=2.0, c2=1e-6) as s:
        for nsteps in (0, 3, 10):
            if nsteps:
                assert s.step(nsteps) == fe.FE_OK
            w, wp, g, info = s.get_state(0)
            assert s.step(1) == fe.FE_OK
            w1, _, _, info1 = s.get_state(0)
            ref = _check_decisions(orc, f, k, th, prm, w, wp, info["L"], info1["L"])
            assert _relmax(w1, ref["u"]) <= STEP_TOL
            assert info1["F"] == pytest.approx(ref["rec"][0, 2], rel=EF_TOL)
            assert info1["G"] == pytest.approx(ref["rec"][0, 3], rel=EG_TOL)
            # fe_get_u returns u = e^w
            np.testing.assert_allclose(s.get_u(0), np.exp(w1.astype(np.float64)), rtol=1e-6)


def test_trajectory_combined_60_iterations(fe, orc, bank):
    """The GPU's accepted L_n replayed in the oracle: trajectories agree to
    1e-4 of max|w| after 60 iterations, energies to 1e-6."""
    k, th = bank
    _, f = _problem(64, 64, seed=0)
    prm = _oprm(orc, beta=0.8, L0=1.0, c2=1e-6, max_iter=1)
    Ls, Hs = [], []
    with _solver(fe, f, k, th, L0=1.0) as s:
        for n in range(60):
            assert s.step(1) == fe.FE_OK
            i = s.info(0)
            Ls.append(i["L"])
            Hs.append(i["H"])
        wg = s.get_state(0)[0]
    w0 = np.log(f.astype(np.float32)).astype(np.float64)
    ref = orc.ipiano_fixed(f, k, th, prm, Ls, w0)
    assert ref["status"] == 0
    assert _relmax(wg, ref["u"]) <= 1e-4
    np.testing.assert_allclose(Hs, ref["rec"][:, 4], rtol=1e-6)


def test_solve_to_tolerance_combined(fe, bank):
    k, th = bank
    _, f = _problem(80, 72, seed=3)
    with _solver(fe, f, k, th, lam=0.02, lam1=550.0) as s:
        st = s.solve(3000, 1e-6)
        i = s.info(0)
    assert st == fe.FE_OK and i["converged"] and i["n"] > 1
    assert i["rel_change"] < 1e-6


def test_combined_model_options(fe, bank):
    k, th = bank
    _, f = _problem(40, 40, seed=1)
    for bad in (dict(lam=0.0, lam1=0.0), dict(lam=-1.0), dict(lam1=float("nan")), dict(tile=48)):
        with pytest.raises(fe.FeError):
            _solver(fe, f, k, th, **bad)
    with pytest.raises(fe.FeError):
        fe.Solver([f], k, th, model=7)


# ---- tensor-core forms of the combined model --------------------------------
# The form's model is the bank rounded once to the operand type; the oracle
# runs with the same rounded bank.  The bound on K^T r at u is the variant
# forms' (tests/test_parity_tc.py: the hi + lo operand split of u and r);
# e^w adds the same first-order term as in the FP32 test above.
TC_GRAD_TOL = {"bf16": 1e-3, "tf32": 2e-5}
TC_STEP_TOL = {"bf16": 2e-5, "tf32": 1e-5}
TC_NOISE = {"bf16": 2e-5, "tf32": 4e-6}


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("shape", [(64, 64), (131, 77), (59, 27)])
def test_tc_gradient_parity_combined(fe, orc, bank, shape, prec):
    from rounding import ROUND
    k, th = bank
    kq = ROUND[prec](k)
    H, W = shape
    _, f = _problem(H, W, seed=H + 2 * W)
    w = np.log(f).astype(np.float32)
    with _solver(fe, f, k, th, prec=prec) as s:
        g, Fg = s.gradient(0, w)
    g_ref, F_ref = orc.gradFw(w, kq, th)
    u = np.exp(w.astype(np.float64))
    v_ref = g_ref / u
    eps = 2.0 ** -24
    A = np.zeros_like(u)
    for i in range(kq.shape[0]):
        ka = np.abs(kq[i]).astype(np.float64)
        z = orc.K(u, kq[i])
        A += th[i] * orc.KT(np.abs(2.0 * (1.0 - z * z) / (1.0 + z * z) ** 2) * orc.K(u, ka), ka)
    bound = u * (TC_GRAD_TOL[prec] * np.max(np.abs(v_ref)) + 4 * eps * A) + 2 * eps * np.abs(g_ref)
    err = np.abs(g.astype(np.float64) - g_ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert Fg == pytest.approx(F_ref, rel=10 * EF_TOL if prec == "bf16" else 2 * EF_TOL)


@pytest.mark.parametrize("shape", [(64, 64), (131, 77), (59, 27)])
def test_bf16r_gradient_parity_combined(fe, orc, bank, shape):
    """FE_BF16R on the combined model: grad_w F = e^w (.) K^T r with r rounded
    once to BF16, so the BF16 form's bound gains e^w 2^-9 sum_i |K_i|^T |r_i|
    per pixel (round-to-nearest BF16 of each response)."""
    from rounding import ROUND
    k, th = bank
    kq = ROUND["bf16"](k)
    H, W = shape
    _, f = _problem(H, W, seed=H + 2 * W)
    w = np.log(f).astype(np.float32)
    with _solver(fe, f, k, th, prec="bf16r") as s:
        g, Fg = s.gradient(0, w)
    g_ref, F_ref = orc.gradFw(w, kq, th)
    u = np.exp(w.astype(np.float64))
    v_ref = g_ref / u
    eps = 2.0 ** -24
    A, Rb = np.zeros_like(u), np.zeros_like(u)
    for i in range(kq.shape[0]):
        ka = np.abs(kq[i]).astype(np.float64)
        z = orc.K(u, kq[i])
        A += th[i] * orc.KT(np.abs(2.0 * (1.0 - z * z) / (1.0 + z * z) ** 2) * orc.K(u, ka), ka)
        Rb += orc.KT(np.abs(th[i] * 2.0 * z / (1.0 + z * z)), ka)
    bound = u * (TC_GRAD_TOL["bf16"] * np.max(np.abs(v_ref)) + 4 * eps * A + 2.0 ** -9 * Rb) + 2 * eps * np.abs(g_ref)
    err = np.abs(g.astype(np.float64) - g_ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert Fg == pytest.approx(F_ref, rel=10 * EF_TOL)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_single_step_parity_combined(fe, orc, bank, prec):
    from rounding import ROUND
    k, th = bank
    kq = ROUND[prec](k)
    _, f = _problem(96, 130, seed=11)
    prm = _oprm(orc, beta=0.8, L0=1.0, eta=2.0, c2=1e-6, max_iter=1)
    with _solver(fe, f, k, th, prec=prec, beta=0.8, L0=1.0, eta=2.0, c2=1e-6) as s:
        for nsteps in (0, 4):
            if nsteps:
                assert s.step(nsteps) == fe.FE_OK
            w, wp, _, info = s.get_state(0)
            assert s.step(1) == fe.FE_OK
            w1, _, _, info1 = s.get_state(0)
            K = int(round(np.log(info1["L"] / info["L"]) / np.log(2.0)))
            ref = None
            for j in range(K + 1):
                r = orc.ipiano_fixed(f, kq, th, prm, [info["L"] * 2.0 ** j], w, wp)
                F1, margin, gd = r["rec"][0, 2], r["rec"][0, 5], r["rec"][0, 6]
                if j < K:
                    if np.isfinite(F1):
                        assert margin <= TC_NOISE[prec] * (abs(F1) + abs(gd))
                else:
                    assert np.isfinite(F1) and margin >= -TC_NOISE[prec] * (abs(F1) + abs(gd))
                    ref = r
            assert _relmax(w1, ref["u"]) <= TC_STEP_TOL[prec]
            np.testing.assert_allclose(s.get_u(0), np.exp(w1.astype(np.float64)), rtol=1e-6)


@pytest.mark.parametrize("form", [("fp32", 64), ("fp32", 32), ("fp32", 32 | 0x100), ("fp32", 64 | 0x100), ("bf16", 0),
                                  ("tf32", 0)])
def test_gradient_parity_combined_distinct_weights(fe, orc, form):
    """A bank of 20 filters with distinct weights theta_i (five groups of
    four on the FP32 path, zero-padded GEMM columns on the tensor-core
    path): the gradient in w against the oracle, with the bounds above."""
    from rounding import ROUND
    from paper_1404_5344_gb300 import synth
    prec, tile = form
    k, _ = synth.filter_bank(20, 7, seed=4, theta=0.1)
    th = np.linspace(0.02, 0.3, 20).astype(np.float32)[::-1].copy()
    kq = k if prec == "fp32" else ROUND[prec](k)
    tol = GRAD_TOL if prec == "fp32" else TC_GRAD_TOL[prec]
    _, f = _problem(96, 80, seed=5)
    w = np.log(f).astype(np.float32)
    kw = {"tile": tile} if prec == "fp32" else {"prec": prec}
    with _solver(fe, f, k, th, **kw) as s:
        g, Fg = s.gradient(0, w)
    g_ref, F_ref = orc.gradFw(w, kq, th)
    u = np.exp(w.astype(np.float64))
    v_ref = g_ref / u
    eps = 2.0 ** -24
    A = np.zeros_like(u)
    for i in range(kq.shape[0]):
        ka = np.abs(kq[i]).astype(np.float64)
        z = orc.K(u, kq[i])
        A += th[i] * orc.KT(np.abs(2.0 * (1.0 - z * z) / (1.0 + z * z) ** 2) * orc.K(u, ka), ka)
    bound = u * (tol * np.max(np.abs(v_ref)) + 4 * eps * A) + 2 * eps * np.abs(g_ref)
    err = np.abs(g.astype(np.float64) - g_ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert Fg == pytest.approx(F_ref, rel=EF_TOL if prec != "bf16" else 10 * EF_TOL)


@pytest.mark.parametrize("L0", [1e-3, 1.0, 100.0])
def test_newton_prox_per_pixel(fe, orc, L0):
    """The Newton prox of the combined model on its own: with theta = 0 the
    first step is w^1 = prox_{alpha G}(w^0) pixel by pixel (every trial is
    accepted: F = 0), which must match the FP64 root to FP32 precision:
    |w - w_ref| <= 1e-6 (1 + |w_ref|) (the FP32 iteration stops at steps
    below 2^-22 (1 + |w|)).  A Newton safeguard that bisects away from a
    converged iterate ends anywhere in the bracket and fails this."""
    from paper_1404_5344_gb300 import synth
    k, _ = synth.filter_bank(8, 7, seed=2, theta=0.1)
    th = np.zeros(8, np.float32)
    _, f = _problem(48, 64, seed=31)
    rng = np.random.default_rng(5)
    u0 = (f * np.exp(rng.normal(0.0, 0.3, f.shape))).astype(np.float32)
    with _solver(fe, f, k, th, u0=u0, L0=L0, beta=0.8) as s:
        w0 = s.get_state(0)[0].copy()
        assert s.step(1) == fe.FE_OK
        w1 = s.get_state(0)[0]
        alpha = s.info(0)["alpha"]
    assert alpha == pytest.approx(2 * (1 - 0.8) / (L0 + 2e-6), rel=1e-12)
    ref = np.array([orc.proxc(float(a), float(b), alpha, L1, L2) for a, b in zip(w0.ravel(), f.ravel())])
    ref = ref.reshape(w1.shape)
    err = np.abs(w1.astype(np.float64) - ref) / (1.0 + np.abs(ref))
    assert float(np.max(err)) <= 1e-6, float(np.max(err))
