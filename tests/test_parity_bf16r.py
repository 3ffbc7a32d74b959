"""GPU parity of the FE_BF16R form: FE_BF16 with the response r_i = theta_i
rho'(z_i) entering the adjoint bank rounded once to BF16 (no lo part).

The forward bank, the energies and the prox are those of FE_BF16 (the same
MMAs on the same window-row ring; checked equal bit for bit).  The gradient
differs from the FP64 oracle run with the
rounded bank by the BF16 form's own error (1e-3 of max|g|, test_parity_tc.py)
plus the rounding of r: round-to-nearest BF16 has relative error at most
2^-9, so per pixel

    |g - g_ref|(p) <= 2^-9 sum_i (|K_i|^T |r_i|)(p) + 1e-3 max|g_ref|,

with r_i and K_i those of the oracle (|K_i| the operator of |k_i|).  A step
u^{n+1} = prox(u^n - alpha g^n + beta (u^n - u^{n-1})) inherits alpha times
that bound per pixel: the prox of the separable convex data term is
non-expansive per pixel.
"""
import numpy as np
import pytest

from rounding import round_bf16

pytestmark = pytest.mark.gpu

BF16_GRAD_TOL = 1e-3     # the FE_BF16 form's gradient tolerance (of max|g_ref|)
R_ROUND = 2.0 ** -9      # unit roundoff of BF16


@pytest.fixture(scope="module")
def fe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_5344_gb300 import build
    build.build()
    from paper_1404_5344_gb300 import fe as fe_mod
    return fe_mod


def _problem(H, W, seed):
    from paper_1404_5344_gb300 import synth
    u = synth.textured_image(H, W, seed=seed)
    return u, synth.speckle(u, L=1.0, seed=seed + 1)


def _r_bound(orc, u, kq, th):
    """sum_i |K_i|^T |r_i| at u, r_i = theta_i rho'(K_i u) (FP64 oracle)."""
    acc = np.zeros(u.shape)
    for i in range(kq.shape[0]):
        z = orc.K(u, kq[i])
        r = th[i] * 2.0 * z / (1.0 + z * z)
        acc += orc.KT(np.abs(r), np.abs(kq[i]))
    return acc


@pytest.mark.parametrize("shape", [(64, 64), (131, 77), (58, 26), (200, 13), (256, 256)])
def test_bf16r_gradient_parity(fe, orc, bank48, shape):
    k, th = bank48
    kq = round_bf16(k)
    H, W = shape
    _, f = _problem(H, W, seed=H + 7 * W)
    with fe.Solver([f], k, th, prec="bf16r") as s:
        g, F = s.gradient(0, f)
    g_ref, F_ref = orc.gradF(f, kq, th)
    bound = R_ROUND * _r_bound(orc, f, kq.astype(np.float64), th) + BF16_GRAD_TOL * np.max(np.abs(g_ref))
    err = np.abs(g.astype(np.float64) - g_ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    # the rounding of r shows: the form is not the BF16 form
    with fe.Solver([f], k, th, prec="bf16") as s:
        g16, F16 = s.gradient(0, f)
    assert not np.array_equal(g, g16)
    assert F == F16  # the forward bank and F are those of FE_BF16


def test_bf16r_energies_equal_bf16(fe, bank48):
    k, th = bank48
    u, f = _problem(131, 77, seed=5)
    with fe.Solver([f], k, th, lam=5.0, prec="bf16r") as a, fe.Solver([f], k, th, lam=5.0, prec="bf16") as b:
        assert a.energy(0, u) == b.energy(0, u)


def test_bf16r_single_step_parity(fe, orc, bank48):
    """One step from the GPU's own state at the GPU's accepted L_n against
    the oracle's fixed-L step with the rounded bank: per pixel within alpha_n
    times the gradient bound at u^n, plus the FE_BF16 step tolerance."""
    k, th = bank48
    kq = round_bf16(k).astype(np.float64)
    _, f = _problem(131, 77, seed=11)
    prm = orc.params(lam=5.0, beta=0.8, L0=1e-3, eta=2.0, c2=1e-6, max_backtrack=30, max_iter=1)
    with fe.Solver([f], k, th, lam=5.0, beta=0.8, L0=1e-3, prec="bf16r") as s:
        for nsteps in (0, 3, 10):
            if nsteps:
                assert s.step(nsteps) == fe.FE_OK
            u, up, g, info = s.get_state(0)
            assert s.step(1) == fe.FE_OK
            u1 = s.get_u(0).astype(np.float64)
            info1 = s.info(0)
            L, alpha = info1["L"], info1["alpha"]
            ref = orc.ipiano_fixed(f, kq, th, prm, [L], u, up)
            g_ref, _ = orc.gradF(u, kq, th)
            gbound = R_ROUND * _r_bound(orc, u.astype(np.float64), kq, th) + BF16_GRAD_TOL * np.max(np.abs(g_ref))
            bound = alpha * gbound + 2e-5 * np.max(np.abs(ref["u"]))
            err = np.abs(u1 - ref["u"])
            assert np.all(err <= bound), float(np.max(err / bound))
            # F at an iterate that differs from the oracle's by the bound above
            assert info1["F"] == pytest.approx(ref["rec"][0, 2], rel=1e-4)


def test_bf16r_batch_and_loop_modes(fe, bank48):
    """An uneven batch in one context equals single-image contexts bit for
    bit; the CUDA-graph loop equals the host loop bit for bit."""
    k, th = bank48
    fs = [_problem(H, W, seed=H)[1] for (H, W) in ((64, 64), (97, 131), (30, 200))]
    with fe.Solver(fs, k, th, prec="bf16r") as s:
        assert s.step(5) == fe.FE_OK
        ub = [s.get_u(j) for j in range(3)]
    for j, f in enumerate(fs):
        with fe.Solver([f], k, th, prec="bf16r") as s:
            s.set_loop_mode(0)
            assert s.step(5) == fe.FE_OK
            assert np.array_equal(s.get_u(0), ub[j])
