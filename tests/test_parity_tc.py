"""GPU parity of the tensor-core forms (FE_BF16, FE_TF32; tcgen05 implicit
GEMMs) against the FP64 oracle run with the same rounded filter bank.

The form's model is the filter bank rounded once to the operand type (BF16
round-to-nearest-even / TF32 round-to-nearest); the data operands u and r
are carried as hi + lo pairs of that type, i.e. to about 2^-17 (BF16) and
2^-22 (TF32) relative.  The oracle, given the same rounded bank, is therefore
the exact reference of the implementation, and the tolerances below follow
from the data splitting:
  * z = k * u: |dz| <~ 2^-17 sum|k||u| (BF16), 2^-22 (TF32); grad F errs by
    ~ that relative to its scale, with a margin of 10: GRAD_TOL.
  * energies: per-pixel FP32 terms of such z, summed in FP64: E_TOL.
The error of the form against the unrounded (FP32) bank is measured and
reported separately (the precision study), not asserted here.
"""
import numpy as np
import pytest

from rounding import ROUND

pytestmark = pytest.mark.gpu

GRAD_TOL = {"bf16": 1e-3, "tf32": 2e-5}
E_TOL = {"bf16": 2e-5, "tf32": 4e-6}
STEP_TOL = {"bf16": 2e-5, "tf32": 1e-5}
NOISE_REL = {"bf16": 2e-5, "tf32": 4e-6}


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


def _problem(H, W, seed=0, L=1.0, kind="textured"):
    from paper_1404_5344_gb300 import synth
    u = synth.textured_image(H, W, seed=seed) if kind == "textured" else synth.piecewise_image(H, W, seed=seed)
    return u, synth.speckle(u, L=L, seed=seed + 1)


def _relmax(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / np.max(np.abs(b)))


SIZES = [(64, 64), (8, 8), (131, 77), (200, 13), (13, 200), (58, 26), (59, 27), (117, 53), (256, 256)]


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("shape", SIZES)
def test_tc_gradient_parity(fe, orc, bank, prec, shape):
    k, th = bank
    kq = ROUND[prec](k)
    H, W = shape
    _, f = _problem(H, W, seed=H * 3 + W)
    with fe.Solver([f], k, th, prec=prec) as s:
        g, Fg = s.gradient(0, f)
    g_ref, F_ref = orc.gradF(f, kq, th)
    err = _relmax(g, g_ref)
    assert err <= GRAD_TOL[prec], err
    assert Fg == pytest.approx(F_ref, rel=E_TOL[prec])


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("shape", [(64, 64), (131, 77)])
def test_tc_energy_parity(fe, orc, bank, prec, shape):
    k, th = bank
    kq = ROUND[prec](k)
    H, W = shape
    u, f = _problem(H, W, seed=3)
    with fe.Solver([f], k, th, lam=5.0, prec=prec) as s:
        E, F, G = s.energy(0, u)
    assert F == pytest.approx(orc.F(u, kq, th), rel=E_TOL[prec])
    assert G == pytest.approx(orc.G(u, f, 5.0), rel=2e-6)


def _check_decisions(orc, f, k, th, prm, u, up, L_start, L_acc, noise_rel, eta=2.0):
    K = int(round(np.log(L_acc / L_start) / np.log(eta)))
    assert abs(L_start * eta ** K - L_acc) <= 1e-12 * L_acc
    for j in range(K + 1):
        r = orc.ipiano_fixed(f, k, th, prm, [L_start * eta ** j], u, up)
        F1, margin, gd = r["rec"][0, 2], r["rec"][0, 5], r["rec"][0, 6]
        noise = noise_rel * (abs(F1) + abs(gd))
        if j < K:
            assert margin <= noise, ("rejected a step the oracle accepts", j, margin, noise)
        else:
            assert margin >= -noise, ("accepted a step the oracle rejects", margin, noise)
    return r


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_single_step_parity(fe, orc, bank, prec):
    k, th = bank
    kq = ROUND[prec](k)
    H, W = 131, 77
    _, f = _problem(H, W, seed=11)
    prm = orc.params(lam=5.0, beta=0.8, L0=1e-3, eta=2.0, c2=1e-6, max_backtrack=30, max_iter=1)
    with fe.Solver([f], k, th, lam=5.0, beta=0.8, L0=1e-3, prec=prec) as s:
        for nsteps in (0, 3, 10):
            if nsteps:
                assert s.step(nsteps) == fe.FE_OK
            u, up, g, info = s.get_state(0)
            assert s.step(1) == fe.FE_OK
            u1 = s.get_u(0)
            info1 = s.info(0)
            ref = _check_decisions(orc, f, kq, th, prm, u, up, info["L"], info1["L"], NOISE_REL[prec])
            assert _relmax(u1, ref["u"]) <= STEP_TOL[prec]
            assert info1["F"] == pytest.approx(ref["rec"][0, 2], rel=E_TOL[prec])


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_trajectory_64x64_100_iterations(fe, orc, bank, prec):
    k, th = bank
    kq = ROUND[prec](k)
    _, f = _problem(64, 64, seed=0, kind="piecewise")
    prm = orc.params(lam=5.0, beta=0.8, L0=1.0, eta=2.0, c2=1e-6, max_iter=1)
    Ls, Hs = [], []
    with fe.Solver([f], k, th, lam=5.0, L0=1.0, prec=prec) as s:
        for n in range(100):
            assert s.step(1) == fe.FE_OK
            i = s.info(0)
            Ls.append(i["L"])
            Hs.append(i["H"])
        ug = s.get_u(0)
    ref = orc.ipiano_fixed(f, kq, th, prm, Ls, f)
    assert ref["status"] == 0
    assert _relmax(ug, ref["u"]) <= 1e-4
    np.testing.assert_allclose(Hs, ref["rec"][:, 4], rtol=1e-6)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_batch_and_loop_modes(fe, bank, prec):
    """Uneven batch in one context equals single-image contexts bit for bit;
    the CUDA-graph loop and the persistent launch equal the host loop bit for
    bit."""
    k, th = bank
    shapes = [(64, 64), (131, 77), (9, 300), (200, 150)]
    fs = [_problem(H, W, seed=30 + i)[1] for i, (H, W) in enumerate(shapes)]
    outs = {}
    for mode in (0, 1, 2):
        with fe.Solver(fs, k, th, L0=1e-2, prec=prec, loop_mode=mode) as s:
            assert s.step(6) == fe.FE_OK
            outs[mode] = [s.get_u(i) for i in range(len(fs))]
    for i in range(len(fs)):
        assert np.array_equal(outs[0][i], outs[1][i])
        assert np.array_equal(outs[0][i], outs[2][i])
        with fe.Solver([fs[i]], k, th, L0=1e-2, prec=prec) as s1:
            s1.step(6)
            assert np.array_equal(s1.get_u(0), outs[1][i])


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_gradient_parity_4096_sampled(fe, orc, bank, prec):
    """The 4096 x 4096 precision-form workload: grad F at sampled pixels
    (corners, borders, tile seams, random) against the oracle's per-pixel
    gradient with the rounded bank."""
    k, th = bank
    kq = ROUND[prec](k)
    H = W = 4096
    _, f = _problem(H, W, seed=1)
    with fe.Solver([f], k, th, prec=prec) as s:
        g, _ = s.gradient(0, f)
    rng = np.random.default_rng(0)
    pts = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (1, 2), (2, W - 3), (H - 3, 1),
           (57, 25), (58, 26), (H - 59, W - 27), (H - 58, W - 26), (H // 2, W // 2)]
    pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, H, 24), rng.integers(0, W, 24))]
    ref = orc.gradF_at(f, kq, th, pts)
    got = np.array([g[p] for p in pts], np.float64)
    assert np.max(np.abs(got - ref)) <= GRAD_TOL[prec] * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_single_tile_shape(fe, bank, prec):
    """The tensor-core forms have one tile shape: tile = 0 gives it, any
    other value is rejected before device work."""
    k, th = bank
    _, f = _problem(70, 90, seed=3)
    with fe.Solver([f], k, th, prec=prec) as s:
        assert s.tile == (58, 26)
    for bad in (32, 64):
        with pytest.raises(fe.FeError):
            fe.Solver([f], k, th, prec=prec, tile=bad)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("nf", [1, 9, 40, 48])
def test_tc_filter_counts_and_distinct_weights(fe, orc, prec, nf):
    """Banks of 1..48 filters with distinct weights theta_i (zero-padded to
    the GEMMs' 48 columns): gradient and energy against the oracle run with
    the same rounded bank."""
    from paper_1404_5344_gb300 import synth
    k, _ = synth.filter_bank(nf, 7, seed=nf, theta=0.1)
    th = np.linspace(0.02, 0.3, nf).astype(np.float32)[::-1].copy()
    kq = ROUND[prec](k)
    _, f = _problem(96, 80, seed=nf)
    with fe.Solver([f], k, th, prec=prec) as s:
        g, Fg = s.gradient(0, f)
    g_ref, F_ref = orc.gradF(f, kq, th)
    # as for the FP32 form (tests/test_parity_fp32.py, _grad_bound), with the
    # data operand u carried to 2^-17 (BF16 hi + lo) or 2^-22 (TF32 hi + lo)
    u = f.astype(np.float64)
    A = np.zeros_like(u)
    for i in range(nf):
        ka = np.abs(kq[i]).astype(np.float64)
        z = orc.K(u, kq[i])
        A += th[i] * orc.KT(np.abs(2.0 * (1.0 - z * z) / (1.0 + z * z) ** 2) * orc.K(u, ka), ka)
    eps_z = {"bf16": 2.0 ** -17, "tf32": 2.0 ** -22}[prec]
    bound = GRAD_TOL[prec] * np.max(np.abs(g_ref)) + 8 * eps_z * A + 2.0 ** -23 * np.abs(g_ref)
    err = np.abs(g.astype(np.float64) - g_ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert Fg == pytest.approx(F_ref, rel=E_TOL[prec])


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_more_than_48_filters_unsupported(fe, prec):
    from paper_1404_5344_gb300 import synth
    k, th = synth.filter_bank(64, 7, seed=1, theta=0.1)
    _, f = _problem(32, 32, seed=1)
    with pytest.raises(fe.FeError):
        fe.Solver([f], k, th, prec=prec)
