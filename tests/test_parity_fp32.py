"""GPU parity of the FP32 path (libfe, called through the C ABI) against the
FP64 oracle, element by element on seeded inputs.

Tolerances (FP32 arithmetic against FP64, derived from the operations):
  * z_i = k_i * u sums 49 products of size up to |k| max|u|; FP32 rounding
    gives |dz| <~ 49 * 2^-24 * sum|k||u| ~ 1e-6 relative to sum|k||u|, and
    rho' has slope <= 2, so grad F errs by ~1e-6 relative to its scale
    sum_i theta_i |k_i|_1 max|rho'|; GRAD_TOL = 1e-5 of max|g_ref| leaves 10x.
  * energies: per-pixel FP32 terms summed in FP64; relative 2e-6.
  * one iPiano step: max|u_gpu - u_ref| / max|u_ref| <= 1e-5 (the required
    per-step bound), oracle started from the GPU's own state and L.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-5
E_TOL = 2e-6
STEP_TOL = 1e-5


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


def _problem(H, W, seed=0, L=1.0, kind="piecewise"):
    from paper_1404_5344_gb300 import synth
    if kind == "piecewise":
        u = synth.piecewise_image(H, W, seed=seed)
    else:
        u = synth.textured_image(H, W, seed=seed)
    f = synth.speckle(u, L=L, seed=seed + 1)
    return u, f


def _relmax(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / np.max(np.abs(b)))


SIZES = [(64, 64), (8, 8), (131, 77), (200, 13), (13, 200), (67, 129), (128, 128)]


# the FP32 kernel's tile shapes: 64 x 64, 32 x 32, and 32 x 32 split over a
# 4-CTA cluster (FE_TILE_CLUSTER4 = 0x100), and 64 x 64 split likewise
TILES = [64, 32, 32 | 0x100, 64 | 0x100]


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("shape", SIZES)
def test_gradient_parity(fe, orc, bank, shape, tile):
    k, th = bank
    H, W = shape
    _, f = _problem(H, W, seed=H * 7 + W)
    with fe.Solver([f], k, th, tile=tile) as s:
        assert s.tile == (tile & 0xff, tile & 0xff)
        assert s.cluster == (4 if tile & 0x100 else 1)
        g, Fg = s.gradient(0, f)
    g_ref, F_ref = orc.gradF(f, k, th)
    assert _relmax(g, g_ref) <= GRAD_TOL
    assert Fg == pytest.approx(F_ref, rel=E_TOL)


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("shape", [(64, 64), (131, 77), (8, 9)])
def test_energy_parity(fe, orc, bank, shape, tile):
    k, th = bank
    H, W = shape
    u, f = _problem(H, W, seed=3)
    lam = 5.0
    with fe.Solver([f], k, th, lam=lam, tile=tile) as s:
        E, F, G = s.energy(0, u)
        info = s.info(0)
    assert F == pytest.approx(orc.F(u, k, th), rel=E_TOL)
    assert G == pytest.approx(orc.G(u, f, lam), rel=E_TOL)
    # the state holds F, G of u^0 = f
    assert info["F"] == pytest.approx(orc.F(f, k, th), rel=E_TOL)
    assert info["G"] == pytest.approx(orc.G(f, f, lam), rel=E_TOL)


# Bound on the FP32 evaluation error of the descent-test quantity
# F(u1) - F(u) - <g,D> - L/2 |D|^2 relative to |F| + |<g,D>|: per-pixel
# energies are FP32 sums of 48 terms theta_i log(1 + z_i^2), each with a few
# ulp of error in the log and in z (see GRAD_TOL), summed exactly enough in
# FP64; 4e-6 covers the worst case of that chain.  Within this margin the GPU
# and the FP64 oracle may legitimately take different decisions.
NOISE_REL = 4e-6


def _oracle_candidate(orc, f, k, th, prm, u, up, L):
    r = orc.ipiano_fixed(f, k, th, prm, [L], u, up)
    assert r["status"] == 0
    return r


def _check_decisions(orc, f, k, th, prm, u, up, L_start, L_acc, eta=2.0):
    """The GPU started at L_start and accepted at L_acc = L_start * eta^K:
    the oracle's FP64 test must reject (or be within noise) at every
    L_start * eta^j, j < K, and accept (or be within noise) at L_acc.
    Returns the oracle's step at L_acc."""
    K = int(round(np.log(L_acc / L_start) / np.log(eta)))
    assert abs(L_start * eta ** K - L_acc) <= 1e-12 * L_acc
    for j in range(K + 1):
        r = _oracle_candidate(orc, f, k, th, prm, u, up, L_start * eta ** j)
        F1, margin, gd = r["rec"][0, 2], r["rec"][0, 5], r["rec"][0, 6]
        noise = NOISE_REL * (abs(F1) + abs(gd))
        if j < K:
            assert margin <= noise, ("GPU rejected a step the oracle accepts by a clear margin",
                                     j, margin, noise)
        else:
            assert margin >= -noise, ("GPU accepted a step the oracle rejects by a clear margin",
                                      margin, noise)
    return r


def _dd_tol(dd_ref, N, umax):
    dD = np.sqrt(N) * STEP_TOL * umax  # |delta D| from the per-step bound
    return 2 * np.sqrt(dd_ref) * dD + dD * dD


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("shape,L0", [((64, 64), 1.0), ((131, 77), 1e-3), ((96, 200), 0.05)])
def test_single_step_parity(fe, orc, bank, shape, L0, tile):
    """After k GPU steps, one more GPU step vs the FP64 oracle started from
    the GPU's own state: same backtracking decisions (up to FP32 noise in the
    energy test) and the same u^{n+1} at the accepted L."""
    k, th = bank
    H, W = shape
    _, f = _problem(H, W, seed=11, kind="textured")
    prm = orc.params(lam=5.0, beta=0.8, L0=L0, eta=2.0, c2=1e-6, max_backtrack=30, max_iter=1)
    with fe.Solver([f], k, th, lam=5.0, beta=0.8, L0=L0, eta=2.0, c2=1e-6, tile=tile) as s:
        for nsteps in (0, 3, 10):
            if nsteps:
                assert s.step(nsteps) == fe.FE_OK
            u, up, g, info = s.get_state(0)
            assert s.step(1) == fe.FE_OK
            u1 = s.get_u(0)
            info1 = s.info(0)
            ref = _check_decisions(orc, f, k, th, prm, u, up, info["L"], info1["L"])
            assert _relmax(u1, ref["u"]) <= STEP_TOL
            assert info1["F"] == pytest.approx(ref["rec"][0, 2], rel=E_TOL)
            assert info1["G"] == pytest.approx(ref["rec"][0, 3], rel=E_TOL)
            assert abs(info1["last_dd"] - ref["rec"][0, 7]) <= _dd_tol(
                ref["rec"][0, 7], H * W, np.max(np.abs(ref["u"])))


@pytest.mark.parametrize("tile", TILES)
def test_trajectory_64x64_100_iterations(fe, orc, bank, tile):
    """64x64 piecewise image, L = 1 speckle, lambda = 5, 100 iterations.  The
    GPU's accepted L_n are replayed in the FP64 oracle (prescribed-L update);
    every GPU decision agrees with the oracle's FP64 test up to FP32 noise and
    the trajectories agree to 1e-4 of max|u| after 100 iterations."""
    k, th = bank
    _, f = _problem(64, 64, seed=0)
    prm = orc.params(lam=5.0, beta=0.8, L0=1.0, eta=2.0, c2=1e-6, max_iter=1)
    Ls, Hs, states = [], [], []
    with fe.Solver([f], k, th, lam=5.0, L0=1.0, tile=tile) as s:
        L_prev = s.info(0)["L"]
        for n in range(100):
            u, up, _, _ = s.get_state(0)
            states.append((u, up, L_prev))
            assert s.step(1) == fe.FE_OK
            i = s.info(0)
            Ls.append(i["L"])
            Hs.append(i["H"])
            L_prev = i["L"]
        ug = s.get_u(0)
    ref = orc.ipiano_fixed(f, k, th, prm, Ls, f)
    assert ref["status"] == 0
    assert _relmax(ug, ref["u"]) <= 1e-4
    np.testing.assert_allclose(Hs, ref["rec"][:, 4], rtol=1e-6)
    # every decision, checked from the GPU's own state at that iteration
    for n in range(0, 100, 7):
        u, up, L_start = states[n]
        _check_decisions(orc, f, k, th, prm, u, up, L_start, Ls[n])


@pytest.mark.parametrize("tile", [0, 32 | 0x100])
def test_loop_modes_bit_identical(fe, bank, tile):
    """The CUDA-graph loop (one while node; for clusters the kernel node carries
    the cluster dimension), the persistent launch (the cluster tile runs as the
    graph loop) and the host loop give the same bits."""
    k, th = bank
    _, f = _problem(100, 90, seed=5)
    outs = []
    for mode in (0, 1, 2):
        with fe.Solver([f], k, th, L0=1e-2, loop_mode=mode, tile=tile) as s:
            assert s.step(25) == fe.FE_OK
            outs.append((s.get_u(0), s.info(0)))
    for m in (1, 2):  # the graph loop and the persistent launch
        assert np.array_equal(outs[0][0], outs[m][0])
        assert outs[0][1]["L"] == outs[m][1]["L"] and outs[0][1]["H"] == outs[m][1]["H"]


def test_checkpoint_resume_bit_exact(fe, bank):
    k, th = bank
    _, f = _problem(80, 70, seed=9)
    with fe.Solver([f], k, th, L0=1e-2) as a:
        a.step(10)
        ck = a.get_state(0)
        a.step(15)
        ua = a.get_u(0)
        ia = a.info(0)
    with fe.Solver([f], k, th, L0=1e-2) as b:
        b.set_state(0, *ck)
        b.step(15)
        ub = b.get_u(0)
        ib = b.info(0)
    assert np.array_equal(ua, ub)
    assert ia["H"] == ib["H"] and ia["L"] == ib["L"] and ia["n"] == ib["n"] == 25


@pytest.mark.parametrize("tile", TILES)
def test_batch_of_uneven_images_matches_single(fe, orc, bank, tile):
    k, th = bank
    shapes = [(64, 64), (131, 77), (9, 300), (200, 150)]
    fs = [_problem(H, W, seed=20 + i)[1] for i, (H, W) in enumerate(shapes)]
    with fe.Solver(fs, k, th, L0=1e-2, tile=tile) as s:
        assert s.step(5) == fe.FE_OK
        ub = [s.get_u(i) for i in range(len(fs))]
        ib = [s.info(i) for i in range(len(fs))]
    for i, f in enumerate(fs):
        with fe.Solver([f], k, th, L0=1e-2, tile=tile) as s1:
            s1.step(5)
            assert np.array_equal(s1.get_u(0), ub[i])
            assert s1.info(0)["L"] == ib[i]["L"]
        g_ref, _ = orc.gradF(ub[i], k, th)
        with fe.Solver([f], k, th) as s2:
            g, _ = s2.gradient(0, ub[i])
        assert _relmax(g, g_ref) <= GRAD_TOL


def test_backtracking_limit_and_invalid_input(fe, bank):
    k, th = bank
    u, f = _problem(32, 32, seed=2)
    # intensities of order 0.01-2.5: responses in the convex part of rho, and
    # a tiny L0 with no backtracking allowed must fail the descent test
    with fe.Solver([f * 0.01], k, th, lam=0.01, L0=1e-6, max_backtrack=0) as s:
        assert s.step(3) == fe.FE_EBACKTRACK
        assert s.info(0)["status"] == fe.FE_EBACKTRACK
    bad = f.copy()
    bad[3, 4] = 0.0
    with pytest.raises(fe.FeError) as e:
        fe.Solver([bad], k, th)
    assert e.value.status == fe.FE_EINVAL
    bad[3, 4] = np.nan
    with pytest.raises(fe.FeError):
        fe.Solver([bad], k, th)


def test_device_pointers_and_stream(fe, bank):
    import torch
    k, th = bank
    _, f = _problem(70, 90, seed=4)
    ft = torch.from_numpy(f).cuda()
    stream = torch.cuda.Stream()
    with fe.Solver([ft], k, th, L0=1e-2, stream=stream) as s:
        s.step(4)
        out = torch.empty_like(ft)
        s.get_u(0, out=out)
        torch.cuda.synchronize()
    with fe.Solver([f], k, th, L0=1e-2) as s2:
        s2.step(4)
        assert np.array_equal(out.cpu().numpy(), s2.get_u(0))


@pytest.mark.parametrize("shape", [(512, 512), (4096, 4096)])
def test_gradient_parity_large_sampled(fe, orc, bank, shape):
    """Full-size images: grad F at sampled pixels (borders, corners, tile
    seams and random interior points) against the oracle's per-pixel form."""
    k, th = bank
    H, W = shape
    _, f = _problem(H, W, seed=1, kind="textured")
    with fe.Solver([f], k, th) as s:
        g, _ = s.gradient(0, f)
    rng = np.random.default_rng(0)
    pts = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (1, 2), (2, W - 3), (H - 3, 1),
           (63, 64), (64, 63), (127, 128), (H // 2, W // 2)]
    pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, H, 24), rng.integers(0, W, 24))]
    ref = orc.gradF_at(f, k, th, pts)
    got = np.array([g[p] for p in pts], np.float64)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= GRAD_TOL * scale


def test_tile_autotune_and_shapes(fe, bank):
    """tile = 0 picks one of the four shapes and caches the choice per list of
    image sizes; a forced tile is kept; the per-pixel arithmetic does not
    depend on the tile, so gradients and one step agree bit for bit."""
    k, th = bank
    _, f = _problem(150, 97, seed=31, kind="textured")
    with fe.Solver([f], k, th) as a:
        ta = a.tile
        assert ta in ((64, 64), (32, 32)) and a.cluster in (1, 4)
        with fe.Solver([f], k, th) as b:
            assert b.tile == ta  # cached
    gs, us = [], []
    for t in (64, 32):  # same per-pixel order: bit-identical
        with fe.Solver([f], k, th, L0=1e-2, beta=0.0, tile=t) as s:
            assert s.tile == (t, t) and s.cluster == 1
            gs.append(s.gradient(0, f)[0])
            assert s.step(1) == fe.FE_OK
            us.append(s.get_u(0))
    assert np.array_equal(gs[0], gs[1])
    assert np.array_equal(us[0], us[1])
    # the cluster variants sum each pixel's filters rank by rank: another FP32
    # summation order, so they agree with the others within the FP32
    # gradient bound (and with each other bit for bit: same ranks, same order)
    gcs = []
    for t in (32, 64):
        with fe.Solver([f], k, th, L0=1e-2, beta=0.0, tile=t | 0x100) as s:
            assert s.tile == (t, t) and s.cluster == 4
            gcs.append(s.gradient(0, f)[0])
        assert float(np.max(np.abs(gcs[-1] - gs[0])) / np.max(np.abs(gs[0]))) <= GRAD_TOL
    assert np.array_equal(gcs[0], gcs[1])
    for bad in (16, 48, 128, -1, 0x100, 16 | 0x100, 0x200 | 64):
        with pytest.raises(fe.FeError):
            fe.Solver([f], k, th, tile=bad)


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("nf", [1, 5, 9, 48, 64])
def test_filter_counts_and_distinct_weights(fe, orc, tile, nf):
    """Banks of 1..64 filters with distinct weights theta_i (the device pads
    the bank to a multiple of 8 filters, i.e. 2..16 groups of 4, and stages
    each group's taps and weights in shared memory; with the cluster tile,
    ranks without a group exist for nf <= 8): gradient, energy and one step
    against the oracle."""
    from paper_1404_5344_gb300 import synth
    k, _ = synth.filter_bank(nf, 7, seed=nf, theta=0.1)
    th = np.linspace(0.02, 0.3, nf).astype(np.float32)[::-1].copy()
    _, f = _problem(96, 80, seed=nf, kind="textured")
    with fe.Solver([f], k, th, lam=5.0, beta=0.8, L0=1e-2, tile=tile) as s:
        g, Fg = s.gradient(0, f)
        assert s.step(2) == fe.FE_OK
        u, up, _, _ = s.get_state(0)
        assert s.step(1) == fe.FE_OK
        u1, L = s.get_u(0), s.info(0)["L"]
    g_ref, F_ref = orc.gradF(f, k, th)
    err = np.abs(g.astype(np.float64) - g_ref)
    bound = _grad_bound(orc, f, k, th, g_ref, GRAD_TOL, 2.0 ** -24)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert Fg == pytest.approx(F_ref, rel=E_TOL)
    ref = orc.ipiano_fixed(f, k, th, orc.params(lam=5.0, beta=0.8, L0=1e-2, max_iter=1), [L], u, up)
    assert ref["status"] == 0
    assert _relmax(u1, ref["u"]) <= STEP_TOL


def _grad_bound(orc, u, k, th, g_ref, tol, eps_z):
    """Per-pixel bound on the gradient error for any bank: tol max|g_ref|
    (the adjoint's FP32 accumulation, as for the 48-filter bank) plus the
    rounding of z = k * u carried through rho'': a 49-term FMA chain errs
    by about sqrt(49) eps_z sum|k||u| in a random-walk model, and
    |d rho'| = |rho''(z)| |dz|, so the gradient errs by up to
    7 eps_z A(p), A = sum_i theta_i |K_i|^T (|rho''(z_i)| |K_i| u); 8 is
    used.  For small banks max|g| is small against A, so a bound relative
    to max|g| alone does not hold there."""
    u = np.asarray(u, np.float64)
    A = np.zeros_like(u)
    for i in range(k.shape[0]):
        ka = np.abs(k[i]).astype(np.float64)
        z = orc.K(u, k[i])
        A += th[i] * orc.KT(np.abs(2.0 * (1.0 - z * z) / (1.0 + z * z) ** 2) * orc.K(u, ka), ka)
    return tol * np.max(np.abs(g_ref)) + 8 * eps_z * A + 2.0 ** -23 * np.abs(g_ref)
