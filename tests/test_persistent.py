"""The persistent trial launch (loop mode 2): one launch runs every trial of
every image; its CTAs take tiles from per-image counters, and the block that
decides an image's trial (the backtracking rule of Sec. II-C) releases the
tiles of that image's next trial at once.

Each image's trials, and each trial's arithmetic and reduction order, are
those of the per-trial launches (loop modes 0 and 1), so every result must be
equal BIT FOR BIT: iterates, energies, L_n, trial and backtrack counts,
statuses.  The batches mix sizes (one tile to hundreds), plane pitches with
and without TMA loads (W % 4), images that stop early and late, and images
that fail.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = ("n", "trials", "backtracks", "L", "alpha", "F", "G", "H", "H_prev", "rel_change", "status", "converged")

SHAPES = [(64, 64), (131, 77), (9, 300), (200, 150), (8, 8), (517, 33), (256, 260)]

FORMS = [("fp32", 64, "variant"), ("fp32", 32, "variant"), ("fp32", 64, "combined"),
         ("bf16", 0, "variant"), ("tf32", 0, "variant"), ("bf16r", 0, "variant"), ("bf16", 0, "combined"),
         ("bf16r", 0, "combined")]


@pytest.fixture(scope="module")
def fe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_5344_gb300 import build
    build.build()
    from paper_1404_5344_gb300 import fe as fe_mod
    return fe_mod


def _fs(shapes, seed):
    from paper_1404_5344_gb300 import synth
    out = []
    for i, (H, W) in enumerate(shapes):
        u = synth.textured_image(H, W, seed=seed + i)
        out.append(synth.speckle(u, L=(1.0, 4.0)[i % 2], seed=seed + 100 + i))
    return out


def _kw(model):
    return dict(model="combined", lam1=160.0, lam=0.02) if model == "combined" else dict(lam=5.0)


def _run(fe, fs, bank, mode, prec, tile, model, fn, L0=1e-2):
    k, th = bank
    with fe.Solver(fs, k, th, L0=L0, prec=prec, tile=tile, loop_mode=mode, **_kw(model)) as s:
        ret = fn(s)
        return ret, [s.get_u(j) for j in range(len(fs))], [s.info(j) for j in range(len(fs))]


def _same(a, b):
    ra, ua, ia = a
    rb, ub, ib = b
    assert ra == rb
    for j in range(len(ua)):
        assert np.array_equal(ua[j], ub[j]), "image %d: iterates differ" % j
        for key in KEYS:
            assert ia[j][key] == ib[j][key], "image %d: %s %r vs %r" % (j, key, ia[j][key], ib[j][key])


@pytest.mark.parametrize("prec,tile,model", FORMS)
def test_persistent_solve_equals_per_trial_launches(fe, bank48, prec, tile, model):
    """fe_solve to a relative tolerance: images stop after different numbers
    of iterations, and the small L0 makes the first trials fail the descent
    test; the persistent launch (in a graph, mode 2, or issued directly,
    mode 3) reproduces the per-trial launches."""
    fs = _fs(SHAPES, seed=3)
    run = lambda s: s.solve(60, 1e-4)
    a = _run(fe, fs, bank48, 0, prec, tile, model, run, L0=1e-4)
    b = _run(fe, fs, bank48, 2, prec, tile, model, run, L0=1e-4)
    _same(a, b)
    _same(a, _run(fe, fs, bank48, 3, prec, tile, model, run, L0=1e-4))  # the same launch without a graph
    assert any(x["backtracks"] > 0 for x in b[2]), "the case exercises rejected trials"
    assert len({x["n"] for x in b[2]}) > 1, "images stop at different iterations"


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_persistent_steps_and_energy_target(fe, bank48, prec):
    """fe_step in pieces (including n = 0) and fe_solve_to_energy."""
    fs = _fs(SHAPES[:5], seed=11)

    def steps(s):
        return [s.step(3), s.step(0), s.step(5)]

    _same(_run(fe, fs, bank48, 0, prec, 0, "variant", steps), _run(fe, fs, bank48, 2, prec, 0, "variant", steps))

    k, th = bank48
    with fe.Solver(fs, k, th, L0=1e-2, prec=prec, loop_mode=0) as s:
        s.step(40)
        target = [s.info(j)["H"] for j in range(len(fs))]

    def to_energy(s):
        return s.solve_to_energy(200, target)

    a = _run(fe, fs, bank48, 0, prec, 0, "variant", to_energy)
    b = _run(fe, fs, bank48, 2, prec, 0, "variant", to_energy)
    _same(a, b)
    assert all(x["converged"] == 1 and x["n"] <= 40 for x in b[2])


def test_persistent_many_images(fe, bank48):
    """More images than one 32-lane scan of the counters covers (70), sizes
    from one tile to a few, solved to tolerance: equal to per-trial launches
    and to one context per image."""
    rng = np.random.default_rng(5)
    shapes = [(int(a), int(b)) for a, b in zip(rng.integers(8, 150, 70), rng.integers(8, 150, 70))]
    fs = _fs(shapes, seed=21)
    run = lambda s: s.solve(40, 1e-3)
    a = _run(fe, fs, bank48, 1, "fp32", 64, "variant", run)
    b = _run(fe, fs, bank48, 2, "fp32", 64, "variant", run)
    _same(a, b)
    for j in (0, 17, 69):
        one = _run(fe, [fs[j]], bank48, 2, "fp32", 64, "variant", run)
        assert np.array_equal(one[1][0], b[1][j])
        assert one[2][0]["n"] == b[2][j]["n"]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_persistent_failing_and_idle_images(fe, bank48, prec):
    """Images that stop with an error (no backtracking allowed from a small
    L0: the first trial fails), and calls with nothing to iterate, end the
    launch with the per-trial launches' statuses."""
    k, th = bank48
    fs = _fs(SHAPES[:4], seed=31)
    outs = []
    for mode in (0, 2):
        with fe.Solver(fs, k, th, L0=1e-4, max_backtrack=0, prec=prec, loop_mode=mode) as s:
            w = s.step(5)
            outs.append((w, [s.info(j) for j in range(len(fs))], [s.get_u(j) for j in range(len(fs))]))
            # every image has stopped: further calls have nothing to run
            assert s.step(3) == w
            with pytest.raises(fe.FeError) as e:
                s.solve(10, 1e-6)
            assert e.value.status == fe.FE_EBACKTRACK
    assert outs[0][0] == outs[1][0] == fe.FE_EBACKTRACK
    for j in range(len(fs)):
        assert np.array_equal(outs[0][2][j], outs[1][2][j])
        for key in KEYS:
            assert outs[0][1][j][key] == outs[1][1][j][key]


def test_persistent_one_trial_launch_per_call(fe, bank48):
    """Loop mode 2 issues one begin kernel and ONE trial launch per fe_step,
    however many trials the images take; mode 1 one launch per trial.  (The
    tile is given: the autotuner may pick a cluster tile for so small a batch,
    and a cluster tile runs mode 2 as mode 1.)"""
    k, th = bank48
    fs = _fs(SHAPES[:3], seed=41)
    with fe.Solver(fs, k, th, L0=1e-2, loop_mode=2, tile=64) as s:
        c0 = s.launch_count()
        s.step(20)
        assert s.launch_count() - c0 == 2
        assert max(s.info(j)["trials"] for j in range(len(fs))) >= 20
    with fe.Solver(fs, k, th, L0=1e-2, loop_mode=2, tile=32 | 0x100) as s:
        c0 = s.launch_count()
        s.step(20)
        assert s.launch_count() - c0 == 1 + max(s.info(j)["trials"] for j in range(len(fs)))
    with fe.Solver(fs, k, th, L0=1e-2, loop_mode=1, tile=64) as s:
        c0 = s.launch_count()
        s.step(20)
        assert s.launch_count() - c0 == 1 + max(s.info(j)["trials"] for j in range(len(fs)))


def test_persistent_claim_wait_is_bounded(fe):
    """The persistent launch's tile claim waits for a trial decision with a
    time limit: with one image counted active, its only tile taken and no
    decision ever coming, the claim gives up after the limit, returns no
    tile and raises the launch's abort flag (the solver's limit is 4 s; the
    self-test runs it at 0.2 s).  Nothing here faults or hangs the GPU."""
    import ctypes as C
    aborted, waited = C.c_int(-1), C.c_double(0.0)
    st = fe.lib.fe_persist_wait_selftest(0.2, C.byref(aborted), C.byref(waited))
    assert st == fe.FE_ETIMEOUT and aborted.value == 1
    assert 0.2 <= waited.value < 3.0, waited.value
    assert fe.lib.fe_persist_wait_selftest(0.0, C.byref(aborted), C.byref(waited)) == fe.FE_EINVAL
