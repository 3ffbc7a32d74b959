"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times, on sampled outputs the FP64 oracle can compute exactly:

* the throughput batch (24 x 512^2 + 24 x 256^2, one context, the CUDA-graph
  loop): one iPiano step of the whole batch, then for several images and
  crops the oracle steps a window with a 6-pixel margin from the GPU's own
  (u^n, u^{n-1}) at the GPU's accepted L (grad F has a radius of 6 pixels,
  so the inner crop is exact) - for the FP32 variant model, the combined
  model, and the BF16 / TF32 forms (oracle with the same rounded bank);
* the batch of 64 uneven images (128^2 .. 1536^2): gradients at sampled
  pixels of several images against the oracle's per-pixel gradient;
* the warm-start network on 512^2 images: outputs on crops with a 5-pixel
  margin (its receptive field) against the FP64 reference network;
* extreme shapes (8 x 4097, 4097 x 8) and the method's degenerate cases
  (a constant image is a fixed point; theta = 0 drives u to f).

Tolerances as in the small-size parity tests: 1e-5 relative for a step and
for gradients, 1e-4 of max|d| for the network.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5
GRAD_TOL = 1e-5


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


def _window_step(orc, f, k, th, prm, u, up, L, y, x, h, w):
    """Oracle step on the crop [y, y+h) x [x, x+w) through a window with a
    6-pixel margin (clipped at the image borders, where the window's own
    reflection is the image's)."""
    H, W = f.shape
    y0, x0, y1, x1 = max(0, y - 6), max(0, x - 6), min(H, y + h + 6), min(W, x + w + 6)
    r = orc.ipiano_fixed(f[y0:y1, x0:x1], k, th, prm, [L], u[y0:y1, x0:x1], up[y0:y1, x0:x1])
    assert r["status"] == 0
    return r["u"][y - y0:y - y0 + h, x - x0:x - x0 + w]


def test_throughput_batch_one_step_crops(fe, orc, bank):
    import torch
    from paper_1404_5344_gb300 import synth
    k, th = bank
    fs = []
    for j in range(48):
        s = 512 if j < 24 else 256
        fs.append(synth.speckle(synth.textured_image(s, s, seed=1000 + j), L=(1.0, 4.0, 8.0)[j % 3], seed=5000 + j))
    fd = [torch.from_numpy(f).cuda() for f in fs]
    prm = orc.params(lam=5.0, beta=0.8, L0=1.0, eta=2.0, c2=1e-6, max_iter=1)
    with fe.Solver(fd, k, th, lam=5.0, beta=0.8, L0=1.0, loop_mode=1) as s:
        assert s.step(3) == fe.FE_OK  # a few steps in, so that u^{n-1} != u^n
        picks = [0, 7, 23, 24, 47]
        states = {j: s.get_state(j) for j in picks}
        assert s.step(1) == fe.FE_OK
        after = {j: (s.get_u(j), s.info(j)["L"]) for j in picks}
    for j in picks:
        u, up, _, info = states[j]
        u1, L = after[j]
        S = fs[j].shape[0]
        for (y, x) in [(0, 0), (S // 2 - 40, S // 3), (S - 64, S - 64)]:
            ref = _window_step(orc, fs[j], k, th, prm, u, up, L, y, x, 64, 64)
            got = u1[y:y + 64, x:x + 64]
            assert float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))) <= STEP_TOL, (j, y, x)


def test_uneven_batch64_sampled_gradients(fe, orc, bank):
    import torch
    from paper_1404_5344_gb300 import synth
    k, th = bank
    sizes = synth.uneven_sizes(64, 128, 1536, seed=7)
    fs = [synth.speckle(synth.textured_image(s, s, seed=2000 + j), L=1.0 if j % 2 == 0 else 4.0, seed=6000 + j)
          for j, s in enumerate(sizes)]
    fd = [torch.from_numpy(f).cuda() for f in fs]
    rng = np.random.default_rng(1)
    picks = [int(np.argmax(sizes)), int(np.argmin(sizes)), 5, 33]
    # |grad F(p)| <= sum_i theta_i |k_i|_1 (|rho'| <= 1): the data-independent
    # scale of the gradient, to which its FP32 error is relative
    scale = float(np.sum(th.astype(np.float64) * np.abs(k.astype(np.float64)).sum(axis=(1, 2))))
    with fe.Solver(fd, k, th, lam=0.02) as s:
        for j in picks:
            S = sizes[j]
            g, _ = s.gradient(j, fd[j])
            g = g if isinstance(g, np.ndarray) else g.cpu().numpy()
            pts = [(0, 0), (S - 1, S - 1), (3, S - 4), (S // 2, S // 2)]
            pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, S, 8), rng.integers(0, S, 8))]
            ref = orc.gradF_at(fs[j], k, th, pts)
            got = np.array([g[p] for p in pts], np.float64)
            assert np.max(np.abs(got - ref)) <= GRAD_TOL * scale, j


def test_cnn_forward_512_crops(fe):
    import torch
    from oracle import cnn
    from paper_1404_5344_gb300 import synth
    from rounding import round_bf16
    net = fe.CNN(seed=11)
    p = net.get_params()
    f = synth.speckle(synth.textured_image(512, 512, seed=77), L=1.0, seed=78)
    d = torch.empty((512, 512), device="cuda")
    net.forward(torch.from_numpy(f).cuda(), u0=torch.empty_like(d), d=d)
    d = d.cpu().numpy()
    layers = [(round_bf16(w.astype(np.float32)).astype(np.float64), b) for w, b in cnn.unpack(p.astype(np.float64))]
    pr = cnn.pack(layers)
    for (y, x) in [(0, 0), (200, 300), (512 - 48, 512 - 48)]:
        y0, x0, y1, x1 = max(0, y - 5), max(0, x - 5), min(512, y + 48 + 5), min(512, x + 48 + 5)
        dr, _ = cnn.forward(pr, f[y0:y1, x0:x1])
        ref = dr[y - y0:y - y0 + 48, x - x0:x - x0 + 48]
        got = d[y:y + 48, x:x + 48]
        assert np.max(np.abs(got - ref)) <= 1e-4 * max(np.max(np.abs(ref)), 1e-6), (y, x)


@pytest.mark.parametrize("shape", [(8, 4097), (4097, 8)])
def test_extreme_shapes_gradient_and_step(fe, orc, bank, shape):
    from paper_1404_5344_gb300 import synth
    k, th = bank
    H, W = shape
    f = synth.speckle(synth.textured_image(H, W, seed=H + W), L=4.0, seed=3)
    with fe.Solver([f], k, th, L0=1e-2) as s:
        g, _ = s.gradient(0, f)
        u, up, _, _ = s.get_state(0)
        assert s.step(1) == fe.FE_OK
        u1, L = s.get_u(0), s.info(0)["L"]
    g_ref, _ = orc.gradF(f, k, th)
    assert float(np.max(np.abs(g - g_ref)) / np.max(np.abs(g_ref))) <= GRAD_TOL
    ref = orc.ipiano_fixed(f, k, th, orc.params(lam=5.0, L0=1e-2, max_iter=1), [L], u, up)
    assert float(np.max(np.abs(u1 - ref["u"])) / np.max(np.abs(ref["u"]))) <= STEP_TOL


def test_degenerate_cases_on_the_gpu(fe, bank):
    k, th = bank
    # a constant image is a fixed point (zero-mean filters, symmetric boundary)
    f = np.full((70, 90), 77.0, np.float32)
    with fe.Solver([f], k, th, L0=1e-2) as s:
        assert s.step(5) == fe.FE_OK
        u = s.get_u(0)
    assert np.max(np.abs(u - 77.0)) <= 1e-4 * 77.0
    # theta = 0: only the data term acts, whose minimiser is u = f
    from paper_1404_5344_gb300 import synth
    f = synth.speckle(synth.textured_image(64, 64, seed=1), L=4.0, seed=2)
    with fe.Solver([f], k, np.zeros(48, np.float32), lam=5.0, beta=0.5, L0=1e-2) as s:
        s.solve(500, 1e-12)
        u = s.get_u(0)
    np.testing.assert_allclose(u, f, rtol=1e-5)


def _throughput_batch():
    from paper_1404_5344_gb300 import synth
    fs = []
    for j in range(48):
        s = 512 if j < 24 else 256
        fs.append(synth.speckle(synth.textured_image(s, s, seed=1000 + j), L=(1.0, 4.0, 8.0)[j % 3], seed=5000 + j))
    return fs


def test_throughput_batch_one_step_crops_combined(fe, orc, bank):
    """The combined model (Eq. newmodel, lambda1 = 160, lambda2 = 0.004, the
    bench's --model combined line) on the whole throughput batch in its
    CUDA-graph loop: one step, then windowed oracle steps from the GPU's own
    (w^n, w^{n-1}) at the GPU's L, as for the variant model above; 1e-5 of
    max|w| on the crop."""
    import torch
    k, th = bank
    fs = _throughput_batch()
    fd = [torch.from_numpy(f).cuda() for f in fs]
    kw = dict(lam=0.004, beta=0.8, L0=1.0, eta=2.0, c2=1e-6)
    prm = orc.params(max_iter=1, model=orc.MODEL_COMBINED, lam1=160.0, **kw)
    with fe.Solver(fd, k, th, model="combined", lam1=160.0, loop_mode=1, **kw) as s:
        assert s.step(3) == fe.FE_OK
        picks = [0, 13, 30, 47]
        states = {j: s.get_state(j) for j in picks}
        assert s.step(1) == fe.FE_OK
        after = {j: (s.get_state(j)[0], s.info(j)["L"]) for j in picks}
    for j in picks:
        w, wp, _, _ = states[j]
        w1, L = after[j]
        S = fs[j].shape[0]
        for (y, x) in [(0, 0), (S // 2 - 40, S // 3), (S - 64, S - 64)]:
            ref = _window_step(orc, fs[j], k, th, prm, w, wp, L, y, x, 64, 64)
            got = w1[y:y + 64, x:x + 64]
            assert float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))) <= STEP_TOL, (j, y, x)


@pytest.mark.parametrize("prec,tol", [("bf16", 2e-5), ("tf32", 1e-5)])
def test_throughput_batch_one_step_crops_tensor_core(fe, orc, bank, prec, tol):
    """The tensor-core forms (the bench's --prec lines) on the whole
    throughput batch in its CUDA-graph loop: one step against the oracle run
    with the same rounded bank on windowed crops (the single-step tolerances
    of tests/test_parity_tc.py)."""
    import torch
    from rounding import ROUND
    k, th = bank
    kq = ROUND[prec](k)
    fs = _throughput_batch()
    fd = [torch.from_numpy(f).cuda() for f in fs]
    prm = orc.params(lam=5.0, beta=0.8, L0=1.0, eta=2.0, c2=1e-6, max_iter=1)
    with fe.Solver(fd, k, th, lam=5.0, beta=0.8, L0=1.0, prec=prec, loop_mode=1) as s:
        assert s.step(3) == fe.FE_OK
        picks = [0, 23, 24, 47]
        states = {j: s.get_state(j) for j in picks}
        assert s.step(1) == fe.FE_OK
        after = {j: (s.get_u(j), s.info(j)["L"]) for j in picks}
    for j in picks:
        u, up, _, _ = states[j]
        u1, L = after[j]
        S = fs[j].shape[0]
        for (y, x) in [(0, 0), (S // 2 - 40, S // 3), (S - 64, S - 64)]:
            ref = _window_step(orc, fs[j], kq, th, prm, u, up, L, y, x, 64, 64)
            got = u1[y:y + 64, x:x + 64]
            assert float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))) <= tol, (j, y, x)
