"""Warm-start CNN: the CUDA inference and training kernels (fe_cnn_*) against
the FP64 reference (oracle/cnn.py) given the same BF16-rounded weights, and
what the trained network gains over plain iPiano.

Tolerances: each activation is an FP32 sum of at most 288 products of BF16
weights and activations; the 32 -> 32 layers run on the tensor cores with
each activation carried as a BF16 hi + lo pair (about 2^-17 relative), so
the network output differs from the FP64 reference by ~1e-5 relative per
layer; 1e-4 of max|d| covers five layers, and u0 = f e^d inherits that
absolute error of d as a relative error.
Gradients are FP32 sums over all pixels of the batch (per-CTA partials
reduced in FP64 in a fixed order): 1e-3 of max|grad| covers the accumulation-order
differences of sums of ~1e3 terms of both signs.
"""
import numpy as np
import pytest

from rounding import round_bf16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_5344_gb300 import build
    build.build()
    from paper_1404_5344_gb300 import fe as fe_mod
    return fe_mod


def _bf16_weights(p):
    """Round the weights (not the biases) as the kernels use them."""
    from oracle import cnn
    layers = [(round_bf16(w.astype(np.float32)).astype(np.float64), b) for w, b in cnn.unpack(p)]
    return cnn.pack(layers)


def _batch(B, H, W, seed):
    """f random in [15, 240]; target u = 3x3 box average of f (a local,
    learnable map), so that training can reduce the loss."""
    from scipy.ndimage import uniform_filter
    rng = np.random.default_rng(seed)
    f = rng.uniform(15, 240, (B, H, W)).astype(np.float32)
    u = np.stack([uniform_filter(x.astype(np.float64), 3, mode="nearest") for x in f]).astype(np.float32)
    return f, u


def test_forward_parity(fe):
    from oracle import cnn
    net = fe.CNN(seed=3)
    rng = np.random.default_rng(0)
    p = (rng.standard_normal(net.num_params) * 0.15).astype(np.float32)
    net.set_params(p)
    f, _ = _batch(2, 20, 37, 1)  # not a multiple of the 16 x 16 tiles
    d = np.empty_like(f)
    u0 = net.forward(f, u0=np.empty_like(f), d=d)
    pr = _bf16_weights(p.astype(np.float64))
    for b in range(2):
        dr, _ = cnn.forward(pr, f[b])
        assert np.max(np.abs(d[b] - dr)) <= 1e-4 * np.max(np.abs(dr))
        np.testing.assert_allclose(u0[b], f[b] * np.exp(dr), rtol=1e-4 * np.max(np.abs(dr)) + 1e-6)


def test_loss_and_gradient_parity(fe):
    from oracle import cnn
    net = fe.CNN(seed=4)
    rng = np.random.default_rng(5)
    p = (rng.standard_normal(net.num_params) * 0.15).astype(np.float32)
    net.set_params(p)
    f, u = _batch(2, 18, 21, 2)
    loss, g = net.loss_grad(f, u)
    lr_, gr = cnn.loss_grad(_bf16_weights(p.astype(np.float64)), f, u)
    assert loss == pytest.approx(lr_, rel=1e-4)
    assert np.max(np.abs(g - gr)) <= 1e-3 * np.max(np.abs(gr))
    # every layer's weights and biases received a gradient
    off = 0
    for co, ci in cnn.layer_shapes():
        nw = co * ci * 9
        assert np.max(np.abs(g[off:off + nw])) > 0 and np.max(np.abs(g[off + nw:off + nw + co])) > 0
        off += nw + co


def test_loss_and_gradient_parity_128(fe):
    """The same at training size: a batch of 2 x 128 x 128 (sums over 32768
    pixels per weight), every parameter's gradient within 1e-3 of the largest
    and each layer's own gradient within 2e-3 of that layer's largest."""
    from oracle import cnn
    net = fe.CNN(seed=11)
    rng = np.random.default_rng(12)
    p = (rng.standard_normal(net.num_params) * 0.12).astype(np.float32)
    net.set_params(p)
    f, u = _batch(2, 128, 128, 13)
    loss, g = net.loss_grad(f, u)
    lr_, gr = cnn.loss_grad(_bf16_weights(p.astype(np.float64)), f, u)
    assert loss == pytest.approx(lr_, rel=1e-4)
    assert np.max(np.abs(g - gr)) <= 1e-3 * np.max(np.abs(gr))
    off = 0
    for co, ci in cnn.layer_shapes():
        n = co * ci * 9 + co
        gl, grl = g[off:off + n], gr[off:off + n]
        assert np.max(np.abs(gl - grl)) <= 2e-3 * np.max(np.abs(grl)), (co, ci)
        off += n


def test_gradients_repeat_bit_for_bit(fe):
    """The weight gradients are per-CTA partial sums (persistent CTAs, each
    taking several tiles) reduced in FP64 in a fixed order, so the same batch
    gives the same loss and gradient bit for bit: twice on one network and
    once on a second network with the same parameters.  Two shapes: crops of
    128 x 128 (more tiles than CTAs; 16-byte loads of the gradient planes)
    and an odd width with ragged 16 x 8 and 16 x 16 edge tiles."""
    import torch
    for (B, H, W), seed in (((8, 128, 128), 21), ((3, 50, 71), 22)):
        f, u = _batch(B, H, W, seed)
        fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u).cuda()
        net = fe.CNN(seed=5)
        l0, g0 = net.loss_grad(fd, ud)
        l1, g1 = net.loss_grad(fd, ud)
        other = fe.CNN(seed=9)
        other.set_params(net.get_params())
        l2, g2 = other.loss_grad(fd, ud)
        assert l0 == l1 == l2
        assert np.array_equal(g0, g1) and np.array_equal(g0, g2)
        assert np.all(np.isfinite(g0)) and np.max(np.abs(g0)) > 0


def test_params_roundtrip_and_training_reduces_loss(fe):
    import torch
    net = fe.CNN(seed=7)
    p0 = net.get_params()
    net.set_params(p0)
    assert np.array_equal(net.get_params(), p0)
    f, u = _batch(8, 32, 32, 3)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u).cuda()
    l0 = net.loss_grad(fd, ud)[0]
    for _ in range(60):
        net.train_step(fd, ud, 3e-3)
    l1 = net.loss_grad(fd, ud)[0]
    assert l1 < 0.5 * l0, (l0, l1)


def test_warm_start_gain(fe):
    """Train on solver-generated pairs (96 observations of 96x96, lambda =
    0.02), then solve 4 held-out 256x256 observations from f and from the
    CNN start to the SAME ENERGY: H* = H_plain + 1e-3 (H(f) - H_plain), with
    H_plain where plain iPiano meets the relative tolerance 1e-6.  Both runs
    must reach H* on every image; the warm start must be taken (H(u0) <
    H(f)) on at least half of the images and need fewer iterations in total
    (an image that fell back to f runs the same solve as plain)."""
    import torch
    from paper_1404_5344_gb300 import synth, warmstart
    k, th = synth.filter_bank(48, 7, seed=0, theta=0.1)
    F, _ = warmstart.make_observations(96, 96, seed=100)
    Fd = torch.from_numpy(F).cuda()
    Ud, its = warmstart.solve_targets(Fd, k, th, tol=1e-6, max_iter=3000, batch=48)
    assert min(its) > 1
    net = fe.CNN(seed=1)
    losses = warmstart.train(net, Fd, Ud, steps=600, batch=16, crop=64, lr=2e-3, seed=0)
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:5])
    Ft, _ = warmstart.make_observations(4, 256, seed=9000)
    res = warmstart.evaluate(net, [torch.from_numpy(x).cuda() for x in Ft], k, th, tol=1e-6)
    for r in res:
        assert r["converged_plain"], r
        assert r["reached_plain_eq"] and r["reached_warm_eq"], r
        assert r["H_plain_eq"] <= r["H_target"] and r["H_warm_eq"] <= r["H_target"], r
        if not r["used_cnn"]:
            assert r["iters_warm_eq"] == r["iters_plain_eq"], r  # fell back to f: the same solve
    assert sum(r["used_cnn"] for r in res) >= 2, res
    assert sum(r["iters_warm_eq"] for r in res) < 0.85 * sum(r["iters_plain_eq"] for r in res), res
