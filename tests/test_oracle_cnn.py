"""Pins of the FP64 warm-start CNN reference (oracle/cnn.py): the convolution
against SciPy's 2-D cross-correlation, the gradients against central finite
differences of the loss, and the parameter layout."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn


def test_param_count_and_layout():
    assert cnn.num_params() == (1 * 32 * 9 + 32) + 3 * (32 * 32 * 9 + 32) + (32 * 9 + 1)
    p = np.arange(cnn.num_params(), dtype=float)
    np.testing.assert_array_equal(cnn.pack(cnn.unpack(p)), p)
    w0, b0 = cnn.unpack(p)[0]
    assert w0.shape == (32, 1, 3, 3) and b0[0] == 288


def test_conv_is_zero_padded_cross_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 9, 11))
    w = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    y = cnn.conv3x3(x, w, b)
    for o in range(2):
        ref = b[o] + sum(correlate2d(x[c], w[o, c], mode="same", boundary="fill") for c in range(3))
        np.testing.assert_allclose(y[o], ref, rtol=1e-13, atol=1e-12)


def test_gradient_finite_differences():
    rng = np.random.default_rng(1)
    p = rng.standard_normal(cnn.num_params()) * 0.2
    f = rng.uniform(20, 200, (2, 6, 7))
    u = f * rng.uniform(0.8, 1.2, f.shape)
    loss, g = cnn.loss_grad(p, f, u)
    idx = list(rng.choice(cnn.num_params(), 8, replace=False)) + [0, cnn.num_params() - 1, 288, 320]
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (cnn.loss_grad(pp, f, u)[0] - cnn.loss_grad(pm, f, u)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=2e-5, abs=1e-9), i


def test_prediction_is_positive_and_exact_at_zero_net():
    p = np.zeros(cnn.num_params())
    f = np.random.default_rng(2).uniform(10, 250, (5, 5))
    np.testing.assert_allclose(cnn.predict(p, f), f, rtol=1e-15)
    loss, g = cnn.loss_grad(p, f[None], f[None])
    assert loss == 0.0 and np.all(g == 0)
