"""Pins for the oracle's boundary extension and filter operators K_i, K_i^T
(Sec. II-A: k_i * u is a convolution; Sec. II-C: K_i is its N x N matrix and
K_i^T the matrix transpose).  Nothing here calls the CUDA path."""
import json
import os

import numpy as np
import pytest
from scipy.signal import convolve2d

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rng(s):
    return np.random.default_rng(s)


def test_pad_matches_numpy_symmetric(orc):
    for (H, W, p) in [(8, 8, 3), (13, 17, 3), (5, 4, 3), (3, 3, 1), (4, 9, 6)]:
        u = _rng(H * W).standard_normal((H, W))
        assert np.array_equal(orc.pad(u, p), np.pad(u, p, mode="symmetric"))


def test_mirror_index_examples(orc):
    # ... c b a | a b c ... : -1 -> 0, -2 -> 1, n -> n-1, n+1 -> n-2
    assert [orc.mirror(j, 5) for j in (-3, -2, -1, 0, 4, 5, 6, 7)] == [2, 1, 0, 0, 4, 4, 3, 2]


def test_pad_adjoint_is_transpose_dense(orc):
    H, W, p = 5, 6, 3
    n, m = H * W, (H + 2 * p) * (W + 2 * p)
    P = np.zeros((m, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        P[:, j] = np.pad(e.reshape(H, W), p, mode="symmetric").ravel()
    PT = np.zeros((n, m))
    for j in range(m):
        e = np.zeros(m)
        e[j] = 1.0
        PT[:, j] = orc.pad_adjoint(e.reshape(H + 2 * p, W + 2 * p), H, W, p).ravel()
    assert np.array_equal(PT, P.T)


def test_conv_valid_is_true_convolution(orc):
    rng = _rng(3)
    up = rng.standard_normal((19, 23))
    k = rng.standard_normal((7, 7))
    np.testing.assert_allclose(orc.conv_valid(up, k), convolve2d(up, k, mode="valid"),
                               rtol=0, atol=1e-12)


def test_golden_single_tap_and_difference(orc):
    g = json.load(open(os.path.join(GOLD, "conv_shift_3x3.json")))
    u = np.array(g["image"], float)
    assert np.array_equal(orc.pad(u, 1), np.array(g["padded_by_1"], float))
    for c in g["cases"]:
        np.testing.assert_array_equal(orc.K(u, np.array(c["kernel"], float)),
                                      np.array(c["K_u"], float))
    t = g["transpose"]
    np.testing.assert_array_equal(orc.KT(np.array(t["r"], float), np.array(t["kernel"], float)),
                                  np.array(t["KT_r"], float))


def _dense_K_library(k, H, W):
    """K as a dense matrix built from library routines only (np.pad +
    scipy convolve2d applied to unit vectors)."""
    p = k.shape[0] // 2
    n = H * W
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = convolve2d(np.pad(e.reshape(H, W), p, mode="symmetric"), k, mode="valid").ravel()
    return M


def _dense_from_operator(op, H, W):
    n = H * W
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = op(e.reshape(H, W)).ravel()
    return M


@pytest.mark.parametrize("shape", [(8, 8), (7, 9)])
def test_K_and_KT_dense_brute_force(orc, shape):
    H, W = shape
    k = _rng(11).standard_normal((7, 7))
    Mlib = _dense_K_library(k, H, W)
    MK = _dense_from_operator(lambda v: orc.K(v, k), H, W)
    MKT = _dense_from_operator(lambda v: orc.KT(v, k), H, W)
    np.testing.assert_allclose(MK, Mlib, rtol=0, atol=1e-13)
    np.testing.assert_allclose(MKT, Mlib.T, rtol=0, atol=1e-13)


@pytest.mark.parametrize("shape", [(8, 8), (13, 17), (64, 64), (3, 40)])
def test_adjoint_identity(orc, shape):
    H, W = shape
    rng = _rng(H * 1000 + W)
    k = rng.standard_normal((7, 7))
    u = rng.standard_normal((H, W))
    v = rng.standard_normal((H, W))
    lhs = float(np.sum(orc.K(u, k) * v))
    rhs = float(np.sum(u * orc.KT(v, k)))
    assert abs(lhs - rhs) <= 1e-13 * max(1.0, np.abs(orc.K(u, k) * v).sum())


def test_zero_mean_filter_kills_constants(orc):
    # symmetric extension keeps a constant image constant, so a zero-mean
    # filter maps it to exactly zero (up to rounding of the filter sum)
    k = _rng(5).standard_normal((7, 7))
    k -= k.mean()
    z = orc.K(np.full((10, 12), 37.5), k)
    assert np.max(np.abs(z)) < 1e-12
