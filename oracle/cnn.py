"""FP64 CPU reference of the warm-start CNN (forward, loss and gradients).

TEST INFRASTRUCTURE ONLY (the oracle package): used by the tests to check the
CUDA inference and training kernels; never imported by the library.

Network, as the library defines it (the paper has no counterpart: it starts
iPiano from the observation): five 3x3 convolutions with zero padding
(cross-correlation), channels 1 -> 32 -> 32 -> 32 -> 32 -> 1, bias, ReLU after
the first four layers.  Input x = log f - 4.5, output d, prediction
u0 = f exp(d); loss = mean_p (d_p - t_p)^2 with t = log u* - log f.
Parameter vector: for each layer W[cout][cin][3][3] then b[cout].

Everything is plain NumPy in float64 with explicit loops over (out channel,
in channel, tap); the backward pass is the chain rule written out layer by
layer.  Pinned by tests/test_oracle_cnn.py (SciPy correlation, finite
differences).
"""
from __future__ import annotations

import numpy as np

WIDTH, DEPTH, M0 = 32, 5, 4.5


def layer_shapes():
    ch = [1] + [WIDTH] * (DEPTH - 1) + [1]
    return [(ch[l + 1], ch[l]) for l in range(DEPTH)]


def num_params():
    return sum(co * ci * 9 + co for co, ci in layer_shapes())


def unpack(params):
    p = np.asarray(params, np.float64).ravel()
    out, off = [], 0
    for co, ci in layer_shapes():
        w = p[off:off + co * ci * 9].reshape(co, ci, 3, 3)
        off += co * ci * 9
        b = p[off:off + co]
        off += co
        out.append((w, b))
    assert off == p.size
    return out


def pack(layers):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


def conv3x3(x, w, b):
    """y[o] = b[o] + sum_c sum_{dy,dx} w[o,c,dy,dx] x_pad[c, y+dy, x+dx]
    (zero padding by 1).  x: [C, H, W]."""
    C, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    y = np.empty((w.shape[0], H, W))
    for o in range(w.shape[0]):
        acc = np.full((H, W), b[o])
        for c in range(C):
            for dy in range(3):
                for dx in range(3):
                    acc += w[o, c, dy, dx] * xp[c, dy:dy + H, dx:dx + W]
        y[o] = acc
    return y


def forward(params, f):
    """Returns (d, activations) for one image f [H, W]."""
    layers = unpack(params)
    a = [np.log(np.asarray(f, np.float64))[None] - M0]
    for l, (w, b) in enumerate(layers):
        z = conv3x3(a[-1], w, b)
        a.append(np.maximum(z, 0.0) if l < DEPTH - 1 else z)
    return a[-1][0], a


def predict(params, f):
    d, _ = forward(params, f)
    return np.asarray(f, np.float64) * np.exp(d)


def loss_grad(params, fs, us):
    """Loss mean over all pixels of the batch and its gradient (FP64).
    fs, us: [B, H, W]."""
    layers = unpack(params)
    fs = np.asarray(fs, np.float64)
    us = np.asarray(us, np.float64)
    n = fs.size
    grads = [(np.zeros_like(w), np.zeros_like(b)) for w, b in layers]
    loss = 0.0
    for f, u in zip(fs, us):
        d, a = forward(params, f)
        e = d - (np.log(u) - np.log(f))
        loss += float(np.sum(e * e))
        g = (2.0 * e / n)[None]  # d loss / d output
        for l in range(DEPTH - 1, -1, -1):
            w, _ = layers[l]
            if l < DEPTH - 1:
                g = g * (a[l + 1] > 0)  # through the ReLU of layer l
            x = a[l]
            C, H, W = x.shape
            xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
            gw, gb = grads[l]
            for o in range(w.shape[0]):
                gb[o] += g[o].sum()
                for c in range(C):
                    for dy in range(3):
                        for dx in range(3):
                            gw[o, c, dy, dx] += np.sum(g[o] * xp[c, dy:dy + H, dx:dx + W])
            if l > 0:
                # d loss / d x: correlation with the transposed, flipped kernel
                gp = np.pad(g, ((0, 0), (1, 1), (1, 1)))
                gx = np.zeros_like(x)
                for c in range(C):
                    for o in range(w.shape[0]):
                        for dy in range(3):
                            for dx in range(3):
                                gx[c] += w[o, c, 2 - dy, 2 - dx] * gp[o, dy:dy + H, dx:dx + W]
                g = gx
    return loss / n, pack(grads)
