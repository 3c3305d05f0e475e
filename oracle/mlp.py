"""FP64 reference of the warm-start MLP (test infrastructure only).

Architecture (the library's): x -> x * in_scale + in_shift -> tanh(W1 x + b1)
-> tanh(W2 h1 + b2) -> z = W3 h2 + b3; outputs y = z * out_scale + out_shift.
Training loss: mean over rows and outputs of (z - t~)^2 with
t~ = (t - out_shift) / out_scale.  Flat parameter layout [W1, b1, W2, b2, W3,
b3], weights row-major (output x input).  The gradient is the chain rule
written out; it is pinned by central finite differences
(tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np


def unpack(p, n_in, width, n_out):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    shapes = [(width, n_in), (width,), (width, width), (width,), (n_out, width), (n_out,)]
    out = []
    for sh in shapes:
        n = int(np.prod(sh))
        out.append(p[o:o + n].reshape(sh))
        o += n
    assert o == p.size
    return out


def n_params(n_in, width, n_out):
    return width * n_in + width + width * width + width + n_out * width + n_out


def forward(p, X, n_in, width, n_out, in_aff=None, out_aff=None):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, width, n_out)
    X = np.asarray(X, dtype=np.float64)
    if in_aff is not None:
        X = X * np.asarray(in_aff[0], np.float64) + np.asarray(in_aff[1], np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    z = h2 @ W3.T + b3
    y = z if out_aff is None else z * np.asarray(out_aff[0], np.float64) + np.asarray(out_aff[1], np.float64)
    return y, (X, h1, h2, z)


def loss_grad(p, X, T, n_in, width, n_out, in_aff=None, out_aff=None):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, width, n_out)
    _, (Xn, h1, h2, z) = forward(p, X, n_in, width, n_out, in_aff, out_aff)
    T = np.asarray(T, dtype=np.float64)
    if out_aff is not None:
        T = (T - np.asarray(out_aff[1], np.float64)) / np.asarray(out_aff[0], np.float64)
    n = X.shape[0]
    d = z - T
    loss = np.sum(d * d) / (n * n_out)
    dz = 2.0 * d / (n * n_out)
    gW3 = dz.T @ h2
    gb3 = dz.sum(axis=0)
    d2 = (dz @ W3) * (1.0 - h2 * h2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (1.0 - h1 * h1)
    gW1 = d1.T @ Xn
    gb1 = d1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
