"""Pins of the FP64 reference MLP: its gradient against central finite
differences of its loss (an identity of calculus, not a retyped formula)."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    n_in, width, n_out, n = 5, 7, 4, 6
    p = rng.standard_normal(mlp.n_params(n_in, width, n_out)) * 0.5
    X = rng.standard_normal((n, n_in))
    T = rng.standard_normal((n, n_out))
    in_aff = (rng.uniform(0.5, 2, n_in), rng.standard_normal(n_in) * 0.1)
    out_aff = (rng.uniform(0.5, 2, n_out), rng.standard_normal(n_out))
    loss, g = mlp.loss_grad(p, X, T, n_in, width, n_out, in_aff, out_aff)
    h = 1e-6
    fd = np.zeros_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = mlp.loss_grad(p + e, X, T, n_in, width, n_out, in_aff, out_aff)
        lm, _ = mlp.loss_grad(p - e, X, T, n_in, width, n_out, in_aff, out_aff)
        fd[i] = (lp - lm) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-8 * max(1.0, np.abs(g).max())
    assert loss > 0


def test_forward_layout_and_affine():
    rng = np.random.default_rng(4)
    n_in, width, n_out = 3, 4, 2
    p = rng.standard_normal(mlp.n_params(n_in, width, n_out))
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, n_in, width, n_out)
    x = rng.standard_normal((1, n_in))
    y, _ = mlp.forward(p, x, n_in, width, n_out, out_aff=(np.array([2.0, 3.0]), np.array([1.0, -1.0])))
    z = W3 @ np.tanh(W2 @ np.tanh(W1 @ x[0] + b1) + b2) + b3
    assert np.allclose(y[0], z * [2.0, 3.0] + [1.0, -1.0], rtol=0, atol=1e-14)
