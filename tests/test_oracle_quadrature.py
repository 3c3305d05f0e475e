"""Pins of the oracle's Gauss-Legendre rules and packet grids."""
import numpy as np
import pytest


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 48])
def test_gl_two_algorithms_and_library(orc, n):
    x1, w1 = orc.gl_newton(n)
    x2, w2 = orc.gl_golub_welsch(n)
    xn, wn = np.polynomial.legendre.leggauss(n)
    # numpy's rule carries ~1e-15 weight error at n = 48 (Golub-Welsch based)
    assert np.allclose(x1, xn, rtol=0, atol=2e-15)
    assert np.allclose(w1, wn, rtol=0, atol=1e-14)
    assert np.allclose(x2, xn, rtol=0, atol=5e-14)
    assert np.allclose(w2, wn, rtol=0, atol=5e-14)


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32])
def test_gl_exact_on_polynomials(orc, n):
    x, w = orc.gl_newton(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x**k) - exact) < 1e-14 * (1 + k)
    # degree 2n is not: P_n vanishes at the nodes, so the rule gives 0 for
    # int P_n^2 = 2/(2n+1)
    Pn = np.polynomial.legendre.legval(x, [0] * n + [1])
    assert abs(np.dot(w, Pn * Pn)) < 1e-13


def test_tangent_edges(orc):
    for N, pmax in [(4, 3.0), (50, 20.0), (300, 20.0)]:
        e = orc.tangent_edges(N, pmax)
        assert e[0] == 0.0 and e[-1] == pmax
        assert np.all(np.diff(e) > 0)
        # tangent map: small bins at small momenta
        assert np.diff(e)[0] < np.diff(e)[-1]


@pytest.mark.parametrize("n", [4, 16, 32])
def test_gl_newton_correctly_rounded(orc, n):
    """40-digit reference (mpmath): the long-double Newton rule rounds to the
    nearest double in every node and weight."""
    mpm = pytest.importorskip("mpmath")
    mpm.mp.dps = 40
    x, w = orc.gl_newton(n)
    xs, ws = [], []
    for i in range(n):
        z = mpm.cos(mpm.pi * (i + mpm.mpf(3) / 4) / (n + mpm.mpf(1) / 2))
        for _ in range(60):
            dp = n * (z * mpm.legendre(n, z) - mpm.legendre(n - 1, z)) / (z * z - 1)
            z = z - mpm.legendre(n, z) / dp
        dp = n * (z * mpm.legendre(n, z) - mpm.legendre(n - 1, z)) / (z * z - 1)
        xs.append(float(z))
        ws.append(float(2 / ((1 - z * z) * dp * dp)))
    assert np.array_equal(x, np.array(xs[::-1]))
    assert np.max(np.abs(w - np.array(ws[::-1])) / np.array(ws[::-1])) <= 2.3e-16
