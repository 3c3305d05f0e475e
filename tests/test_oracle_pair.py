"""Pins of the oracle's two-body input: v_l and the pair diagonalisation
(Sec. 2.2, Eq. vpot and Eq. exp_z)."""
import numpy as np
import pytest
from scipy import integrate, special


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
def test_scaled_bessel_vs_library(orc, l):
    """exp(-z) i_l(z) = sqrt(pi/(2z)) * ive(l + 1/2, z) (scipy, exponentially
    scaled modified Bessel function)."""
    for z in [1e-8, 1e-3, 0.1, 1.0, 5.0, 20.0, 29.9, 30.1, 60.0, 200.0, 700.0]:
        ref = np.sqrt(np.pi / (2 * z)) * special.ive(l + 0.5, z)
        got = orc.sph_i_scaled(l, z)
        assert abs(got - ref) <= 2e-13 * abs(ref) + 1e-300, (l, z, got, ref)
    assert orc.sph_i_scaled(l, 0.0) == (1.0 if l == 0 else 0.0)


def _vl_radial(l, p, pp, V, a):
    """(2/pi) int_0^inf r^2 j_l(pr) V(r) j_l(p'r) dr by adaptive quadrature."""
    def f(r):
        Vr = sum(Vk * np.exp(-r * r / ak) for Vk, ak in zip(V, a))
        return r * r * special.spherical_jn(l, p * r) * Vr * special.spherical_jn(l, pp * r)
    rmax = 12.0 * np.sqrt(max(a))
    val, _ = integrate.quad(f, 0.0, rmax, limit=800, epsabs=1e-15, epsrel=1e-13)
    return 2.0 / np.pi * val


@pytest.mark.parametrize("l", [0, 1, 2, 4])
def test_vl_closed_form_vs_radial_integral(orc, l):
    pots = [([-3.0], [1.0]), ([-6.0, 2.0], [0.5, 0.1])]
    for V, a in pots:
        for p, pp in [(0.05, 0.3), (0.5, 0.5), (1.0, 2.5), (3.0, 3.2), (6.0, 1.0)]:
            ref = _vl_radial(l, p, pp, V, a)
            got = orc.vl(l, p, pp, V, a)
            assert abs(got - ref) <= 1e-10 * max(abs(ref), 1e-6), (l, p, pp, got, ref)


def test_jacobi_eigensolver_vs_library(orc):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 30))
    A = A + A.T
    ev, V = orc.jacobi_eigh(A)
    evn, Vn = np.linalg.eigh(A)
    assert np.allclose(ev, evn, atol=1e-12)
    for k in range(30):
        assert abs(abs(np.dot(V[k], Vn[:, k])) - 1) < 1e-10
        assert V[k, np.argmax(np.abs(V[k]))] > 0  # sign convention
    assert np.allclose(V @ A @ V.T, np.diag(ev), atol=1e-11)


def _numerov_bound(V, a, l=0, rmax=80.0, n=40000):
    """Ground-state energy of -u'' + (V(r) + l(l+1)/r^2) u = E u by Numerov
    shooting and bisection (hbar^2/(2 mu) = 1)."""
    r = np.linspace(0.0, rmax, n + 1)
    h = r[1] - r[0]
    Vr = sum(Vk * np.exp(-r * r / ak) for Vk, ak in zip(V, a))

    def end_value(E):
        k2 = E - Vr
        u_prev, u = 0.0, h ** (l + 1)
        f = 1 + h * h * k2 / 12.0
        nodes = 0
        for i in range(1, n):
            u_next = ((12 - 10 * f[i]) * u - f[i - 1] * u_prev) / f[i + 1]
            if u_next * u < 0:
                nodes += 1
            u_prev, u = u, u_next
        return u, nodes

    lo, hi = -10.0, -1e-9
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        _, nodes = end_value(mid)
        if nodes >= 1:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def test_pair_bound_state_converges_to_numerov(orc):
    """The packet-basis dimer energy is variational (above the exact one) and
    converges to the coordinate-space Numerov value as the bins shrink."""
    V, a = [-3.0], [1.0]
    ref = _numerov_bound(V, a)
    errs = []
    for N in [100, 200, 400]:
        e = np.linspace(0.0, 10.0, N + 1)
        v, h, eps, O = orc.pair(e, 8, 0, V, a)
        assert eps[0] < 0 < eps[1]  # exactly one bound state
        assert eps[0] > ref
        # h1 is diagonalised: O h O^T = diag(eps), O orthogonal
        assert np.allclose(O @ h @ O.T, np.diag(eps), atol=1e-12 * np.abs(h).max())
        assert np.allclose(O @ O.T, np.eye(N), atol=1e-11)
        errs.append(eps[0] - ref)
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[2] > 3.0  # about second order in the bin width
    assert errs[2] < 0.02 * abs(ref)


def test_pair_tangent_grid_binds_one_dimer(orc):
    """The s-wave Gaussian V = -3 exp(-r^2) binds exactly one dimer on the
    tangent grid up to p_max = 20, and no p- or d-wave state."""
    e = orc.tangent_edges(50, 20.0)
    _, _, eps0, _ = orc.pair(e, 8, 0, [-3.0], [1.0])
    assert eps0[0] < 0 < eps0[1]
    for l in (1, 2):
        _, _, epsl, _ = orc.pair(e, 8, l, [-3.0], [1.0])
        assert epsl[0] > 0
