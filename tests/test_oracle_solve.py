"""Pins of the oracle's channel resolvent G1 (Sec. 2.1 Eq. g_tot, Sec. 2.3
energy averaging) and of the summation of the iterated Faddeev kernel
(Sec. 3.3: iterations plus Pade summation)."""
import numpy as np
import pytest
from scipy import integrate


def _g_quad(qa, qb, Elo, Ehi, ek):
    """(1/(D Bq)) int_{qa}^{qb} q^2 dq (1/D) int_{Elo}^{Ehi} dE P/(E - ek - 3q^2/4)
    with the E integral of the principal value done analytically (the log of
    a ratio) and the q integral adaptive, with the log singularities passed
    as break points; imaginary part from the delta function."""
    D = Ehi - Elo
    Bq = (qb**3 - qa**3) / 3
    pts = [np.sqrt(a / 0.75) for a in (Ehi - ek, Elo - ek) if a > 0]
    pts = [x for x in pts if qa < x < qb]
    f = lambda q: q * q * np.log(abs((Ehi - ek - 0.75 * q * q) / (Elo - ek - 0.75 * q * q)))
    re, _ = integrate.quad(f, qa, qb, points=pts or None, epsabs=0, epsrel=1e-13, limit=400)
    ind = lambda q: q * q * (Elo < ek + 0.75 * q * q < Ehi)
    im, _ = integrate.quad(ind, qa, qb, points=pts or None, epsabs=1e-15, epsrel=1e-13, limit=400)
    return re / (D * Bq) - 1j * np.pi * im / (D * Bq)


@pytest.mark.parametrize("E", [-0.005, 0.5, 3.0])
def test_G1_closed_form_vs_quadrature(orc, E):
    qe = orc.tangent_edges(30, 20.0)
    eps_b = -0.0093
    eps = np.array([[eps_b, 1e-4, 0.03, 0.4, 2.0, 7.5, 50.0]])
    g, j0, D = orc.G1(eps, qe, E, eps_b)
    Elo = eps_b + 0.75 * qe[j0] ** 2
    Ehi = eps_b + 0.75 * qe[j0 + 1] ** 2
    assert abs((Ehi - Elo) - D) < 1e-14 * D
    worst = 0.0
    for k in range(eps.shape[1]):
        for j in range(30):
            ref = _g_quad(qe[j], qe[j + 1], Elo, Ehi, eps[0, k])
            got = g[0, k, j]
            worst = max(worst, abs(got - ref) / abs(ref))
    assert worst < 1e-9


def test_G1_bound_channel_imaginary_part(orc):
    """Im g_{1j} = -pi/D delta_{j j0} for the bound channel (the on-shell bin
    is exactly the bin of q0)."""
    qe = orc.tangent_edges(40, 20.0)
    eps_b = -0.01
    for E in [-0.009, 0.2, 4.0]:
        g, j0, D = orc.G1(np.array([[eps_b, 0.5]]), qe, E, eps_b)
        q0 = np.sqrt((E - eps_b) / 0.75)
        assert qe[j0] <= q0 < qe[j0 + 1]
        im = g[0, 0].imag
        assert abs(im[j0] + np.pi / D) < 1e-12 * np.pi / D
        others = np.delete(im, j0)
        assert np.max(np.abs(others)) < 1e-12 * np.pi / D


def test_wynn_on_known_series(orc):
    # geometric series sum (-2)^n: divergent, Pade [1/1] from S_0..S_2 is
    # exactly 1/3
    wynn = lambda S, est: orc.lib().orc_wynn(
        len(S), np.ascontiguousarray(np.asarray(S, complex).view(np.float64)).ctypes.data_as(orc._D),
        est.ctypes.data_as(orc._D))
    S = np.cumsum([(-2.0) ** n for n in range(8)])
    est = np.zeros(2)
    assert wynn(S[:3], est) == 0
    assert abs(est[0] - 1.0 / 3.0) < 1e-15 and est[1] == 0.0
    # with more terms the next column divides by an exact zero: breakdown is
    # reported and the exact value is still returned
    assert wynn(S, est) == orc.EBREAKDOWN
    assert abs(est[0] - 1.0 / 3.0) < 1e-15
    # log(1 + x) at x = 1 (slowly convergent alternating series)
    S = np.cumsum([(-1.0) ** (n + 1) / n for n in range(1, 22)])
    assert wynn(S, est) == 0
    assert abs(est[0] - np.log(2.0)) < 1e-14


def _problem(orc, N, M, n_ch, nodes=(4, 4, 16), V=(-6.0,), a=(1.0,)):
    # a deeper well than the benchmark potential, so that the coarse test
    # grids still bind the dimer
    desc = dict(pe=orc.tangent_edges(N, 20.0), qe=orc.tangent_edges(M, 20.0), n_p=nodes[0],
                n_q=nodes[1], n_x=nodes[2], n_ch=n_ch, V=list(V), a=list(a), n_pair_nodes=8)
    return orc.Problem(desc)


@pytest.mark.parametrize("n_ch,E,wynn_tol", [(1, 0.5, 2e-6), (1, 2.0, 1e-8), (3, 0.5, 2e-6)])
def test_solve_matches_dense_LU(orc, n_ch, E, wynn_tol):
    """Iteration + Pade (Wynn) and the Krylov form both reproduce the direct
    solution of (I - K) u = u0 (numpy LU) for U00.  Wynn's accuracy is bounded
    by eps * rho(K)^n (rho = 3.2 at E = 0.5 here, 2.0 at E = 2)."""
    pr = _problem(orc, 14, 12, n_ch)
    assert pr.eps_b < 0
    K, u0, j0, D = pr.dense_K(E)
    u = np.linalg.solve(np.eye(len(u0)) - K, u0)
    ref = u[pr.r0(j0)]
    w = pr.solve_wynn(E, max_iter=80, tol=1e-11)
    assert abs(w["U00"] - ref) < wynn_tol * abs(ref), (w, ref)
    gm = pr.solve_gmres(E, tol=1e-12)
    assert gm["status"] == 0 and gm["relres"] < 1e-11
    assert abs(gm["U00"] - ref) < 1e-10 * abs(ref)
    # first iterate is the Born term u0 = O P0 Vt e0
    assert np.allclose(pr.born(j0), u0, rtol=0, atol=1e-13 * np.abs(u0).max())


def test_unitarity_below_breakup(orc):
    """|S| = 1 below the breakup threshold, where Im G1 is rank one on the
    entrance channel (S = 1 - 2 pi i U00 / D)."""
    pr = _problem(orc, 20, 20, 3)
    E = 0.5 * pr.eps_b
    j0, Elo, Ehi, q0 = orc.onshell(pr.qe, E, pr.eps_b)
    assert Ehi < 0.0 and Ehi < pr.eps[0, 1] and Ehi < pr.eps[1:].min()
    gm = pr.solve_gmres(E, tol=1e-13)
    S, _ = pr.amplitudes(E, gm["U00"])
    assert abs(abs(S) - 1.0) < 1e-10
    # the scalar Pade route loses digits as rho(K)^n grows (two trimer
    # eigenvalues lie outside the unit circle below breakup)
    w = pr.solve_wynn(E, max_iter=80, tol=1e-10)
    S2, _ = pr.amplitudes(E, w["U00"])
    assert abs(abs(S2) - 1.0) < 1e-5
    # above breakup the elastic channel loses flux
    gm = pr.solve_gmres(1.0, tol=1e-12)
    S3, _ = pr.amplitudes(1.0, gm["U00"])
    assert abs(S3) < 1.0


def test_U00_one_value_per_onshell_bin(orc):
    """The energy enters G1 only through its on-shell bin (the average over
    the energy bin [E_lo, E_hi], Sec. 2.3) and the Born term only through
    that bin's unit vector, so two energies of one bin give the same U00 bit
    for bit; a neighbouring bin gives another.  (The full-size parity checks
    solve the oracle once per distinct bin on this ground.)"""
    pe, qe = orc.tangent_edges(16, 20.0), orc.tangent_edges(14, 20.0)
    pr = orc.Problem(dict(pe=pe, qe=qe, n_p=3, n_q=3, n_x=8, n_ch=2, V=[-6.0], a=[1.0], n_pair_nodes=6))
    j0, Elo, Ehi, _ = orc.onshell(qe, 0.5, pr.eps_b)
    Es = [Elo + f * (Ehi - Elo) for f in (0.1, 0.5, 0.93)]
    assert all(orc.onshell(qe, e, pr.eps_b)[0] == j0 for e in Es)
    U = [pr.solve_gmres(e, tol=1e-12)["U00"] for e in Es]
    assert U[0] == U[1] == U[2]
    other = pr.solve_gmres(Ehi + 0.5 * (Ehi - Elo), tol=1e-12)["U00"]
    assert abs(other - U[0]) > 1e-6 * abs(U[0])
