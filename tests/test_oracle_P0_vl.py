"""Pins of the oracle's variable-limit P0 (Sec. 3.2, after Eq. gal: the cell
overlap reduced to an integral with variable limits).  For every (p, q) GL
node of the source cell the y-interval [-1, 1] is cut where p'^2 or q'^2
crosses a squared bin edge (both are linear in y), so the theta functions of
Eq. perm are exact in y; each piece is integrated by GL.  Pinned by:
  - the l = 0 sum rule: the pieces tile [-1, 1], so every node's weight 2 W
    lands once, in the grid or outside it: sum + out-of-grid = 2 B_i Bq_j;
  - for every (l, l'): sum over targets + out-of-grid = the un-binned
    integral of P_l(y) P_l'(y'(y)) over [-1, 1] (an independent 256-point GL
    rule per node);
  - convergence to the brute-force exact overlap (adaptive quadrature), much
    faster than node binning at equal node counts;
  - the symmetry of the exact overlap (P is Hermitian).
"""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss, legval

PE = np.array([0.0, 0.6, 1.2, 2.0, 3.0])
QE = np.array([0.0, 0.5, 1.1, 1.9, 3.0])


def _rows(P):
    return np.repeat(np.arange(len(P["row_ptr"]) - 1), np.diff(P["row_ptr"]))


@pytest.mark.parametrize("nodes", [(4, 4, 16), (3, 5, 7)])
def test_vl_sum_rule_l0(orc, nodes):
    pe, qe = orc.tangent_edges(20, 20.0), orc.tangent_edges(16, 20.0)
    P = orc.P0_vl(pe, qe, *nodes, 1, normalize=False, with_outgrid=True)
    tot = np.bincount(_rows(P), weights=P["val"][:, 0], minlength=320) + P["outgrid"][:, 0]
    ref = np.outer(orc.bnorm(pe), orc.bnorm(qe)).ravel() * 2.0
    assert np.max(np.abs(tot - ref) / ref) < 1e-13


def _Pl(l, y):
    c = np.zeros(l + 1)
    c[l] = 1.0
    return legval(y, c)


@pytest.mark.parametrize("nx,tol_lp0,tol_all", [(24, 1e-12, None), (256, 1e-12, 1e-6)])
def test_vl_unbinned_totals_all_pairs(orc, nx, tol_lp0, tol_all):
    """binned + out-of-grid = the un-binned y-integral, node by node summed
    over the cell; the reference integrates [-1, 1] in one 1024-point rule.
    For l' = 0 the integrand P_l(y) is a polynomial, exact on every piece:
    the pieces must tile [-1, 1] to rounding.  For l' > 0, where |p'| comes
    close to 0 at y = -1 (p/2 near 3q/4), y' turns over a short stretch of y
    and the per-piece rule needs many points (measured in the worst cell:
    1e-3 at 24 points, 2e-9 at 256)."""
    pe, qe = orc.tangent_edges(8, 10.0), orc.tangent_edges(7, 10.0)
    n_p, n_q, n_ch = 3, 4, 5
    P = orc.P0_vl(pe, qe, n_p, n_q, nx, n_ch, normalize=False, with_outgrid=True)
    rows = _rows(P)
    ty, wy = leggauss(1024)
    tp, wp = leggauss(n_p)
    tq, wq = leggauss(n_q)
    pairs = orc.pair_list(n_ch)
    lp0 = np.array([lp == 0 for _, lp in pairs])
    N, M = 8, 7
    for c in range(N * M):
        i, j = divmod(c, M)
        ref = np.zeros(len(pairs))
        for a in range(n_p):
            hp, mp = 0.5 * (pe[i + 1] - pe[i]), 0.5 * (pe[i + 1] + pe[i])
            p = mp + hp * tp[a]
            for b in range(n_q):
                hq, mq = 0.5 * (qe[j + 1] - qe[j]), 0.5 * (qe[j + 1] + qe[j])
                q = mq + hq * tq[b]
                W = hp * wp[a] * p * p * hq * wq[b] * q * q
                # recoupled momenta from their vector definition: p' = -(p/2 + 3q/4), q' = p - q/2
                p2 = p * p / 4 + 9 * q * q / 16 + 0.75 * p * q * ty
                q2 = p * p + q * q / 4 - p * q * ty
                yp = np.clip((-p * p / 2 - p * q * ty / 2 + 3 * q * q / 8) / np.sqrt(p2 * q2), -1, 1)
                for k, (l, lp) in enumerate(pairs):
                    ref[k] += W * np.sum(wy * _Pl(l, ty) * _Pl(lp, yp))
        got = P["val"][rows == c].sum(axis=0) + P["outgrid"][c]
        scale = np.abs(P["val"][rows == c]).sum(axis=0) + np.abs(P["outgrid"][c]) + 1e-300
        err = np.abs(got - ref) / scale
        assert np.max(err[lp0]) < tol_lp0, c
        if tol_all:
            assert np.max(err) < tol_all, c


def test_vl_converges_to_exact_overlap(orc):
    """Against the brute-force exact overlap of one source row: the
    variable-limit error falls with the (p, q) nodes and stays well below
    node binning's at equal (p, q) nodes (node binning given 4x the y nodes)."""
    c = 6
    fine = orc.P0(PE, QE, 64, 64, 256, 1, normalize=False)
    hit = set(fine["col"][fine["row_ptr"][c]:fine["row_ptr"][c + 1]].tolist())
    for (l, lp), k in [((0, 0), 0), ((0, 2), 1), ((2, 2), 4)]:
        exact = np.array([orc.exact_overlap(PE, QE, c, t, l, lp, epsrel=1e-9) if t in hit else 0.0
                          for t in range(16)])
        ev, eb = [], []
        for n in (4, 8, 16, 32):
            for fn, nx, errs in ((orc.P0_vl, 8, ev), (orc.P0, 32, eb)):
                P = fn(PE, QE, n, n, nx, 3, normalize=False)
                row = np.zeros(16)
                sl = slice(P["row_ptr"][c], P["row_ptr"][c + 1])
                row[P["col"][sl]] = P["val"][sl, k]
                errs.append(np.abs(row - exact).sum() / np.abs(exact).sum())
        assert ev[-1] < 1e-3 and ev[-1] < 0.2 * ev[0], (l, lp, ev)
        assert all(v < b for v, b in zip(ev, eb)), (l, lp, ev, eb)


def test_vl_asymmetry_small_and_shrinking(orc):
    pe, qe = orc.tangent_edges(6, 8.0), orc.tangent_edges(6, 8.0)
    asym, asym_b = [], []
    for n in (4, 8, 16):
        D = orc.P0_dense(orc.P0_vl(pe, qe, n, n, 16, 3))
        asym.append(np.linalg.norm(D - D.T) / np.linalg.norm(D))
        B = orc.P0_dense(orc.P0(pe, qe, n, n, 64, 3))
        asym_b.append(np.linalg.norm(B - B.T) / np.linalg.norm(B))
    assert asym[0] > asym[1] > asym[2]
    assert all(a < b for a, b in zip(asym, asym_b)), (asym, asym_b)
