"""Pins of the oracle's node-binned lattice P0 (Sec. 3.2, Eqs. perm and gal).

The node sum is the method's quadrature, so it is pinned by what the
mathematics fixes: the l = 0 sum rule (every node weight lands exactly once,
inside the grid or outside it), energy conservation of the recoupling (the
pattern), convergence to the exact cell overlap computed by a different
algorithm, and the symmetry of the exact overlap (P is Hermitian).
"""
import numpy as np
import pytest

PE = np.array([0.0, 0.6, 1.2, 2.0, 3.0])
QE = np.array([0.0, 0.5, 1.1, 1.9, 3.0])


def _rows(P):
    return np.repeat(np.arange(len(P["row_ptr"]) - 1), np.diff(P["row_ptr"]))


@pytest.mark.parametrize("nodes", [(4, 4, 16), (3, 5, 7)])
def test_sum_rule_l0(orc, nodes):
    """sum over targets + out-of-grid weight = 2 B_i Bq_j for l = l' = 0."""
    pe = orc.tangent_edges(20, 20.0)
    qe = orc.tangent_edges(16, 20.0)
    P = orc.P0(pe, qe, *nodes, 1, normalize=False, with_outgrid=True)
    rows = _rows(P)
    tot = np.bincount(rows, weights=P["val"][:, 0], minlength=20 * 16) + P["outgrid"][:, 0]
    ref = np.outer(orc.bnorm(pe), orc.bnorm(qe)).ravel() * 2.0
    assert np.max(np.abs(tot - ref) / ref) < 1e-13
    # weight does leave the grid for large p, q and never for the smallest cells
    assert P["outgrid"][:, 0].max() > 0
    assert P["outgrid"][0, 0] == 0


def test_sum_rule_all_pairs(orc):
    """for every (l, l'): binned sum + out-of-grid = un-binned node sum."""
    pe = orc.tangent_edges(10, 20.0)
    qe = orc.tangent_edges(12, 20.0)
    P = orc.P0(pe, qe, 4, 4, 16, 5, normalize=False, with_outgrid=True)
    tot = orc.P0_node_totals(pe, qe, 4, 4, 16, 5)
    rows = _rows(P)
    for k in range(orc.n_pairs(5)):
        s = np.bincount(rows, weights=P["val"][:, k], minlength=120) + P["outgrid"][:, k]
        scale = np.bincount(rows, weights=np.abs(P["val"][:, k]), minlength=120) + 1e-300
        assert np.max(np.abs(s - tot[:, k]) / scale) < 1e-13


def test_pattern_conserves_energy(orc):
    """every stored target cell overlaps the source cell's energy band
    p^2 + 3q^2/4 (the recoupling conserves H0)."""
    pe = orc.tangent_edges(30, 20.0)
    qe = orc.tangent_edges(25, 20.0)
    P = orc.P0(pe, qe, 4, 4, 16, 1)
    M = 25
    rows, cols = _rows(P), P["col"]
    def band(c):
        i, j = np.divmod(c, M)
        return pe[i] ** 2 + 0.75 * qe[j] ** 2, pe[i + 1] ** 2 + 0.75 * qe[j + 1] ** 2
    slo, shi = band(rows)
    tlo, thi = band(cols)
    assert np.all((tlo < shi) & (slo < thi))
    # columns sorted and unique within each row
    for c in range(0, 30 * 25, 37):
        cc = cols[P["row_ptr"][c]:P["row_ptr"][c + 1]]
        assert np.all(np.diff(cc) > 0)


def test_cross_parity_blocks_zero(orc):
    P = orc.P0(PE, QE, 4, 4, 16, 3)
    D = orc.P0_dense(P)
    nc = 16
    for l in range(3):
        for lp in range(3):
            blk = D[l * nc:(l + 1) * nc, lp * nc:(lp + 1) * nc]
            if (l + lp) % 2:
                assert np.all(blk == 0)
            else:
                assert np.any(blk != 0)
    assert orc.n_pairs(1) == 1 and orc.n_pairs(3) == 5 and orc.n_pairs(5) == 13


@pytest.mark.parametrize("l,lp", [(0, 0), (0, 2), (1, 1), (2, 2)])
def test_exact_overlap_symmetric(orc, l, lp):
    """The exact overlap is symmetric: I(c, t; l, l') = I(t, c; l', l), since P
    is Hermitian; a wrong sign or factor in the recoupled momenta breaks it."""
    # cells away from p = 0 and q = 0, where y' is smooth in y
    pairs = [(5, 5), (6, 9), (10, 7), (11, 13), (13, 14)]
    n_nonzero = 0
    for c, t in pairs:
        a = orc.exact_overlap(PE, QE, c, t, l, lp)
        b = orc.exact_overlap(PE, QE, t, c, lp, l)
        assert abs(a - b) <= 1e-9 * max(abs(a), abs(b), 1e-12), (c, t, a, b)
        n_nonzero += abs(a) > 1e-6
    assert n_nonzero >= 3


def test_node_binning_converges_to_exact_overlap(orc):
    """The node-binned estimate approaches the exact overlap as the nodes
    grow, for every target of a source row and for l' = 0 and 2."""
    c = 6  # cell (i=1, j=2)
    targets = range(16)
    fine = orc.P0(PE, QE, 64, 64, 256, 1, normalize=False)
    hit = set(fine["col"][fine["row_ptr"][c]:fine["row_ptr"][c + 1]].tolist())
    for (l, lp), k in [((0, 0), 0), ((0, 2), 1)]:
        exact = np.array([orc.exact_overlap(PE, QE, c, t, l, lp, epsrel=1e-8) if t in hit else 0.0
                          for t in targets])
        errs = []
        for nodes in [(4, 4, 16), (8, 8, 32), (16, 16, 64), (32, 32, 128)]:
            P = orc.P0(PE, QE, *nodes, 3, normalize=False)
            row = np.zeros(16)
            sl = slice(P["row_ptr"][c], P["row_ptr"][c + 1])
            row[P["col"][sl]] = P["val"][sl, k]
            errs.append(np.abs(row - exact).sum() / np.abs(exact).sum())
        assert errs[-1] < errs[0]
        assert errs[-1] < 0.5 * errs[1]
        assert errs[-1] < 0.02, (l, lp, errs)


def test_node_binned_asymmetry_shrinks(orc):
    """Node binning is not exactly symmetric; its asymmetry must fall as the
    node count grows (it does not for a wrong mapping)."""
    pe = orc.tangent_edges(6, 8.0)
    qe = orc.tangent_edges(6, 8.0)
    asym = []
    for nodes in [(4, 4, 16), (8, 8, 32), (16, 16, 64)]:
        D = orc.P0_dense(orc.P0(pe, qe, *nodes, 3))
        asym.append(np.linalg.norm(D - D.T) / np.linalg.norm(D))
    assert asym[0] > asym[1] > asym[2]
