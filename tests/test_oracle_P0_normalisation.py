"""Pin of the overall scale of the oracle's P0 and of its per-block factors
sqrt((2l+1)(2l'+1)) (Sec. 3.2, Eqs. perm and gal).

The symmetry tests cannot see a factor that is symmetric in (l, l'), and the
unitarity of S is blind to the scale of P0.  What fixes both is the action
of P = P12 P23 + P13 P23 on a function f of the three momenta that is
totally symmetric, or totally antisymmetric, under exchange of the
particles: each cyclic permutation maps f to itself, so P f = 2 f exactly.

With single-particle momenta in the centre-of-mass frame k1 = p - q/2,
k2 = -p - q/2, k3 = q (p, q the Jacobi momenta of the free energy
p^2 + 3 q^2 / 4 = (k1^2 + k2^2 + k3^2)/2), an L = 0 function of (p, q, y),
y = p.q / (|p| |q|), has the bipolar partial waves

    f_l(p, q) ~ sqrt(2l + 1) int_{-1}^{1} dy P_l(y) f(p, q, y)

(the bipolar harmonic of (l, l) L = 0 is (-1)^l sqrt(2l+1)/(4 pi) P_l(y); the
common factor and the sign (-1)^l drop out, since P0 couples only l, l' of
equal parity).  Projected on the cells, F_(l,c) = int_c p^2 q^2 f_l / sqrt(B_c),
the node-binned P0 must give P0 F -> 2 F block by block as the lattice and
the node counts grow.  The functions used:

  symmetric      exp(-a H) (k1^4 + k2^4 + k3^4)      partial waves l = 0, 2
  symmetric      exp(-a H) (k1^8 + k2^8 + k3^8)      l = 0, 2, 4
  antisymmetric  exp(-a H) (k1^2 - k2^2)(k2^2 - k3^2)(k3^2 - k1^2)   l = 1, 3

(|k1|^2 = p^2 + q^2/4 - p q y, |k2|^2 = p^2 + q^2/4 + p q y.)  The
antisymmetric one pins the odd blocks and the sign convention of y' (a wrong
sign of one recoupled momentum flips those blocks and gives P0 F = -2 F).
Each test also shows that the pin has power: the same check with the
(l, l') factor dropped, the odd blocks negated, or the whole matrix doubled
misses by far more than the tolerance.
"""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss, legval

KMAX = 7.0  # f has decayed to below 1e-13 of its peak there


def _legendre(l, y):
    c = np.zeros(l + 1)
    c[l] = 1.0
    return legval(y, c)


def _k2(p, q, y):
    a = p * p + q * q / 4
    return a - p * q * y, a + p * q * y, q * q


def f_sym4(p, q, y, a):
    k1, k2, k3 = _k2(p, q, y)
    return np.exp(-a * (p * p + 0.75 * q * q)) * (k1 ** 2 + k2 ** 2 + k3 ** 2)


def f_sym8(p, q, y, a):
    k1, k2, k3 = _k2(p, q, y)
    return np.exp(-a * (p * p + 0.75 * q * q)) * (k1 ** 4 + k2 ** 4 + k3 ** 4)


def f_anti(p, q, y, a):
    k1, k2, k3 = _k2(p, q, y)
    return np.exp(-a * (p * p + 0.75 * q * q)) * (k1 - k2) * (k2 - k3) * (k3 - k1)


def cell_projection(f, pe, qe, n_ch, a, ng=8, ny=24):
    """F[l][c] = int_c p^2 dp q^2 dq f_l(p, q) / sqrt(B_i Bq_j), by an ng x ng
    GL rule per cell and an ny-point rule in y (f is a polynomial in y)."""
    t, w = leggauss(ng)
    ty, wy = leggauss(ny)
    N, M = len(pe) - 1, len(qe) - 1
    pm, ph = (pe[1:] + pe[:-1]) / 2, (pe[1:] - pe[:-1]) / 2
    qm, qh = (qe[1:] + qe[:-1]) / 2, (qe[1:] - qe[:-1]) / 2
    P = pm[:, None] + ph[:, None] * t[None, :]
    Q = qm[:, None] + qh[:, None] * t[None, :]
    WP, WQ = ph[:, None] * w[None, :] * P ** 2, qh[:, None] * w[None, :] * Q ** 2
    Bp, Bq = (pe[1:] ** 3 - pe[:-1] ** 3) / 3, (qe[1:] ** 3 - qe[:-1] ** 3) / 3
    F = np.zeros((n_ch, N * M))
    for l in range(n_ch):
        fl = np.zeros((N, ng, M, ng))
        for k in range(ny):
            fl += wy[k] * _legendre(l, ty[k]) * f(P[:, :, None, None], Q[None, None, :, :], ty[k], a)
        I = np.einsum("ia,iajb,jb->ij", WP, fl * np.sqrt(2 * l + 1), WQ)
        F[l] = (I / np.sqrt(np.outer(Bp, Bq))).ravel()
    return F


def apply_P0(orc, P, F, n_ch, mistake=None):
    """(P0 F)[l] = sum_(l, l') P0_(l,l') F[l'] from the oracle's block-CSR;
    `mistake` plants an error in the product (never in the oracle)."""
    rows = np.repeat(np.arange(len(P["row_ptr"]) - 1), np.diff(P["row_ptr"]))
    out = np.zeros_like(F)
    for k, (l, lp) in enumerate(orc.pair_list(n_ch)):
        v = P["val"][:, k]
        if mistake == "no_2l+1":
            v = v / np.sqrt((2 * l + 1) * (2 * lp + 1))
        elif mistake == "odd_sign" and l % 2:
            v = -v
        out[l] += np.bincount(rows, weights=v * F[lp][P["col"]], minlength=F.shape[1])
    return 2.0 * out if mistake == "x2" else out


def block_errors(G, F, ls):
    return {l: np.linalg.norm(G[l] - 2 * F[l]) / np.linalg.norm(2 * F[l]) for l in ls}


def _run(orc, f, n_ch, a, N, nodes, ls, mistake=None, builder=None):
    e = np.linspace(0.0, KMAX, N + 1)
    P = (builder or orc.P0)(e, e, *nodes, n_ch)
    F = cell_projection(f, e, e, n_ch, a)
    for l in range(n_ch):
        if l not in ls:  # no content of this parity: the block product vanishes too
            assert np.abs(F[l]).max() < 1e-12 * np.abs(F).max()
    return block_errors(apply_P0(orc, P, F, n_ch, mistake), F, ls)


def test_symmetric_l0_l2_converges_to_2f(orc):
    coarse = _run(orc, f_sym4, 3, 1.0, 24, (4, 4, 16), (0, 2))
    fine = _run(orc, f_sym4, 3, 1.0, 48, (8, 8, 32), (0, 2))
    assert fine[0] < 1.5e-2 and fine[2] < 4e-2, fine
    # second order in the cell size (measured 3.8x and 4.1x for a halving)
    assert coarse[0] > 2.5 * fine[0] and coarse[2] > 2.5 * fine[2], (coarse, fine)
    # the pin has power: each planted mistake misses by far more
    assert _run(orc, f_sym4, 3, 1.0, 48, (8, 8, 32), (0, 2), "no_2l+1")[2] > 0.5
    assert min(_run(orc, f_sym4, 3, 1.0, 48, (8, 8, 32), (0, 2), "x2").values()) > 0.9


def test_antisymmetric_l1_l3_converges_to_2f(orc):
    """odd partial waves: a totally antisymmetric f is also mapped to 2 f by
    the two cyclic permutations"""
    coarse = _run(orc, f_anti, 4, 1.0, 24, (4, 4, 16), (1, 3))
    fine = _run(orc, f_anti, 4, 1.0, 48, (8, 8, 32), (1, 3))
    assert fine[1] < 3e-2 and fine[3] < 5e-2, fine
    assert coarse[1] > 2.5 * fine[1] and coarse[3] > 2.5 * fine[3], (coarse, fine)
    assert min(_run(orc, f_anti, 4, 1.0, 48, (8, 8, 32), (1, 3), "odd_sign").values()) > 1.9
    assert _run(orc, f_anti, 4, 1.0, 48, (8, 8, 32), (1, 3), "no_2l+1")[3] > 0.5


def test_symmetric_l4_block(orc):
    """l = 4: its cell projection is small next to l = 0, so its block is
    limited by the y nodes; 64 of them"""
    got = _run(orc, f_sym8, 5, 0.5, 64, (8, 8, 64), (0, 2, 4))
    assert got[0] < 5e-3 and got[2] < 1e-2 and got[4] < 0.15, got
    assert _run(orc, f_sym8, 5, 0.5, 64, (8, 8, 64), (0, 2, 4), "no_2l+1")[4] > 0.5


def test_variable_limit_P0_converges_to_2f(orc):
    """The same pin for the variable-limit P0 (y-interval cut at the squared
    bin edges, each piece integrated by GL): symmetric f with l = 0, 2 and
    antisymmetric f with l = 1, 3, second order in the cell size."""
    for f, n_ch, ls in ((f_sym4, 3, (0, 2)), (f_anti, 4, (1, 3))):
        coarse = _run(orc, f, n_ch, 1.0, 24, (4, 4, 8), ls, builder=orc.P0_vl)
        fine = _run(orc, f, n_ch, 1.0, 48, (4, 4, 8), ls, builder=orc.P0_vl)
        for l in ls:
            assert fine[l] < 4e-2 and coarse[l] > 2.5 * fine[l], (l, coarse, fine)
