"""GPU parity of the variable-limit P0 (Sec. 3.2: the element as an integral
with variable limits, WPCD_FP64_VL) against the oracle's, element by element
on the same lattices: the pattern exactly (the limits are IEEE divisions of
identically rounded values on both sides), values to rel 1e-10 of each
element plus 1e-13 of its row's largest; bit-reproducible; and a solve on
the variable-limit P0 matching the oracle's solve on its own."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07441_gb300 import build, wpcd

    build.build()
    return wpcd


def _edges(N, M, jitter):
    from paper_1508_07441_gb300 import inputs

    if jitter is None:
        return inputs.tangent_edges(N, 20.0), inputs.tangent_edges(M, 20.0)
    return inputs.jittered_edges(N, 20.0, jitter), inputs.jittered_edges(M, 20.0, jitter + 1)


def _check_vl(W, orc, pe, qe, nodes, n_ch):
    N, M = len(pe) - 1, len(qe) - 1
    grid = W.Grid(pe, qe, *nodes)
    P = grid.wpcd_assemble_P(n_ch, W.WPCD_FP64_VL)
    rp, col, val = P.wpcd_P_export()
    ref = orc.P0_vl(pe, qe, *nodes, n_ch)
    assert np.array_equal(rp, ref["row_ptr"])
    assert np.array_equal(col, ref["col"])
    rows = np.repeat(np.arange(N * M), np.diff(rp))
    rowmax = np.zeros(N * M)
    np.maximum.at(rowmax, rows, np.abs(ref["val"]).max(axis=1))
    bar = 1e-10 * np.abs(ref["val"]) + 1e-13 * rowmax[rows][:, None]
    assert np.all(np.abs(val.T - ref["val"]) <= bar), np.max(np.abs(val.T - ref["val"]) / bar)
    again = grid.wpcd_assemble_P(n_ch, W.WPCD_FP64_VL).wpcd_P_export()
    assert all(np.array_equal(x, y) for x, y in zip((rp, col, val), again))
    return np.diff(rp).max()


@pytest.mark.parametrize("N,M,nodes,n_ch,jit", [(20, 16, (4, 4, 8), 1, None), (12, 14, (3, 5, 6), 3, None),
                                               (17, 23, (4, 6, 5), 2, 11), (26, 22, (8, 8, 8), 5, 21)])
def test_vl_assembly_matches_oracle(W, orc, N, M, nodes, n_ch, jit):
    pe, qe = _edges(N, M, jit)
    _check_vl(W, orc, pe, qe, nodes, n_ch)


def test_vl_assembly_fine_lattice(W, orc):
    """150 x 150 bins, 8 x 8 nodes: up to about 9000 (node, target) pieces
    per source cell, which the row's hash set of distinct targets (about
    300) absorbs"""
    from paper_1508_07441_gb300 import inputs

    pe = inputs.tangent_edges(150, 20.0)
    assert _check_vl(W, orc, pe, pe, (8, 8, 2), 1) > 250


def test_vl_assembly_row_beyond_first_hash_size(W, orc):
    """60 fine bins and one coarse outer bin, 16 x 16 nodes: the coarse cells'
    rows hold about 530 targets, more than the first hash set of 4 (N + M)
    slots takes (384 = 3/4 of 512), so the row pass runs again with twice
    the slots"""
    pe = np.concatenate([np.linspace(0.0, 4.0, 61), [8.0]])
    assert _check_vl(W, orc, pe, pe, (16, 16, 2), 1) > 384


def test_vl_solve_matches_oracle(W, orc):
    pe, qe = _edges(24, 22, None)
    nodes, n_ch, V, a = (4, 4, 8), 3, (-6.0,), (1.0,)
    grid = W.Grid(pe, qe, *nodes)
    P = grid.wpcd_assemble_P(n_ch, W.WPCD_FP64_VL)
    pr = grid.wpcd_pair_create(V, a, n_ch)
    opr = orc.Problem(dict(pe=pe, qe=qe, n_p=nodes[0], n_q=nodes[1], n_x=nodes[2], n_ch=n_ch, V=list(V),
                           a=list(a), n_pair_nodes=8), P=orc.P0_vl(pe, qe, *nodes, n_ch))
    E = [0.5 * pr.eps_bound, 0.7, 2.5]
    for prec in (W.WPCD_SOLVE_FP64, W.WPCD_SOLVE_MIXED):
        U, stats, st = pr.wpcd_solve(P, E, tol=1e-12, max_iter=200, precision=prec, batch=len(E))
        assert st == W.WPCD_OK
        for k, e in enumerate(E):
            ref = opr.solve_gmres(e, tol=1e-13, max_iter=300)["U00"]
            assert abs(U[k] - ref) <= 1e-8 * abs(ref), (prec, e)
    # below breakup the S-matrix of the variable-limit system is unitary too
    assert abs(abs(complex(*stats[0].S)) - 1.0) < 1e-9
