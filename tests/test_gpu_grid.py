"""The boundary split into grid, pair and P0 (Sec. 3.3: P0 depends on the
lattice only and is computed once for many potentials and energies): one P0
assembled on a grid serves problems with different potentials on that grid,
each solve matching the oracle; a P0 is refused for another grid or channel
count; handles outlive the caller's grid reference."""
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


POTS = [((-6.0,), (1.0,)), ((-8.0, 2.0), (1.0, 0.25))]


def test_one_P0_two_potentials(W, orc):
    from paper_1508_07441_gb300 import inputs

    N, M, nodes, n_ch = 26, 22, (4, 4, 16), 3
    pe, qe = inputs.tangent_edges(N, 20.0), inputs.tangent_edges(M, 20.0)
    grid = W.Grid(pe, qe, *nodes)
    P = grid.wpcd_assemble_P(n_ch)
    # the same P0 as a problem's own assembly, bit for bit
    own = W.Problem(pe, qe, *nodes, n_ch, *POTS[0])
    for x, y in zip(P.wpcd_P_export(), own.wpcd_assemble_P(W.WPCD_FP64).wpcd_P_export()):
        assert np.array_equal(x, y)
    ref_P = orc.P0(pe, qe, *nodes, n_ch)
    probs = [grid.wpcd_pair_create(V, a, n_ch) for V, a in POTS]
    grid.close()  # the problems and P0 keep the lattice alive
    E = [0.7, 2.0]
    Us = []
    for pr, (V, a) in zip(probs, POTS):
        assert pr.eps_bound < 0.0
        for prec in (W.WPCD_SOLVE_FP64, W.WPCD_SOLVE_MIXED):
            U, stats, st = pr.wpcd_solve(P, E, tol=1e-12, max_iter=200, precision=prec, batch=len(E))
            assert st == W.WPCD_OK
            opr = orc.Problem(dict(pe=pe, qe=qe, n_p=nodes[0], n_q=nodes[1], n_x=nodes[2], n_ch=n_ch,
                                   V=list(V), a=list(a), n_pair_nodes=8), P=ref_P)
            for k, e in enumerate(E):
                ref = opr.solve_gmres(e, tol=1e-13, max_iter=300)["U00"]
                assert abs(U[k] - ref) <= 1e-8 * abs(ref), (V, prec, e)
        Us.append(U)
    assert np.max(np.abs(Us[0] - Us[1])) > 1e-3 * np.max(np.abs(Us[0]))  # two different systems
    for pr in probs:
        pr.close()
    P.close()


def test_P0_refused_for_other_grid_or_channels(W):
    from paper_1508_07441_gb300 import inputs

    pe = inputs.tangent_edges(20, 20.0)
    g1, g2 = W.Grid(pe, pe, 4, 4, 16), W.Grid(pe, pe, 4, 4, 16)
    P = g1.wpcd_assemble_P(3)
    other = g2.wpcd_pair_create((-6.0,), (1.0,), 3)
    fewer = g1.wpcd_pair_create((-6.0,), (1.0,), 2)
    for pr in (other, fewer):
        with pytest.raises(W.WpcdError) as ei:
            pr.wpcd_solve(P, [0.7])
        assert ei.value.status == W.WPCD_EINVAL
    same = g1.wpcd_pair_create((-6.0,), (1.0,), 3)
    U, _, st = same.wpcd_solve(P, [0.7])
    assert st == W.WPCD_OK and np.isfinite(U[0])
