"""GPU parity of the grouped solve over problems of uneven grid size
(wpcd_solve_batch, through the C ABI) against the FP64 oracle: every
(problem, energy) amplitude within rel 1e-6 of the oracle's own GMRES solve of
the same discretised equation, the same results as one wpcd_solve per problem,
identical results with and without CUDA-graph replay, and argument checks."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NODES = (4, 4, 16)
V, A = (-6.0,), (1.0,)


@pytest.fixture(scope="module")
def W():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07441_gb300 import build, wpcd

    build.build()
    return wpcd


def _make(W, orc, N, M, n_ch=3, prec=None):
    from paper_1508_07441_gb300 import inputs

    pe, qe = inputs.tangent_edges(N, 20.0), inputs.tangent_edges(M, 20.0)
    pr = W.Problem(pe, qe, *NODES, n_ch, V, A)
    P = pr.wpcd_assemble_P(W.WPCD_FP64 if prec is None else prec)
    opr = orc.Problem(dict(pe=pe, qe=qe, n_p=NODES[0], n_q=NODES[1], n_x=NODES[2], n_ch=n_ch,
                           V=list(V), a=list(A), n_pair_nodes=8))
    return pr, P, opr


@pytest.fixture(scope="module")
def group(W, orc):
    """Four problems of different grids (ragged against the 32 x 64 GEMM
    tiles and the warp row layout), 1 to 5 energies each."""
    shapes = [(14, 12), (22, 25), (31, 30), (18, 17)]
    energies = [[0.7], [-0.3, 1.1, 3.0], [-0.5, 0.1, 0.6, 2.2, 4.4], [0.25, 1.9]]
    items = [_make(W, orc, N, M) for N, M in shapes]
    return items, energies


def _oracle(opr, E):
    return np.array([opr.solve_gmres(e, tol=1e-13, max_iter=400)["U00"] for e in E])


def test_group_fp64_matches_oracle(W, group):
    items, energies = group
    U, stats, st = W.wpcd_solve_batch([i[0] for i in items], [i[1] for i in items], energies,
                                      tol=1e-12, max_iter=300, check_every=1)
    assert st == W.WPCD_OK
    for (pr, P, opr), E, u, sl in zip(items, energies, U, stats):
        ref = _oracle(opr, E)
        assert np.max(np.abs(u - ref) / np.abs(ref)) < 1e-9
        for s, e in zip(sl, E):
            assert s.status == W.WPCD_OK and s.relres <= 1e-12
            S_ref, A_ref = opr.amplitudes(e, s.U00[0] + 1j * s.U00[1])
            assert abs(complex(*s.S) - S_ref) < 1e-12 and abs(complex(*s.A) - A_ref) < 1e-12 * abs(A_ref)
            if e < 0:  # below breakup the elastic S-matrix is unitary
                assert abs(abs(complex(*s.S)) - 1.0) < 1e-8


@pytest.mark.parametrize("resid", ["MIXED", "MIXED_FP64"])
@pytest.mark.parametrize("prec", ["FP64", "FP32C"])
def test_group_mixed_matches_oracle(W, orc, group, prec, resid):
    """Both refinement residuals: float-float (WPCD_SOLVE_MIXED) and native
    FP64 (WPCD_SOLVE_MIXED_FP64)."""
    items, energies = group
    if prec == "FP32C":
        items = [(pr, pr.wpcd_assemble_P(W.WPCD_FP32C), opr) for pr, _, opr in items]
    U, stats, st = W.wpcd_solve_batch([i[0] for i in items], [i[1] for i in items], energies,
                                      tol=1e-12, precision=getattr(W, "WPCD_SOLVE_" + resid))
    assert st == W.WPCD_OK
    worst = 0.0
    for (pr, P, opr), E, u, sl in zip(items, energies, U, stats):
        for s in sl:
            assert s.status == W.WPCD_OK and s.relres <= 1e-12 and s.n_kapply32 >= 10
        worst = max(worst, np.max(np.abs(u - _oracle(opr, E)) / np.abs(_oracle(opr, E))))
    # FP64 values: the FP64 system refined to residual 1e-12 (1e-8 with the
    # conditioning of about 1e2 as margin); FP32C values: the
    # FP32-valued P0 shifts U00 by its node-evaluation error (the same bar as
    # the single-problem mixed solve)
    assert worst < (1e-8 if prec == "FP64" else 2e-5), worst


def test_group_float_float_odd_segment_offsets(W, orc):
    """Segments that start on an odd complex element (n_ch N M B odd), so
    the float-float block products of the later problems read panels that
    are only 8-byte aligned; float-float residual against the oracle."""
    shapes = [(13, 11), (15, 9), (20, 16)]
    energies = [[0.3, 1.7, 2.9], [0.9], [-0.4, 2.2]]
    items = [_make(W, orc, N, M) for N, M in shapes]
    U, stats, st = W.wpcd_solve_batch([i[0] for i in items], [i[1] for i in items], energies,
                                      tol=1e-12, precision=W.WPCD_SOLVE_MIXED)
    assert st == W.WPCD_OK
    for (pr, P, opr), E, u, sl in zip(items, energies, U, stats):
        assert all(s.status == W.WPCD_OK and s.relres <= 1e-12 for s in sl)
        ref = _oracle(opr, E)
        assert np.max(np.abs(u - ref) / np.abs(ref)) < 1e-8


def test_group_tensor_core_products(W, orc, monkeypatch):
    """An even group (every batch even, so every segment is 16-byte aligned)
    runs its FP32 block products as one grouped tensor-core launch each, over
    problems of one and two 128-row tiles; the amplitudes match the oracle
    and the same group with the SIMT products (WPCD_GEMM=simt)."""
    shapes = [(130, 20), (40, 36), (90, 70)]
    energies = [[0.4, 2.6], [-0.2, 0.8, 1.5, 3.9], [0.3, 1.1, 2.0, 2.7, 3.3, 4.6]]
    items = [_make(W, orc, N, M) for N, M in shapes]
    args = ([i[0] for i in items], [i[1] for i in items], energies)
    U, stats, st = W.wpcd_solve_batch(*args, tol=1e-12, precision=W.WPCD_SOLVE_MIXED)
    assert st == W.WPCD_OK
    monkeypatch.setenv("WPCD_GEMM", "simt")
    Us, _, st2 = W.wpcd_solve_batch(*args, tol=1e-12, precision=W.WPCD_SOLVE_MIXED)
    assert st2 == W.WPCD_OK
    for (pr, P, opr), E, u, us, sl in zip(items, energies, U, Us, stats):
        assert all(s.status == W.WPCD_OK and s.relres <= 1e-12 for s in sl)
        ref = _oracle(opr, E)
        assert np.max(np.abs(u - ref) / np.abs(ref)) < 1e-8
        assert np.max(np.abs(u - us) / np.abs(us)) < 1e-9


def test_group_equals_per_problem_solves(W, group):
    items, energies = group
    U, _, _ = W.wpcd_solve_batch([i[0] for i in items], [i[1] for i in items], energies,
                                 tol=1e-12, max_iter=300)
    for (pr, P, _), E, u in zip(items, energies, U):
        u1, _, _ = pr.wpcd_solve(P, E, tol=1e-12, max_iter=300)
        assert np.max(np.abs(u - u1) / np.abs(u1)) < 1e-10


def test_group_graph_and_eager_identical(W, group):
    import torch

    items, energies = group
    args = ([i[0] for i in items], [i[1] for i in items], energies)
    Ug, _, _ = W.wpcd_solve_batch(*args, precision=W.WPCD_SOLVE_MIXED, use_graph=1,
                                  stream=torch.cuda.Stream())
    Ue, _, _ = W.wpcd_solve_batch(*args, precision=W.WPCD_SOLVE_MIXED, use_graph=0)
    for a, b in zip(Ug, Ue):
        assert np.array_equal(a, b)


def test_group_of_sixteen_uneven_grids(W, orc):
    """The batching workload's shape: 16 problems with N = M drawn from
    [40, 160] (seed 1234), 8 seeded energies each, 3 channels; every energy
    converges and one energy per problem is checked against the oracle."""
    from paper_1508_07441_gb300 import inputs

    sizes = inputs.uneven_sizes(16, 40, 160, 1234)
    items = [_make(W, orc, int(n), int(n)) for n in sizes]
    energies = [inputs.random_energies(abs(opr.eps_b), 8, 5000 + g) for g, (_, _, opr) in enumerate(items)]
    U, stats, st = W.wpcd_solve_batch([i[0] for i in items], [i[1] for i in items], energies,
                                      tol=1e-10, precision=W.WPCD_SOLVE_MIXED)
    assert st == W.WPCD_OK
    assert all(s.status == W.WPCD_OK for sl in stats for s in sl)
    for g, ((pr, P, opr), E, u) in enumerate(zip(items, energies, U)):
        k = g % 8
        ref = opr.solve_gmres(E[k], tol=1e-12, max_iter=400)["U00"]
        assert abs(u[k] - ref) / abs(ref) < 1e-6


def test_group_rejects_bad_arguments(W, orc, group):
    items, energies = group
    prs, Ps = [i[0] for i in items], [i[1] for i in items]
    one_ch = _make(W, orc, 12, 12, n_ch=1)
    with pytest.raises(W.WpcdError, match="channel count"):
        W.wpcd_solve_batch(prs[:1] + [one_ch[0]], Ps[:1] + [one_ch[1]], energies[:2])
    with pytest.raises(W.WpcdError, match="WPCD_GROUP_MAX_E"):
        W.wpcd_solve_batch(prs[:1], Ps[:1], [np.linspace(0.1, 2.0, 33)])
    with pytest.raises(W.WpcdError, match="another lattice"):
        W.wpcd_solve_batch(prs[:2], [Ps[1], Ps[0]], energies[:2])
    with pytest.raises(W.WpcdError, match="dimer threshold"):
        W.wpcd_solve_batch(prs[:1], Ps[:1], [[-50.0]])
