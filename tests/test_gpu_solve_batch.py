"""GPU parity of the batched and mixed-precision solves (through the C ABI)
against the FP64 oracle: amplitudes rel 1e-6, residuals at the requested
FP64 tolerance, identical results with and without CUDA-graph replay."""
import os

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


@pytest.fixture(scope="module")
def sys3(W, orc):
    """3-channel system, 30 x 28 lattice, 4x4x16 nodes, V = -6 exp(-r^2)."""
    from paper_1508_07441_gb300 import inputs

    pe, qe = inputs.tangent_edges(30, 20.0), inputs.tangent_edges(28, 20.0)
    pr = W.Problem(pe, qe, 4, 4, 16, 3, (-6.0,), (1.0,))
    P64 = pr.wpcd_assemble_P(W.WPCD_FP64)
    P32 = pr.wpcd_assemble_P(W.WPCD_FP32C)
    opr = orc.Problem(dict(pe=pe, qe=qe, n_p=4, n_q=4, n_x=16, n_ch=3, V=[-6.0], a=[1.0],
                           n_pair_nodes=8))
    return pr, P64, P32, opr


ENERGIES = [-0.3, 0.25, 0.9, 2.0, 4.5]


def _ref(opr, E):
    return np.array([opr.solve_gmres(e, tol=1e-13, max_iter=300)["U00"] for e in E])


def test_batched_fp64_matches_oracle(W, sys3):
    pr, P64, _, opr = sys3
    U, stats, st = pr.wpcd_solve(P64, ENERGIES, tol=1e-12, max_iter=200, batch=len(ENERGIES))
    assert st == W.WPCD_OK
    ref = _ref(opr, ENERGIES)
    assert np.max(np.abs(U - ref) / np.abs(ref)) < 1e-9
    # one batch of 5 applies K to all five energies at once; each energy
    # reports its own count of steps to the tolerance (+ the Born term)
    assert all(2 <= s.n_kapply <= 201 for s in stats)


@pytest.mark.parametrize("residual", ["float-float", "fp64"])
@pytest.mark.parametrize("pname", ["P64", "P32"])
def test_mixed_matches_oracle(W, sys3, pname, residual):
    """Both refinement residuals (float-float on the FP32 pipe, native
    FP64) reach the FP64 tolerance and the oracle's U00."""
    pr, P64, P32, opr = sys3
    P = P64 if pname == "P64" else P32
    prec = W.WPCD_SOLVE_MIXED if residual == "float-float" else W.WPCD_SOLVE_MIXED_FP64
    U, stats, st = pr.wpcd_solve(P, ENERGIES, tol=1e-12, precision=prec, batch=len(ENERGIES))
    assert st == W.WPCD_OK
    for s in stats:
        assert s.status == W.WPCD_OK and s.relres <= 1e-12
        assert s.n_outer >= 1 and s.n_kapply32 >= 10
    ref = _ref(opr, ENERGIES)
    err = np.max(np.abs(U - ref) / np.abs(ref))
    # FP64 values: refined to the FP64 system at residual 1e-12; the U00
    # error is the residual times the conditioning of (I - K), about 1e2 on
    # this strongly bound system, so 1e-8 holds with margin (at residual
    # 1e-10 it sat at the bar); FP32C values: the refinement converges to the FP32C-valued
    # system, whose U00 differs from the FP64 one by the FP32 node-evaluation
    # error of P0 amplified by the conditioning (6e-6 measured on this
    # strongly bound test system; stated, not hidden)
    assert err < (1e-8 if pname == "P64" else 2e-5), err


def test_mixed_graph_and_eager_identical(W, sys3):
    pr, P64, _, _ = sys3
    Ug, sg, _ = pr.wpcd_solve(P64, ENERGIES, precision=W.WPCD_SOLVE_MIXED, use_graph=1,
                              stream=__import__("torch").cuda.Stream())
    Ue, se, _ = pr.wpcd_solve(P64, ENERGIES, precision=W.WPCD_SOLVE_MIXED, use_graph=0)
    assert np.array_equal(Ug, Ue)
    assert [s.n_outer for s in sg] == [s.n_outer for s in se]


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_energies_sharing_on_shell_bins(W, sys3, precision):
    """Energies that share on-shell bins (out of order): G1 and the Born term
    are formed once per bin; every energy matches the oracle, and energies of
    one bin, whose discretised equation is the same, give the same U00."""
    pr, P64, _, opr = sys3
    E = [0.9, 0.9001, 2.0, 0.8995, 2.0002, -0.3]
    U, stats, st = pr.wpcd_solve(P64, E, tol=1e-12, max_iter=300, batch=len(E),
                                 precision=getattr(W, "WPCD_SOLVE_" + precision))
    assert st == W.WPCD_OK
    j0 = [s.j0 for s in stats]
    assert len(set(j0)) < len(E)
    ref = np.array([opr.solve_gmres(e, tol=1e-13, max_iter=400)["U00"] for e in E])
    assert np.max(np.abs(U - ref) / np.abs(ref)) < 1e-9
    for a in range(len(E)):
        for b in range(len(E)):
            if j0[a] == j0[b]:
                assert abs(U[a] - U[b]) <= 1e-11 * abs(U[a])


def test_batch_of_128_energies(W, orc):
    """The batching workload's energy grid (128 energies uniform in
    [-0.9 |E_d|, 5]) solved in one batch, mixed precision, on a 3-channel
    lattice; a sample of energies checked against the oracle."""
    from paper_1508_07441_gb300 import inputs

    pe, qe = inputs.tangent_edges(36, 20.0), inputs.tangent_edges(36, 20.0)
    pr = W.Problem(pe, qe, 4, 4, 16, 3, (-3.0,), (1.0,))
    P = pr.wpcd_assemble_P(W.WPCD_FP32C)
    E = inputs.batch_energies(pr.eps_bound, 128)
    U, stats, st = pr.wpcd_solve(P, E, precision=W.WPCD_SOLVE_MIXED, batch=128, tol=1e-10)
    assert st == W.WPCD_OK and all(s.status == W.WPCD_OK for s in stats)
    opr = orc.Problem(dict(pe=pe, qe=qe, n_p=4, n_q=4, n_x=16, n_ch=3, V=[-3.0], a=[1.0],
                           n_pair_nodes=8))
    for k in [0, 1, 40, 90, 127]:
        ref = opr.solve_gmres(E[k], tol=1e-13, max_iter=400)["U00"]
        assert abs(U[k] - ref) / abs(ref) < 1e-6, (k, E[k])


def test_solution_vectors_and_warm_start(W, sys3):
    import torch

    pr, P64, _, opr = sys3
    E = [0.9, 2.0]
    u = torch.zeros(2 * len(E) * pr.dim, dtype=torch.float64, device="cuda")
    U, s1, _ = pr.wpcd_solve(P64, E, tol=1e-12, max_iter=200, u_out=u)
    for k, e in enumerate(E):
        ref = opr.solve_gmres(e, tol=1e-13, max_iter=300)["u"]
        got = u[2 * k * pr.dim:2 * (k + 1) * pr.dim].cpu().numpy().view(np.complex128)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-9
    # restarting from the solution needs no Krylov step
    U2, s2, st = pr.wpcd_solve(P64, E, tol=1e-10, max_iter=200, u_init=u)
    assert st == W.WPCD_OK
    assert all(s.n_kapply <= 2 for s in s2)  # Born term + one residual
    assert np.max(np.abs(U2 - U) / np.abs(U)) < 1e-10
    # the mixed solve from the same warm start needs no refinement cycle
    U3, s3, st = pr.wpcd_solve(P64, E, tol=1e-10, precision=W.WPCD_SOLVE_MIXED, u_init=u)
    assert st == W.WPCD_OK and all(s.n_outer == 0 for s in s3)


def test_autotuner(W, sys3, tmp_path, monkeypatch):
    pr, P64, P32, _ = sys3
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("WPCD_TUNE_CACHE", str(cache))
    for B in (1, 3, 8, 64):
        for mode, P in ((W.WPCD_SPMM_FP64, P64), (W.WPCD_SPMM_FP32, P32), (W.WPCD_SPMM_FF, P64)):
            rpw, el, ept = pr.wpcd_tune_spmm(P, B, mode=mode)
            tiled = mode == W.WPCD_SPMM_FP32 and el == 32 and rpw in (2, 4)  # the row-tiled kernel
            assert tiled or (rpw * el <= 32 and 32 % (rpw * el) == 0)
            assert ept in (1, 2, 4)
            if B == 1:
                assert el == 1
    assert cache.exists() and len(cache.read_text().splitlines()) >= 1


def test_invalid_solve_options(W, sys3):
    pr, P64, _, _ = sys3
    with pytest.raises(W.WpcdError):
        pr.wpcd_solve(P64, [1.0], method=W.WPCD_SUM_WYNN, precision=W.WPCD_SOLVE_MIXED)
    with pytest.raises(W.WpcdError):
        pr.wpcd_solve(P64, [1.0], batch=5000)
    with pytest.raises(W.WpcdError):
        pr.wpcd_solve(P64, [1.0], inner_iter=500)
