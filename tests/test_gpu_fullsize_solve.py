"""GPU parity of the batched mixed solve at the full bench workload: the
3-channel 200 x 200 lattice (8x8x32 nodes per cell, dimension 120 000) with
the bench's 128 energies in one batch on a side stream (FP32 inner cycles on
the tensor cores from a CUDA graph, FP64-class residual from digit planes,
tolerance 1e-10); every energy against the FP64 oracle's own Krylov solve.
G1 and the Born term depend on an energy only through its on-shell q-bin,
so the oracle's U00 is one value per bin: one oracle solve per distinct bin
(30 for these 128 energies) checks all 128."""
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


def test_full_size_batch_matches_oracle(W, orc):
    import torch
    from paper_1508_07441_gb300 import inputs

    w = inputs.workload("bosons3_200")
    pr = W.Problem(w["p_edges"], w["q_edges"], *w["nodes"], w["n_ch"], w["V"], w["a"], n_pair_nodes=8)
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    E = [float(x) for x in inputs.batch_energies(pr.eps_bound, 128)]
    stream = torch.cuda.Stream()
    U, stats, st = pr.wpcd_solve(P, E, precision=W.WPCD_SOLVE_MIXED, tol=1e-10, batch=len(E), stream=stream)
    assert st == W.WPCD_OK
    assert max(s.relres for s in stats) <= 1e-10
    opr = orc.Problem(dict(pe=w["p_edges"], qe=w["q_edges"], n_p=w["nodes"][0], n_q=w["nodes"][1],
                           n_x=w["nodes"][2], n_ch=w["n_ch"], V=list(w["V"]), a=list(w["a"]), n_pair_nodes=8))
    j0 = [orc.onshell(w["q_edges"], e, opr.eps_b)[0] for e in E]
    first = {}
    for k, j in enumerate(j0):
        first.setdefault(j, k)
    assert len(first) == 30
    ref = {j: opr.solve_gmres(E[k], tol=1e-12, max_iter=300)["U00"] for j, k in first.items()}
    for k, j in enumerate(j0):
        assert stats[k].j0 == j, k
        assert abs(U[k] - ref[j]) <= 1e-6 * abs(ref[j]), (k, U[k], ref[j])
    P.close()
    pr.close()
