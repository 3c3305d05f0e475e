"""GPU checks of the FP64-class channel-block products built from bf16 digit
planes on the tensor cores (wpcd_channel_gemm mode WPCD_GEMM_DIGITS, through
the C ABI) against FP64 numpy products of the same blocks: one and two
128-row tiles, ragged K chunks (N not a multiple of 16), ragged column tiles,
columns of very different magnitude (per-column exponents), a zero block,
and the N limit; then the mixed solve, whose residual and Born-term products
take this path, against the FP64 oracle and against the float-float SIMT
products."""
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


def _problem(W, N, M, n_ch=3):
    from paper_1508_07441_gb300 import inputs

    return W.Problem(inputs.tangent_edges(N, 20.0), inputs.tangent_edges(M, 20.0), 2, 2, 4, n_ch,
                     (-3.0,), (1.0,))


def _blocks(pr, which):
    out = []
    for l in range(pr.n_ch):
        eps, O, v = pr.wpcd_problem_pair(l)
        out.append(O if which == 1 else v @ O.T)  # Vt = v O^T
    return np.stack(out)


def _run(W, pr, which, x, g, B):
    import torch

    n = x.size
    y = torch.full((2 * n,), float("nan"), dtype=torch.float64, device="cuda")
    ms = pr.wpcd_channel_gemm(which, W.WPCD_GEMM_DIGITS,
                              None if g is None else torch.from_numpy(g.view(np.float64)).cuda(),
                              torch.from_numpy(x.view(np.float64)).cuda(), y, B, timed=True)
    assert ms > 0.0
    return y.cpu().numpy().view(np.complex128)


# (N, M, B): one row tile with three K chunks; two row tiles, N = 130 (the
# second tile two rows deep, the last K chunk two deep); N = 200 (the bench
# lattice's row count: 13 K chunks); N = 256 (the limit, full tiles); M B odd
# (ncol = 2 M B not a multiple of the 32-column tile)
@pytest.mark.parametrize("N,M,B", [(40, 12, 3), (130, 20, 5), (200, 16, 8), (256, 6, 4), (17, 7, 1)])
@pytest.mark.parametrize("which", [0, 1])
def test_digit_gemm_matches_fp64(W, N, M, B, which):
    """Error against the FP64 product below 5e-14 of the magnitude sum
    sum_k |a_ik| |x'_kj|: the float-float panel itself holds each FP64
    value to 2^-48 relative, the digit planes keep 56 bits below the row and
    column scales, the tensor sums are exact and the combination is one FP64
    sum (measured: 7e-15 at most)."""
    from paper_1508_07441_gb300 import inputs

    pr = _problem(W, N, M)
    n = pr.n_ch * N * M * B
    x = inputs.random_complex(n, 11)
    g = inputs.random_complex(n, 12) if which == 0 else None
    A = _blocks(pr, which)
    xc = x.reshape(pr.n_ch, N, M * B)
    if g is not None:
        xc = xc * g.reshape(pr.n_ch, N, M * B)
    ref = np.einsum("cik,ckj->cij", A, xc)
    scale = np.einsum("cik,ckj->cij", np.abs(A), np.abs(xc))
    got = _run(W, pr, which, x, g, B).reshape(ref.shape)
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref) / scale
    assert err.max() < 5e-14, err.max()


def test_digit_gemm_column_scales_and_zero_block(W):
    """Columns whose magnitudes span 2^-60 .. 2^60 (each gets its own
    exponent, so each keeps its full relative accuracy) and an all-zero
    channel block (exponent 0, digits 0, output exactly 0)."""
    from paper_1508_07441_gb300 import inputs

    N, M, B = 64, 10, 4
    pr = _problem(W, N, M)
    n = pr.n_ch * N * M * B
    x = inputs.random_complex(n, 13).reshape(pr.n_ch, N, M * B)
    cols = np.exp2(np.linspace(-60.0, 60.0, M * B))
    x = x * cols[None, None, :]
    x[1] = 0.0
    x = np.ascontiguousarray(x).reshape(-1)
    A = _blocks(pr, 1)
    xc = x.reshape(pr.n_ch, N, M * B)
    ref = np.einsum("cik,ckj->cij", A, xc)
    scale = np.einsum("cik,ckj->cij", np.abs(A), np.abs(xc))
    got = _run(W, pr, 1, x, None, B).reshape(ref.shape)
    assert np.all(got[1] == 0.0)
    live = scale > 0
    assert np.max(np.abs(got - ref)[live] / scale[live]) < 5e-14


def test_digit_gemm_rejects_large_n(W):
    import torch

    pr = _problem(W, 257, 4, n_ch=1)
    x = torch.zeros(2 * pr.dim, dtype=torch.float64, device="cuda")
    with pytest.raises(W.WpcdError, match="N <= 256"):
        pr.wpcd_channel_gemm(1, W.WPCD_GEMM_DIGITS, None, x, x.clone(), 1)


@pytest.mark.parametrize("residual", ["digits", "ff"])
def test_mixed_solve_with_either_residual_product(W, orc, monkeypatch, residual):
    """The batched mixed solve with its refinement residual and Born term
    from the digit-plane products (default) or the float-float SIMT products
    (WPCD_RESIDUAL_GEMM=ff): both refine to the residual tolerance 1e-12,
    U00 within 1e-8 of the oracle, and the two agree to 1e-9."""
    from paper_1508_07441_gb300 import inputs

    if residual == "ff":
        monkeypatch.setenv("WPCD_RESIDUAL_GEMM", "ff")
    else:
        monkeypatch.delenv("WPCD_RESIDUAL_GEMM", raising=False)
    pe, qe = inputs.tangent_edges(30, 20.0), inputs.tangent_edges(28, 20.0)
    pr = W.Problem(pe, qe, 4, 4, 16, 3, (-6.0,), (1.0,))
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    E = [-0.3, 0.25, 0.9, 2.0, 4.5]
    U, stats, st = pr.wpcd_solve(P, E, tol=1e-12, precision=W.WPCD_SOLVE_MIXED, batch=len(E))
    assert st == W.WPCD_OK and all(s.relres <= 1e-12 for s in stats)
    opr = orc.Problem(dict(pe=pe, qe=qe, n_p=4, n_q=4, n_x=16, n_ch=3, V=[-6.0], a=[1.0], n_pair_nodes=8))
    ref = np.array([opr.solve_gmres(e, tol=1e-13, max_iter=300)["U00"] for e in E])
    assert np.max(np.abs(U - ref) / np.abs(ref)) < 1e-8
    _mixed_cache[residual] = np.asarray(U)
    if len(_mixed_cache) == 2:
        a, b = _mixed_cache["digits"], _mixed_cache["ff"]
        assert np.max(np.abs(a - b) / np.abs(b)) < 1e-9


_mixed_cache = {}
