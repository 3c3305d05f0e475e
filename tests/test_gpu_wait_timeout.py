"""The wait-limit path of the tensor-core GEMMs, exercised on valid input and
without a fault.  A host knob gives the first mbarrier wait of one role a
limit of zero spins: that wait runs out, the CTA raises its abort flag, the
other roles leave at their next wait, the producer still waits (with the
full limit) for every copy it issued and the MMA issuer for every MMA, and
the tensor memory is freed.  The operation must return WPCD_ETIMEOUT, and
the next operation in the same process, with the knob cleared, must give the
same products bit for bit and solves that match the oracle."""
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
    yield wpcd
    wpcd.wpcd_debug_expire_first_wait(0)


def _problem(W, N, M, n_ch=3, V=(-6.0,), a=(1.0,)):
    from paper_1508_07441_gb300 import inputs

    return W.Problem(inputs.tangent_edges(N, 20.0), inputs.tangent_edges(M, 20.0), 4, 4, 16, n_ch, V, a)


def _expect_timeout(W, fn):
    with pytest.raises(W.WpcdError) as ei:
        fn()
    assert ei.value.status == W.WPCD_ETIMEOUT, ei.value


def _gemm(W, pr, mode, which, g, x, B, dtype):
    import torch

    y = torch.full((x.numel(),), float("nan"), dtype=dtype, device="cuda")
    pr.wpcd_channel_gemm(which, mode, g, x, y, B)
    return y


# N = 200: 13 K chunks per tile, more than the raw-chunk ring holds, so the
# producer waits too (role 0); ncol = 2 M B = 256: two column tiles
@pytest.mark.parametrize("role", [0, 1, 2, 3])
def test_tf32x3_gemm_role_times_out_then_recovers(W, role):
    import torch

    pr = _problem(W, 200, 16)
    B = 8
    n = pr.n_ch * pr.N * pr.M * B
    gen = torch.Generator().manual_seed(11 + role)
    x = torch.randn(2 * n, generator=gen, dtype=torch.float32).cuda()
    g = torch.randn(2 * n, generator=gen, dtype=torch.float32).cuda()
    for which, gg in ((0, g), (1, None)):
        ref = _gemm(W, pr, W.WPCD_GEMM_TF32X3, which, gg, x, B, torch.float32)
        assert torch.isfinite(ref).all()
        W.wpcd_debug_expire_first_wait(1, role)
        try:
            _expect_timeout(W, lambda: _gemm(W, pr, W.WPCD_GEMM_TF32X3, which, gg, x, B, torch.float32))
        finally:
            W.wpcd_debug_expire_first_wait(0)
        again = _gemm(W, pr, W.WPCD_GEMM_TF32X3, which, gg, x, B, torch.float32)
        assert torch.equal(again, ref), (role, which)
    pr.close()


def test_digit_plane_gemm_times_out_then_recovers(W):
    import torch

    pr = _problem(W, 130, 20)
    B = 5
    n = pr.n_ch * pr.N * pr.M * B
    gen = torch.Generator().manual_seed(5)
    x = torch.randn(2 * n, generator=gen, dtype=torch.float64).cuda()
    ref = _gemm(W, pr, W.WPCD_GEMM_DIGITS, 1, None, x, B, torch.float64)
    assert torch.isfinite(ref).all()
    W.wpcd_debug_expire_first_wait(2, 0)
    try:
        _expect_timeout(W, lambda: _gemm(W, pr, W.WPCD_GEMM_DIGITS, 1, None, x, B, torch.float64))
    finally:
        W.wpcd_debug_expire_first_wait(0)
    assert torch.equal(_gemm(W, pr, W.WPCD_GEMM_DIGITS, 1, None, x, B, torch.float64), ref)
    pr.close()


def _oracle_U00(orc, pr_args, E):
    pe, qe, nodes, n_ch, V, a = pr_args
    ref_P = orc.P0(pe, qe, *nodes, n_ch)
    opr = orc.Problem(dict(pe=pe, qe=qe, n_p=nodes[0], n_q=nodes[1], n_x=nodes[2], n_ch=n_ch,
                           V=list(V), a=list(a), n_pair_nodes=8), P=ref_P)
    return np.array([opr.solve_gmres(e, tol=1e-13, max_iter=300)["U00"] for e in E])


# (knob kernel, role, solve precision): the warp-specialised GEMM of the FP32
# inner cycles (MMA issuer, epilogue), and the digit-plane GEMM of the
# float-float refinement residual
@pytest.mark.parametrize("kernel,role,prec", [(1, 1, "MIXED_FP64"), (1, 3, "MIXED"), (2, 0, "MIXED")])
def test_solve_times_out_then_matches_oracle(W, orc, kernel, role, prec):
    from paper_1508_07441_gb300 import inputs

    N, M, nodes, n_ch, V, a = 26, 22, (4, 4, 16), 3, (-6.0,), (1.0,)
    pe, qe = inputs.tangent_edges(N, 20.0), inputs.tangent_edges(M, 20.0)
    pr = W.Problem(pe, qe, *nodes, n_ch, V, a)
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    E = [0.7, 2.0]
    precision = getattr(W, "WPCD_SOLVE_" + prec)
    W.wpcd_debug_expire_first_wait(kernel, role)
    try:
        _expect_timeout(W, lambda: pr.wpcd_solve(P, E, tol=1e-12, max_iter=200, precision=precision,
                                                 batch=len(E)))
    finally:
        W.wpcd_debug_expire_first_wait(0)
    U, _, st = pr.wpcd_solve(P, E, tol=1e-12, max_iter=200, precision=precision, batch=len(E))
    assert st == W.WPCD_OK
    ref = _oracle_U00(orc, (pe, qe, nodes, n_ch, V, a), E)
    assert np.all(np.abs(U - ref) <= 1e-8 * np.abs(ref)), (U, ref)
    P.close()
    pr.close()


def test_grouped_solve_times_out_then_matches_oracle(W, orc):
    from paper_1508_07441_gb300 import inputs

    nodes, n_ch, V, a = (4, 4, 16), 3, (-6.0,), (1.0,)
    lattices = [(26, 22), (30, 18)]
    prs, Ps, args = [], [], []
    for N, M in lattices:
        pe, qe = inputs.tangent_edges(N, 20.0), inputs.tangent_edges(M, 20.0)
        pr = W.Problem(pe, qe, *nodes, n_ch, V, a)
        prs.append(pr)
        Ps.append(pr.wpcd_assemble_P(W.WPCD_FP64))
        args.append((pe, qe, nodes, n_ch, V, a))
    Es = [[0.7, 2.0], [1.1, 1.5]]
    W.wpcd_debug_expire_first_wait(1, 3)
    try:
        _expect_timeout(W, lambda: W.wpcd_solve_batch(prs, Ps, Es, tol=1e-12, max_iter=200,
                                                      precision=W.WPCD_SOLVE_MIXED_FP64))
    finally:
        W.wpcd_debug_expire_first_wait(0)
    Us, _, st = W.wpcd_solve_batch(prs, Ps, Es, tol=1e-12, max_iter=200, precision=W.WPCD_SOLVE_MIXED_FP64)
    assert st == W.WPCD_OK
    for U, E, arg in zip(Us, Es, args):
        ref = _oracle_U00(orc, arg, E)
        assert np.all(np.abs(U - ref) <= 1e-8 * np.abs(ref)), (U, ref)
    for x in Ps + prs:
        x.close()
