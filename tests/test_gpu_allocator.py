"""The caller's device allocator (wpcd_set_allocator, through the C ABI):
with PyTorch's caching allocator installed, problem tables, P0 and the
solves' work space come from PyTorch (its allocated bytes grow while the
handles live and return when they are destroyed), and the amplitudes are
identical to those with the library's own allocator."""
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


def _run(W, E):
    from paper_1508_07441_gb300 import inputs

    pe, qe = inputs.tangent_edges(30, 20.0), inputs.tangent_edges(26, 20.0)
    pr = W.Problem(pe, qe, 4, 4, 16, 3, (-6.0,), (1.0,))
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    U, stats, st = pr.wpcd_solve(P, E, tol=1e-12, batch=len(E), precision=W.WPCD_SOLVE_MIXED)
    assert st == W.WPCD_OK
    return pr, P, U


def test_torch_allocator(W):
    import gc

    import torch

    gc.collect()  # handles of earlier tests, if any, are destroyed first
    E = [0.4, 1.3, 2.7, 4.1]
    pr, P, U_own = _run(W, E)
    P.close()
    pr.close()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    W.use_torch_allocator()
    try:
        pr, P, U_torch = _run(W, E)
        live = torch.cuda.memory_allocated()
        assert live > base  # tables and P0 held by PyTorch's allocator
        # while handles live the allocator cannot be switched
        with pytest.raises(W.WpcdError, match="live"):
            W.use_torch_allocator(False)
        P.close()
        pr.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base
    finally:
        W.use_torch_allocator(False)
    assert np.array_equal(U_own, U_torch)
