"""The warm-start network: the library's FP32 forward/backward kernels
against the FP64 oracle MLP, BF16 inference error, training, and what the
trained network gains over the plain iteration at equal residual."""
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


def _setup(W, n_in=9, width=32, n_out=6, n=40, seed=11):
    import torch

    rng = np.random.default_rng(seed)
    m = W.MLP(n_in, width, n_out, seed=seed)
    p = (rng.standard_normal(m.n_params) * 0.3).astype(np.float32)
    m.wpcd_mlp_params(set=p)
    aff = [rng.uniform(0.5, 2.0, n_in), rng.standard_normal(n_in) * 0.1, rng.uniform(0.5, 2.0, n_out),
           rng.standard_normal(n_out)]
    aff = [a.astype(np.float32) for a in aff]
    m.wpcd_mlp_set_affine(*aff)
    X = rng.standard_normal((n, n_in)).astype(np.float32)
    T = rng.standard_normal((n, n_out)).astype(np.float32)
    return m, p, aff, X, T, torch


def test_gradient_matches_oracle(W):
    from oracle import mlp as om

    m, p, aff, X, T, torch = _setup(W)
    g = torch.zeros(m.n_params, dtype=torch.float32, device="cuda")
    loss = m.wpcd_mlp_loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), grad=g)
    lref, gref = om.loss_grad(p.astype(np.float64), X, T, 9, 32, 6, (aff[0], aff[1]), (aff[2], aff[3]))
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(loss - lref) < 1e-5 * lref
    assert np.linalg.norm(gg - gref) < 1e-4 * np.linalg.norm(gref)


def test_forward_fp32_and_bf16(W):
    from oracle import mlp as om

    m, p, aff, X, T, torch = _setup(W, n=64)
    Xd = torch.from_numpy(X).cuda()
    Y = torch.zeros(64 * 6, dtype=torch.float32, device="cuda")
    m.wpcd_mlp_forward(Xd, Y)
    yref, _ = om.forward(p.astype(np.float64), X, 9, 32, 6, (aff[0], aff[1]), (aff[2], aff[3]))
    y = Y.cpu().numpy().reshape(64, 6)
    assert np.max(np.abs(y - yref)) < 1e-5 * np.abs(yref).max()
    m.wpcd_mlp_forward(Xd, Y, bf16=True)
    yb = Y.cpu().numpy().reshape(64, 6)
    rel = np.linalg.norm(yb - yref) / np.linalg.norm(yref)
    assert 1e-6 < rel < 3e-2  # BF16 weights: about 8 bits of mantissa


def test_training_reduces_loss(W):
    import torch

    rng = np.random.default_rng(5)
    n = 1024
    x = rng.uniform(-1, 1, (n, 2)).astype(np.float32)
    t = np.stack([np.sin(3 * x[:, 0]) * x[:, 1], np.cos(2 * x[:, 0] + x[:, 1])], axis=1).astype(np.float32)
    m = W.MLP(2, 64, 2, seed=3)
    X, T = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    l0 = m.wpcd_mlp_loss_grad(X, T)
    hist = m.wpcd_mlp_train(X, T, epochs=200, batch=128, lr=3e-3)
    l1 = m.wpcd_mlp_loss_grad(X, T)
    assert l1 < 0.02 * l0 and hist[-1] < hist[0]


def test_warm_softmax_matches_numpy(W):
    """mixture weights of the warm start: row softmax of the logits as (w, 0)
    pairs, one warp per row; k beyond 32 (several entries per lane) and a
    ragged last row block"""
    import torch

    rng = np.random.default_rng(7)
    for n, k in ((13, 64), (3, 5), (9, 100)):
        z = (rng.standard_normal((n, k)) * 8).astype(np.float32)
        C = torch.full((n * 2 * k,), float("nan"), dtype=torch.float32, device="cuda")
        W.wpcd_warm_softmax(torch.from_numpy(z).cuda(), n, k, C)
        got = C.cpu().numpy().reshape(n, k, 2)
        e = np.exp(z.astype(np.float64) - z.max(axis=1, keepdims=True))
        ref = e / e.sum(axis=1, keepdims=True)
        assert np.all(got[:, :, 1] == 0.0)
        assert np.max(np.abs(got[:, :, 0] - ref)) < 2e-6, (n, k)


def test_warm_start_saves_iterations(W, orc):
    """Trained on the method's own solutions of a 3-channel system, the
    network's warm start reaches the same FP64 relative residual (1e-8) in
    fewer K applications than the zero start, on held-out energies, and the
    amplitudes agree with the oracle."""
    from paper_1508_07441_gb300 import inputs
    from paper_1508_07441_gb300.warmstart import WarmStart

    pe, qe = inputs.tangent_edges(48, 20.0), inputs.tangent_edges(48, 20.0)
    pr = W.Problem(pe, qe, 4, 4, 16, 3, (-3.0,), (1.0,))
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    ws = WarmStart(pr, P, k=48, kf=12, width=128, seed=2026)
    lo, hi = -0.9 * abs(pr.eps_bound), 5.0
    ws.e_lo, ws.e_hi = lo, hi
    ws.build_basis(ws.snapshot_energies(lo, hi))
    X, T = ws.dataset(inputs.random_energies(pr.eps_bound, 384, seed=2026))
    hist = ws.fit(X, T, epochs=400, batch=128, lr=2e-3, decay=(0.1, 0.01))
    assert hist[-1] < 0.2 * hist[0]
    E = inputs.random_energies(pr.eps_bound, 48, seed=2027)
    cold, rc, _, Uc = ws.iterations(E, tol=1e-8)
    ug = ws.predict(E)
    warm, rw, fb, Uw = ws.iterations(E, u_init=ug, tol=1e-8)
    assert np.all(rc <= 1e-8) and np.all(rw <= 1e-8)   # equal residual
    print(f"warm start: {cold.mean():.2f} -> {warm.mean():.2f} K applications, fallbacks {fb.sum()}")
    # measured 12.85 -> 2.54 (80 % fewer): the snapshots hold the solutions
    # of the bins that carry most of the energy range, and the mixture
    # weights pick the energy's own bin
    assert warm.mean() < 0.5 * cold.mean(), (warm.mean(), cold.mean())
    assert np.max(np.abs(Uw - Uc) / np.abs(Uc)) < 1e-6
    opr = orc.Problem(dict(pe=pe, qe=qe, n_p=4, n_q=4, n_x=16, n_ch=3, V=[-3.0], a=[1.0], n_pair_nodes=8))
    for k in (0, 17, 47):
        ref = opr.solve_gmres(E[k], tol=1e-12, max_iter=400)["U00"]
        assert abs(Uw[k] - ref) / abs(ref) < 1e-6
