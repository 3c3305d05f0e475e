"""GPU checks of the dense channel-block products of the K application
(wpcd_channel_gemm, through the C ABI): the tensor-core TF32x3 kernel and the
FP32/FP64 SIMT kernels against an FP64 numpy product of the same blocks, on
grids that cover one to three 128-row tiles and ragged column tiles; and the
mixed solve with the tensor-core products against the FP64 oracle."""
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


def _reference(A, x, g, N, M, B):
    """FP64 products on [n_ch][N][M][B] complex blocks."""
    xc = x.reshape(A.shape[0], N, M * B)
    if g is not None:
        xc = xc * g.reshape(A.shape[0], N, M * B)
    return np.einsum("cik,ckj->cij", A, xc), np.einsum("cik,ckj->cij", np.abs(A), np.abs(xc))


# panels with M B even take the persistent bulk-copy kernel, (40, 15, 3) (M B
# odd: rows not 16-byte aligned) the one-tile-per-CTA register path;
# (40, 160, 64) gives 480 column tiles, so each persistent CTA takes three or
# four tiles and the stage rings and accumulator buffers wrap; (450, 40, 8)
# has four row tiles (one accumulator buffer)
# the persistent kernel's rings hand every panel chunk from the TMA producer
# to the converters and every operand stage to the MMA thread; a slot released
# too early shows as products that differ from call to call.  Repeated calls
# must agree bit for bit: 200 rows (three A stages, four raw chunks) and 450
# rows (two A stages, two raw chunks with G1, one accumulator buffer), each
# over enough column tiles that every ring wraps many times
@pytest.mark.parametrize("N,M,B", [(200, 40, 64), (450, 40, 16)])
@pytest.mark.parametrize("which", [0, 1])
def test_tensor_core_gemm_bit_identical_across_calls(W, N, M, B, which):
    import torch

    pr = _problem(W, N, M)
    n = pr.n_ch * N * M * B
    gen = torch.Generator().manual_seed(N + which)
    x = torch.randn(2 * n, generator=gen, dtype=torch.float32).cuda()
    g = torch.randn(2 * n, generator=gen, dtype=torch.float32).cuda() if which == 0 else None
    outs = []
    for _ in range(4):
        y = torch.full((2 * n,), float("nan"), dtype=torch.float32, device="cuda")
        pr.wpcd_channel_gemm(which, W.WPCD_GEMM_TF32X3, g, x, y, B)
        outs.append(y)
    assert torch.isfinite(outs[0]).all()
    for y in outs[1:]:
        assert torch.equal(y, outs[0])
    pr.close()


# the same for the digit-plane product (bf16 planes on the tensor cores, FP64
# in and out; A digits by bulk copy ahead of the MMAs)
@pytest.mark.parametrize("which", [0, 1])
def test_digit_plane_gemm_bit_identical_across_calls(W, which):
    import torch

    N, M, B = 200, 40, 16
    pr = _problem(W, N, M)
    n = pr.n_ch * N * M * B
    gen = torch.Generator().manual_seed(7 + which)
    x = torch.randn(2 * n, generator=gen, dtype=torch.float64).cuda()
    g = torch.randn(2 * n, generator=gen, dtype=torch.float64).cuda() if which == 0 else None
    outs = []
    for _ in range(4):
        y = torch.full((2 * n,), float("nan"), dtype=torch.float64, device="cuda")
        pr.wpcd_channel_gemm(which, W.WPCD_GEMM_DIGITS, g, x, y, B)
        outs.append(y)
    assert torch.isfinite(outs[0]).all()
    for y in outs[1:]:
        assert torch.equal(y, outs[0])
    pr.close()


@pytest.mark.parametrize("N,M,B", [(30, 28, 3), (130, 20, 5), (200, 16, 8), (300, 12, 2), (40, 15, 3),
                                   (40, 160, 64), (450, 40, 8)])
@pytest.mark.parametrize("which", [0, 1])
def test_tensor_core_gemm_matches_fp64(W, N, M, B, which):
    import torch
    from paper_1508_07441_gb300 import inputs

    pr = _problem(W, N, M)
    n = pr.n_ch * N * M * B
    x = inputs.random_complex(n, 11 + N).astype(np.complex64)
    g = inputs.random_complex(n, 12 + N).astype(np.complex64) if which == 0 else None
    A = _blocks(pr, which)
    ref, scale = _reference(A, x.astype(np.complex128), None if g is None else g.astype(np.complex128), N, M, B)
    xd = torch.from_numpy(x.view(np.float32)).cuda()
    gd = None if g is None else torch.from_numpy(g.view(np.float32)).cuda()
    # FP32 SIMT: the recursive-sum bound n 2^-24 of the magnitude sum (2.7e-5
    # at N = 450), at least 2e-6
    for mode, tol in ((W.WPCD_GEMM_TF32X3, 2e-5), (W.WPCD_GEMM_FP32, max(2e-6, N * 2.0**-24))):
        yd = torch.full((2 * n,), float("nan"), dtype=torch.float32, device="cuda")
        pr.wpcd_channel_gemm(which, mode, gd, xd, yd, B)
        got = yd.cpu().numpy().view(np.complex64).astype(np.complex128).reshape(ref.shape)
        err = np.abs(got - ref) / np.maximum(scale, 1e-30)
        # every output written (no NaN left) and within the FP32-class bound
        assert np.all(np.isfinite(got)), mode
        assert err.max() < tol, (mode, err.max())


@pytest.mark.parametrize("mode,tol", [("FP64", 1e-14), ("FF", 1e-12), ("DIGITS", 1e-13)])
@pytest.mark.parametrize("which", [0, 1])
def test_fp64_class_channel_gemm_matches_numpy(W, mode, tol, which):
    """FP64 SIMT and float-float (FP32 pipe) products against FP64 numpy on
    the same blocks.  The float-float sum carries its low part in one float,
    so its error grows like n 2^-48 of the magnitude sum (5e-13 for the
    n = 140 blocks here; FP64: n 2^-53)."""
    import torch
    from paper_1508_07441_gb300 import inputs

    N, M, B = 140, 30, 4
    pr = _problem(W, N, M)
    n = pr.n_ch * N * M * B
    x = inputs.random_complex(n, 5)
    g = inputs.random_complex(n, 6) if which == 0 else None
    ref, scale = _reference(_blocks(pr, which), x, g, N, M, B)
    yd = torch.full((2 * n,), float("nan"), dtype=torch.float64, device="cuda")
    m = {"FP64": W.WPCD_GEMM_FP64, "FF": W.WPCD_GEMM_FF, "DIGITS": W.WPCD_GEMM_DIGITS}[mode]
    ms = pr.wpcd_channel_gemm(which, m, None if g is None else torch.from_numpy(g.view(np.float64)).cuda(),
                              torch.from_numpy(x.view(np.float64)).cuda(), yd, B, timed=True)
    assert ms > 0.0
    got = yd.cpu().numpy().view(np.complex128).reshape(ref.shape)
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref) / scale) < tol


def test_channel_gemm_rejects_bad_arguments(W):
    import torch

    pr = _problem(W, 20, 10)
    x = torch.zeros(2 * pr.dim, dtype=torch.float32, device="cuda")
    with pytest.raises(W.WpcdError, match="mode"):
        pr.wpcd_channel_gemm(0, 7, None, x, x.clone(), 1)
    with pytest.raises(W.WpcdError, match="which"):
        pr.wpcd_channel_gemm(2, W.WPCD_GEMM_FP32, None, x, x.clone(), 1)
    with pytest.raises(W.WpcdError, match="bad vectors"):
        pr.wpcd_channel_gemm(0, W.WPCD_GEMM_FP32, None, x, x, 1)


@pytest.mark.parametrize("gemm", ["tc", "simt"])
def test_mixed_solve_with_either_fp32_product(W, orc, monkeypatch, gemm):
    """The mixed solve refines to the FP64 residual tolerance whichever FP32
    channel product its inner cycles use; U00 against the oracle."""
    from paper_1508_07441_gb300 import inputs

    monkeypatch.setenv("WPCD_GEMM", gemm)
    pe, qe = inputs.tangent_edges(30, 20.0), inputs.tangent_edges(28, 20.0)
    pr = W.Problem(pe, qe, 4, 4, 16, 3, (-6.0,), (1.0,))
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    E = [-0.3, 0.25, 0.9, 2.0, 4.5]
    U, stats, st = pr.wpcd_solve(P, E, tol=1e-12, precision=W.WPCD_SOLVE_MIXED, batch=len(E))
    assert st == W.WPCD_OK and all(s.relres <= 1e-12 for s in stats)
    opr = orc.Problem(dict(pe=pe, qe=qe, n_p=4, n_q=4, n_x=16, n_ch=3, V=[-6.0], a=[1.0], n_pair_nodes=8))
    ref = np.array([opr.solve_gmres(e, tol=1e-13, max_iter=300)["U00"] for e in E])
    assert np.max(np.abs(U - ref) / np.abs(ref)) < 1e-8


@pytest.mark.parametrize("B", [1, 6, 40])
def test_spmm_matches_oracle_P0(W, orc, B):
    """wpcd_spmm (z = P0 y, FP64 and FP32 vectors, tuned shapes) against the
    oracle's own P0 applied with scipy sparse products, per (l, l') block."""
    import scipy.sparse as sp
    import torch
    from paper_1508_07441_gb300 import inputs

    pe, qe = inputs.tangent_edges(26, 20.0), inputs.tangent_edges(22, 20.0)
    n_ch = 3
    pr = W.Problem(pe, qe, 4, 4, 16, n_ch, (-6.0,), (1.0,))
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    ref_P = orc.P0(pe, qe, 4, 4, 16, n_ch, with_abs=True)
    n_cells = 26 * 22
    y = inputs.random_complex(n_ch * n_cells * B, 77 + B).reshape(n_ch, n_cells, B)
    ref = np.zeros_like(y)
    mag = np.zeros(y.shape)
    for m, (l, lp) in enumerate(orc.pair_list(n_ch)):
        A = sp.csr_matrix((ref_P["val"][:, m], ref_P["col"], ref_P["row_ptr"]), shape=(n_cells, n_cells))
        ref[l] += A @ y[lp]
        # the term-magnitude sums of P0's elements: an element that is a
        # cancelling sum of node terms carries FP64 rounding relative to its
        # terms (the assembly's bar: 1e-10 |ref| + 1e-13 of that sum), not to
        # its own small value
        S = sp.csr_matrix((ref_P["absval"][:, m], ref_P["col"], ref_P["row_ptr"]), shape=(n_cells, n_cells))
        mag[l] += (abs(A) + S) @ np.abs(y[lp])
    # FP32: plain blocked sums, bounded by n 2^-24 of the magnitude sum with n
    # the terms of the longest row (nonzero cells x channel pairs)
    n_terms = int(np.max(np.diff(ref_P["row_ptr"]))) * len(orc.pair_list(n_ch))
    tol32 = max(3e-6, n_terms * 2.0**-24)
    modes = [(W.WPCD_SPMM_FP64, np.complex128, 1e-9), (W.WPCD_SPMM_FF, np.complex128, 1e-9),
             (W.WPCD_SPMM_FP32, np.complex64, tol32)]
    if B % 2 == 0:  # the row-tiled kernel takes even batches
        modes.append((W.WPCD_SPMM_FP32_BLOCKED, np.complex64, tol32))
    for mode, dt, tol in modes:
        fp32 = mode in (W.WPCD_SPMM_FP32, W.WPCD_SPMM_FP32_BLOCKED)
        yd = torch.from_numpy(y.astype(dt).reshape(-1).view(np.float32 if fp32 else np.float64)).cuda()
        zd = torch.full_like(yd, float("nan"))
        ms = pr.wpcd_spmm(P, yd, zd, B, mode=mode, timed=True)
        assert ms > 0.0
        got = zd.cpu().numpy().view(dt).astype(np.complex128).reshape(ref.shape)
        assert np.all(np.isfinite(got))
        # the P0 values themselves agree with the oracle's to 1e-10 (FP64
        # assembly); FF carries them to ~2^-48
        assert np.max(np.abs(got - ref) / np.maximum(mag, 1e-30)) < tol, mode


@pytest.mark.parametrize("N,M,rpw,cps", [(23, 19, 2, 1), (25, 21, 4, 2), (21, 17, 8, 1), (24, 20, 16, 2),
                                          (31, 27, 4, 1), (27, 23, 8, 2)])
def test_spmv_one_rhs_every_shape(W, orc, tmp_path, monkeypatch, N, M, rpw, cps):
    """The one-right-hand-side SpMV (FP64 and FP32) in every rows-per-warp
    shape with one and two chunks per step, forced through the autotuner's
    cache file, element by element against the oracle's P0 applied with
    scipy; the lattices give nnz odd (element loads of the values and a chunk
    at the end of the arrays), nnz = 2 mod 4 (8-byte value loads) and
    nnz = 0 mod 4 (16-byte value loads)."""
    import scipy.sparse as sp
    import torch
    from paper_1508_07441_gb300 import inputs

    n_ch = 3
    cache = tmp_path / "tune.txt"
    with open(cache, "w") as f:
        for mode in (0, 1):  # FP64 and FP32 vectors, B = 1
            key = ((((n_ch * 4096 + N) * 4096 + M) * 4096 + 1) * 4 + mode)
            f.write(f"{key} {rpw} 1 {cps}\n")
    monkeypatch.setenv("WPCD_TUNE_CACHE", str(cache))
    pe, qe = inputs.tangent_edges(N, 20.0), inputs.tangent_edges(M, 20.0)
    pr = W.Problem(pe, qe, 4, 4, 16, n_ch, (-6.0,), (1.0,))
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    ref_P = orc.P0(pe, qe, 4, 4, 16, n_ch, with_abs=True)
    n_cells = N * M
    y = inputs.random_complex(n_ch * n_cells, 5 + N).reshape(n_ch, n_cells, 1)
    ref, mag = np.zeros_like(y), np.zeros(y.shape)
    for m, (l, lp) in enumerate(orc.pair_list(n_ch)):
        A = sp.csr_matrix((ref_P["val"][:, m], ref_P["col"], ref_P["row_ptr"]), shape=(n_cells, n_cells))
        ref[l] += A @ y[lp]
        # the term-magnitude sums of P0's elements: an element that is a
        # cancelling sum of node terms carries FP64 rounding relative to its
        # terms (the assembly's bar: 1e-10 |ref| + 1e-13 of that sum), not to
        # its own small value
        S = sp.csr_matrix((ref_P["absval"][:, m], ref_P["col"], ref_P["row_ptr"]), shape=(n_cells, n_cells))
        mag[l] += (abs(A) + S) @ np.abs(y[lp])
    n_terms = int(np.max(np.diff(ref_P["row_ptr"]))) * len(orc.pair_list(n_ch))
    for fp32, dt, tol in ((False, np.complex128, 1e-9), (True, np.complex64, max(3e-6, n_terms * 2.0**-24))):
        yd = torch.from_numpy(y.astype(dt).reshape(-1).view(np.float32 if fp32 else np.float64)).cuda()
        zd = torch.full_like(yd, float("nan"))
        pr.wpcd_spmm(P, yd, zd, 1, mode=W.WPCD_SPMM_FP32 if fp32 else W.WPCD_SPMM_FP64)
        assert pr.wpcd_tune_spmm(P, 1, fp32=fp32) == (rpw, 1, cps)  # the forced shape ran
        got = zd.cpu().numpy().view(dt).astype(np.complex128).reshape(ref.shape)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref) / np.maximum(mag, 1e-30)) < tol, (fp32, rpw)


@pytest.mark.parametrize("N,M,B,tile,ept,fab", [(19, 23, 6, 2, 4, 1), (20, 17, 40, 2, 2, 2), (17, 21, 130, 4, 2, 1),
                                               (22, 19, 128, 2, 4, 2), (18, 25, 64, 4, 2, 2), (21, 20, 2, 2, 2, 1)])
def test_spmm_tiled_every_shape(W, orc, tmp_path, monkeypatch, N, M, B, tile, ept, fab):
    """The row-tiled FP32 SpMM (tiles of 2 cells with 4 or 2 energies per
    lane, of 2 x 2 cells with 2; plain blocks of 32 (fab 1) or 64 (fab 2)
    columns), forced through the autotuner's cache file,
    element by element against the oracle's P0 applied with scipy; odd
    lattice sizes give tiles cut by the lattice edge, and batches of 6, 40,
    130 leave lanes without energies."""
    import scipy.sparse as sp
    import torch
    from paper_1508_07441_gb300 import inputs

    n_ch = 3
    cache = tmp_path / "tune.txt"
    key = ((((n_ch * 4096 + N) * 4096 + M) * 4096 + B) * 4 + 1)
    cache.write_text(f"{key} {fab} 32 {ept} {tile}\n")
    monkeypatch.setenv("WPCD_TUNE_CACHE", str(cache))
    pe, qe = inputs.tangent_edges(N, 20.0), inputs.tangent_edges(M, 20.0)
    pr = W.Problem(pe, qe, 4, 4, 16, n_ch, (-6.0,), (1.0,))
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    ref_P = orc.P0(pe, qe, 4, 4, 16, n_ch, with_abs=True)
    n_cells = N * M
    y = inputs.random_complex(n_ch * n_cells * B, 900 + B).reshape(n_ch, n_cells, B)
    ref, mag = np.zeros_like(y), np.zeros(y.shape)
    for m, (l, lp) in enumerate(orc.pair_list(n_ch)):
        A = sp.csr_matrix((ref_P["val"][:, m], ref_P["col"], ref_P["row_ptr"]), shape=(n_cells, n_cells))
        ref[l] += A @ y[lp]
        # the term-magnitude sums of P0's elements: an element that is a
        # cancelling sum of node terms carries FP64 rounding relative to its
        # terms (the assembly's bar: 1e-10 |ref| + 1e-13 of that sum), not to
        # its own small value
        S = sp.csr_matrix((ref_P["absval"][:, m], ref_P["col"], ref_P["row_ptr"]), shape=(n_cells, n_cells))
        mag[l] += (abs(A) + S) @ np.abs(y[lp])
    n_terms = int(np.max(np.diff(ref_P["row_ptr"]))) * len(orc.pair_list(n_ch))
    yd = torch.from_numpy(y.astype(np.complex64).reshape(-1).view(np.float32)).cuda()
    zd = torch.full_like(yd, float("nan"))
    pr.wpcd_spmm(P, yd, zd, B, mode=W.WPCD_SPMM_FP32)
    assert pr.wpcd_tune_spmm(P, B, fp32=True) == (tile, 32, ept)  # the forced shape ran
    got = zd.cpu().numpy().view(np.complex64).astype(np.complex128).reshape(ref.shape)
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref) / np.maximum(mag, 1e-30)) < max(3e-6, n_terms * 2.0**-24)
