"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances: P0 elements rel 1e-10 in FP64 and 1e-5 in FP32C.  Some
elements are exactly zero in exact arithmetic (for l' = 0 the GL rule
integrates P_l(y) to zero when all y-nodes of a (p, q) pair land in one
target), and in FP32 a node term W P_l(y) P_l'(y') carries an absolute error
of order eps_32 W |P_l(y)| even where P_l'(y') passes through a root; so the
bar is per element |d| <= rel |ref| + abs S, with S = sum_nodes W |P_l(y)|
(the magnitude bounding every term, |P_l'| <= 1) from the oracle:
(rel, abs) = (1e-10, 1e-13) in FP64 and (1e-5, 1e-6) in FP32C.  The pattern
(row pointers and columns) must match exactly, so a misbinned node is an
error.  Amplitudes rel 1e-6.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-10, 1e-13), "fp32c": (1e-5, 1e-6)}


@pytest.fixture(scope="module")
def W():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07441_gb300 import build, wpcd

    build.build()
    return wpcd


def _inputs(N, M, jitter=None, kmax=20.0):
    from paper_1508_07441_gb300 import inputs

    if jitter is None:
        return inputs.tangent_edges(N, kmax), inputs.tangent_edges(M, kmax)
    return inputs.jittered_edges(N, kmax, jitter), inputs.jittered_edges(M, kmax, jitter + 1)


def _excess(val, ref, absref, prec):
    """max over elements of |d| / (rel |ref| + abs S); <= 1 passes"""
    rel, ab = TOL[prec]
    return np.max(np.abs(val - ref) / (rel * np.abs(ref) + ab * absref + 1e-300))


def _measure_stats(val, ref, absref, row_ptr, n_ch, prec):
    """The per-element measure |d| / max(|ref|, 1e-12 rowmax) (rowmax: the
    largest |ref| of the element's matrix row (l, c)), and how many elements
    meet the bar only through its absolute term (their measure is above rel)."""
    rel, ab = TOL[prec]
    pairs = [(l, lp) for l in range(n_ch) for lp in range(n_ch) if (l + lp) % 2 == 0]
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    rowmax = np.zeros((len(row_ptr) - 1, n_ch))
    for k, (l, _) in enumerate(pairs):
        np.maximum.at(rowmax[:, l], rows, np.abs(ref[:, k]))
    rm = np.stack([rowmax[rows, l] for l, _ in pairs], axis=1)
    d = np.abs(val - ref)
    meas = d / np.maximum(np.abs(ref), 1e-12 * rm + 1e-300)
    bar = d <= rel * np.abs(ref) + ab * absref
    return dict(n=d.size, max_measure=float(meas.max()), n_abs_only=int((bar & (meas > rel)).sum()))


CASES = [
    # (N, M, nodes, n_ch, jitter seed)
    (20, 16, (4, 4, 16), 1, None),
    (12, 14, (3, 5, 7), 3, None),
    (17, 23, (4, 6, 12), 2, 11),
    (26, 22, (8, 8, 32), 5, 21),
    # n_x a multiple of 32 (a warp step is one (p, q) pair's y nodes):
    # 64 y nodes, and a node count that is not a power of two
    (14, 18, (3, 2, 64), 3, 5),
    (19, 13, (3, 5, 32), 2, None),
    (50, 50, (4, 4, 16), 1, None),  # the s-wave benchmark lattice
]


@pytest.mark.parametrize("N,M,nodes,n_ch,jit", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_assemble_matches_oracle(W, orc, N, M, nodes, n_ch, jit, prec):
    pe, qe = _inputs(N, M, jit)
    pr = W.Problem(pe, qe, *nodes, n_ch, (-6.0,), (1.0,))
    P = pr.wpcd_assemble_P(W.WPCD_FP64 if prec == "fp64" else W.WPCD_FP32C)
    rp, col, val = P.wpcd_P_export()
    ref = orc.P0(pe, qe, *nodes, n_ch, with_abs=True)
    assert np.array_equal(rp, ref["row_ptr"])
    assert np.array_equal(col, ref["col"])
    assert _excess(val.T, ref["val"], ref["absval"], prec) <= 1.0
    st = _measure_stats(val.T, ref["val"], ref["absval"], ref["row_ptr"], n_ch, prec)
    print(f"P0-measure {prec} {N}x{M} n_ch={n_ch}: {st}")
    # elements that pass only through the absolute term: vanishing sums and
    # FP32 terms at roots of P_l'; a bounded minority
    assert st["n_abs_only"] <= (0.01 if prec == "fp32c" else 0.005) * st["n"], st


def test_assemble_rows_beyond_first_hash_set(W, orc):
    """60 fine bins and one coarse outer bin, 16 x 16 x 32 nodes per cell (the
    8192-node maximum): rows of the coarse cells reach 327 targets, more than
    half the count pass's first hash set (512 slots for N + M = 122), so the
    pass runs again with the full set; the result matches the oracle as
    everywhere else"""
    pe = np.concatenate([np.linspace(0.0, 4.0, 61), [8.0]])
    nodes, n_ch = (16, 16, 32), 1
    pr = W.Problem(pe, pe, *nodes, n_ch, (-6.0,), (1.0,))
    ref = orc.P0(pe, pe, *nodes, n_ch, with_abs=True)
    assert np.diff(ref["row_ptr"]).max() > 256
    for prec in ("fp64", "fp32c"):
        P = pr.wpcd_assemble_P(W.WPCD_FP64 if prec == "fp64" else W.WPCD_FP32C)
        rp, col, val = P.wpcd_P_export()
        assert np.array_equal(rp, ref["row_ptr"])
        assert np.array_equal(col, ref["col"])
        assert _excess(val.T, ref["val"], ref["absval"], prec) <= 1.0


def test_assemble_deterministic(W):
    pe, qe = _inputs(30, 30)
    pr = W.Problem(pe, qe, 8, 8, 32, 3, (-6.0,), (1.0,))
    a = pr.wpcd_assemble_P(W.WPCD_FP64).wpcd_P_export()
    b = pr.wpcd_assemble_P(W.WPCD_FP64).wpcd_P_export()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_assemble_full_size_3_channels(W, orc):
    """The 3-channel, 200 x 200 lattice with 8x8x32 nodes (dimension 120 000)
    compared element by element with the oracle (FP64 and FP32C)."""
    from paper_1508_07441_gb300 import inputs

    w = inputs.workload("bosons3_200")
    pr = W.Problem(w["p_edges"], w["q_edges"], *w["nodes"], w["n_ch"], w["V"], w["a"])
    ref = orc.P0(w["p_edges"], w["q_edges"], *w["nodes"], w["n_ch"], with_abs=True)
    for prec, name in [(W.WPCD_FP64, "fp64"), (W.WPCD_FP32C, "fp32c")]:
        P = pr.wpcd_assemble_P(prec)
        rp, col, val = P.wpcd_P_export()
        assert np.array_equal(rp, ref["row_ptr"])
        assert np.array_equal(col, ref["col"])
        assert _excess(val.T, ref["val"], ref["absval"], name) <= 1.0
        st = _measure_stats(val.T, ref["val"], ref["absval"], ref["row_ptr"], w["n_ch"], name)
        print(f"P0-measure {name} 200x200 n_ch=3: {st}")
        # measured: 11 881 (FP32C) and 1 306 (FP64) of 14 974 110
        assert st["n_abs_only"] <= (0.002 if name == "fp32c" else 0.0005) * st["n"], st


# the potential matrices are formed on the device (a thread per bin pair,
# the Bessel recurrence per node pair serving every l), the eigenproblems on
# the host: one Gaussian and three channels, and the short-range repulsive
# sum of two Gaussians with five channels (l up to 4, large z = p p' a / 2)
@pytest.mark.parametrize("N,n_ch,V,a", [(60, 3, (-3.0,), (1.0,)), (50, 5, (-6.0, 2.0), (0.5, 0.1))])
def test_pair_setup_matches_oracle(W, orc, N, n_ch, V, a):
    pe, qe = _inputs(N, 40)
    pr = W.Problem(pe, qe, 4, 4, 16, n_ch, V, a, n_pair_nodes=8)
    for l in range(n_ch):
        eps, O, v = pr.wpcd_problem_pair(l)
        v2, _, eps2, O2 = orc.pair(pe, 8, l, list(V), list(a))
        assert np.max(np.abs(eps - eps2)) < 1e-12 * np.abs(eps2).max()
        assert np.max(np.abs(v - v2)) < 1e-12 * np.abs(v2).max()
        assert np.max(np.abs(O - O2)) < 1e-8


@pytest.mark.parametrize("E", [-0.3, 0.5, 3.0])
def test_resolvent_matches_oracle(W, orc, E):
    import torch

    pe, qe = _inputs(30, 40)
    pr = W.Problem(pe, qe, 4, 4, 16, 3, (-6.0,), (1.0,))
    g = torch.zeros(2 * pr.dim, dtype=torch.float64, device="cuda")
    j0, D = pr.wpcd_resolvent([E], g)
    eps = np.stack([pr.wpcd_problem_pair(l)[0] for l in range(3)])
    ref, j0r, Dr = orc.G1(eps, qe, E, pr.eps_bound)
    got = g.cpu().numpy().view(np.complex128).reshape(3, 30, 40)
    assert j0[0] == j0r and abs(D[0] - Dr) <= 1e-15 * Dr
    assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)) < 1e-9


def test_resolvent_many_energies_shared_bins(W, orc):
    """Several energies, some in the same on-shell bin and out of order: G1
    is computed once per bin and written for each of its energies; every
    energy's block matches the oracle's G1 at that energy."""
    import torch

    pe, qe = _inputs(30, 40)
    pr = W.Problem(pe, qe, 4, 4, 16, 3, (-6.0,), (1.0,))
    E = [0.5, 3.0, 0.5001, -0.3, 2.9999, 0.52, 0.5]
    g = torch.zeros(2 * pr.dim * len(E), dtype=torch.float64, device="cuda")
    j0, D = pr.wpcd_resolvent(E, g)
    assert len(set(j0)) < len(E)  # some bins are shared
    eps = np.stack([pr.wpcd_problem_pair(l)[0] for l in range(3)])
    got = g.cpu().numpy().view(np.complex128).reshape(len(E), 3, 30, 40)
    for k, e in enumerate(E):
        ref, j0r, Dr = orc.G1(eps, qe, e, pr.eps_bound)
        assert j0[k] == j0r
        assert np.max(np.abs(got[k] - ref) / np.maximum(np.abs(ref), 1e-300)) < 1e-9


def _kapply_bound(opr, x, g):
    """Per output of y = O P0 Vt (g o x): the sum of the magnitudes of its
    terms, |O| |P0| |Vt| |g o x| (the oracle's K application on the absolute
    values), which bounds the rounding error of any summation order."""
    import copy

    a = copy.copy(opr)
    a.O, a.Vt = np.abs(opr.O), np.abs(opr.Vt)
    a.P = dict(opr.P)
    a.P["val"] = np.abs(opr.P["val"])
    gx = np.abs(x * (g if g is not None else 1.0)).astype(np.complex128)
    return a.kapply(gx, None).real


def test_kapply_matches_oracle(W, orc):
    """Element by element on the same inputs: the oracle applies the library's
    own O, Vt = v O^T and P0 (exported), so the two sides differ by rounding
    only, and |y - y_ref| <= gamma S per output, S the sum of its terms'
    magnitudes and gamma = 4 (N + n_terms + N) 2^-53 (three summations, of
    N, of at most n_pairs times the longest row, and of N terms): a wrong
    small block cannot hide under a norm.  End to end (the oracle's own pair
    setup and P0, whose eigenvectors agree with the library's to about 1e-8)
    the results agree in norm."""
    import torch
    from paper_1508_07441_gb300 import inputs

    pe, qe = _inputs(28, 24)
    nodes, n_ch = (4, 4, 16), 3
    pr = W.Problem(pe, qe, *nodes, n_ch, (-6.0,), (1.0,))
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    opr = orc.Problem(dict(pe=pe, qe=qe, n_p=4, n_q=4, n_x=16, n_ch=n_ch, V=[-6.0], a=[1.0],
                           n_pair_nodes=8))
    same = orc.Problem(dict(pe=pe, qe=qe, n_p=4, n_q=4, n_x=16, n_ch=n_ch, V=[-6.0], a=[1.0],
                            n_pair_nodes=8), P=opr.P)
    rp, col, val = P.wpcd_P_export()
    same.P = dict(row_ptr=rp, col=col, val=np.ascontiguousarray(val.T))
    pairs = [pr.wpcd_problem_pair(l) for l in range(n_ch)]
    same.O = np.ascontiguousarray(np.stack([O for _, O, _ in pairs]))
    same.Vt = np.ascontiguousarray(np.einsum("lij,lkj->lik", np.stack([v for _, _, v in pairs]), same.O))
    rowlen = int(np.diff(rp).max()) * orc.n_pairs(n_ch)
    gamma = 4 * (28 + rowlen + 28) * 2.0 ** -53
    x = inputs.random_complex(pr.dim, 7)
    g = torch.zeros(2 * pr.dim, dtype=torch.float64, device="cuda")
    pr.wpcd_resolvent([0.7], g)
    gx = g.cpu().numpy().view(np.complex128)
    xd = torch.from_numpy(x.view(np.float64).copy()).cuda()
    yd = torch.zeros_like(xd)
    for gg, gh in ((g, gx), (None, None)):  # with G1, and G1 = 1
        pr.wpcd_kapply(P, gg, xd, yd)
        y = yd.cpu().numpy().view(np.complex128)
        ref = same.kapply(x, gh)
        S = _kapply_bound(same, x, gh)
        assert np.all(np.abs(y - ref) <= gamma * S), np.max(np.abs(y - ref) / S)
        # the bar has power: the outputs are far above it
        assert np.median(np.abs(ref) / S) > 1e3 * gamma
        end = opr.kapply(x, gh)
        assert np.linalg.norm(y - end) / np.linalg.norm(end) < 1e-11


def _problems(W, orc, N, M, nodes, n_ch, V=(-6.0,), a=(1.0,), prec=None):
    pe, qe = _inputs(N, M)
    pr = W.Problem(pe, qe, *nodes, n_ch, V, a)
    P = pr.wpcd_assemble_P(W.WPCD_FP64 if prec is None else prec)
    opr = orc.Problem(dict(pe=pe, qe=qe, n_p=nodes[0], n_q=nodes[1], n_x=nodes[2], n_ch=n_ch,
                           V=list(V), a=list(a), n_pair_nodes=8))
    return pr, P, opr


@pytest.mark.parametrize("n_ch,E", [(1, 0.5), (3, 0.5), (3, 2.5), (3, -0.2)])
def test_solve_krylov_matches_oracle(W, orc, n_ch, E):
    pr, P, opr = _problems(W, orc, 24, 22, (4, 4, 16), n_ch)
    U, stats, st = pr.wpcd_solve(P, [E], method=W.WPCD_SUM_KRYLOV, tol=1e-12, max_iter=150)
    assert st == W.WPCD_OK and stats[0].status == W.WPCD_OK
    ref = opr.solve_gmres(E, tol=1e-13)["U00"]
    assert abs(U[0] - ref) / abs(ref) < 1e-6
    assert abs(U[0] - ref) / abs(ref) < 1e-9  # FP64 end to end: far inside the bar
    S, A = opr.amplitudes(E, ref)
    assert abs(complex(*stats[0].S) - S) < 1e-6 * abs(S)
    assert abs(complex(*stats[0].A) - A) < 1e-6 * abs(A)


def test_solve_s_wave_benchmark_lattice(W, orc):
    """The s-wave 50 x 50 lattice, V = -3 exp(-r^2), E = 0.5: both summations."""
    from paper_1508_07441_gb300 import inputs

    w = inputs.workload("swave_50")
    pr = W.Problem(w["p_edges"], w["q_edges"], *w["nodes"], 1, w["V"], w["a"])
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    opr = orc.Problem(dict(pe=w["p_edges"], qe=w["q_edges"], n_p=4, n_q=4, n_x=16, n_ch=1,
                           V=list(w["V"]), a=list(w["a"]), n_pair_nodes=8))
    ref = opr.solve_gmres(0.5, tol=1e-13)["U00"]
    U, stats, st = pr.wpcd_solve(P, [0.5], method=W.WPCD_SUM_KRYLOV, tol=1e-12)
    assert abs(U[0] - ref) / abs(ref) < 1e-9
    Uw, sw, stw = pr.wpcd_solve(P, [0.5], method=W.WPCD_SUM_WYNN, tol=1e-10, max_iter=80,
                                check_every=1)
    ow = opr.solve_wynn(0.5, tol=1e-10, max_iter=80)
    assert abs(Uw[0] - ow["U00"]) / abs(ow["U00"]) < 1e-6
    assert abs(Uw[0] - ref) / abs(ref) < 1e-6


def test_unitarity_below_breakup_gpu(W, orc):
    pr, P, opr = _problems(W, orc, 24, 24, (4, 4, 16), 3)
    E = 0.5 * pr.eps_bound
    U, stats, st = pr.wpcd_solve(P, [E], tol=1e-13, max_iter=200)
    assert abs(abs(complex(*stats[0].S)) - 1.0) < 1e-9


def test_fp32c_P_amplitude_error_stated(W, orc):
    """FP32C-assembled P0, FP64 solve: amplitude error against the FP64 oracle
    stays at the FP32 rounding level of P0."""
    pr, P, opr = _problems(W, orc, 24, 22, (4, 4, 16), 3, prec=W.WPCD_FP32C)
    U, stats, st = pr.wpcd_solve(P, [1.5], tol=1e-12)
    ref = opr.solve_gmres(1.5, tol=1e-13)["U00"]
    assert abs(U[0] - ref) / abs(ref) < 1e-5


def test_invalid_energies_rejected(W):
    pe, qe = _inputs(20, 20)
    pr = W.Problem(pe, qe, 4, 4, 16, 1, (-6.0,), (1.0,))
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    for E, code in [(pr.eps_bound - 0.1, W.WPCD_ENOBOUND), (float("nan"), W.WPCD_EINVAL),
                    (1e6, W.WPCD_EINVAL)]:
        with pytest.raises(W.WpcdError) as ei:
            pr.wpcd_solve(P, [E])
        assert ei.value.status == code
    with pytest.raises(W.WpcdError):
        pr.wpcd_assemble_P(7)


def test_enoconv_returns_best_estimate(W):
    pe, qe = _inputs(20, 20)
    pr = W.Problem(pe, qe, 4, 4, 16, 1, (-6.0,), (1.0,))
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    U, stats, st = pr.wpcd_solve(P, [1.0], tol=1e-30, max_iter=3, check_every=1)
    assert st == W.WPCD_ENOCONV and stats[0].status == W.WPCD_ENOCONV
    assert np.isfinite(U[0])
