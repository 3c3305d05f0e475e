"""FP64 CPU oracle for the WPCD Faddeev hot path (arXiv:1508.07441).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  Nothing here is shared with
the CUDA library: the C sources in this folder are compiled on their own
(``build()``) and loaded through ctypes.

Parity status of each piece (pins live in ``tests/test_oracle_*.py``):

- Gauss-Legendre rules: pinned (two algorithms, library routine, exactness).
- v_l closed form: pinned (radial quadrature of the Bessel integral).
- pair diagonalisation: pinned (library eigensolver, Numerov bound state).
- node-binned P0: pinned by the l = 0 sum rule, convergence to the exact cell
  overlap (``exact_overlap`` below, a different algorithm), symmetry of the
  exact overlap, cross-parity zeros and the energy-shell pattern; its overall
  scale and the sqrt((2l+1)(2l'+1)) factor of every block with l, l' <= 4 by
  P f = 2 f for totally symmetric and antisymmetric f (the two cyclic
  permutations map such an f to itself), block by block, converging at
  second order in the cell size.  The node
  sum itself is the method's quadrature, so its agreement with the exact
  integral is a convergence statement, not an identity.
- G1: pinned (adaptive quadrature of the defining integral, closed-form
  imaginary part on the bound channel).
- Wynn / Krylov summation: pinned (dense LU of (I - K) u = u0, unitarity of
  S below breakup).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wpcd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENOCONV, EBREAKDOWN, ENOBOUND = 0, -1, -2, -4, -5, -7


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)
_INT = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            c_int, c_double, c_i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
            sig = {
                "orc_num_threads": (c_int, []),
                "orc_set_threads": (None, [c_int]),
                "orc_gl_newton": (c_int, [c_int, _D, _D]),
                "orc_gl_golub_welsch": (c_int, [c_int, _D, _D]),
                "orc_jacobi_eigh": (c_int, [c_int, _D, _D, _D]),
                "orc_tangent_edges": (None, [c_int, c_double, _D]),
                "orc_sph_i_scaled": (c_double, [c_int, c_double]),
                "orc_vl": (c_double, [c_int, c_double, c_double, c_int, _D, _D]),
                "orc_pair": (c_int, [c_int, _D, c_int, c_int, c_int, _D, _D, _D, _D, _D, _D]),
                "orc_n_pairs": (c_int, [c_int]),
                "orc_P0_count": (c_i64, [c_int, _D, c_int, _D, c_int, c_int, c_int, _I64]),
                "orc_P0_fill": (c_int, [c_int, _D, c_int, _D, c_int, c_int, c_int, c_int, _I64,
                                        _I32, _D, _D, _D]),
                "orc_P0_node_totals": (c_int, [c_int, _D, c_int, _D, c_int, c_int, c_int, c_int, _D]),
                "orc_P0_normalize": (None, [c_int, _D, c_int, _D, c_int, _I64, _I32, _D]),
                "orc_P0_vl_count": (c_i64, [c_int, _D, c_int, _D, c_int, c_int, c_int, _I64]),
                "orc_P0_vl_fill": (c_int, [c_int, _D, c_int, _D, c_int, c_int, c_int, c_int, _I64,
                                           _I32, _D, _D]),
                "orc_onshell": (c_int, [c_int, _D, c_double, c_double, _INT, _D, _D, _D]),
                "orc_G1": (c_int, [c_int, c_int, _D, c_int, _D, c_double, c_double, _D, _INT, _D]),
                "orc_kapply": (None, [c_int, c_int, c_int, _D, _D, _I64, _I32, _D, _D, _D, _D]),
                "orc_wynn": (c_int, [c_int, _D, _D]),
                "orc_solve_wynn": (c_int, [c_int, c_int, c_int, _D, _D, _I64, _I32, _D, _D, c_int,
                                           c_int, c_int, c_double, _D, _INT, _D]),
                "orc_solve_gmres": (c_int, [c_int, c_int, c_int, _D, _D, _I64, _I32, _D, _D, _D, _D,
                                            c_int, c_double, _INT, _D]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a, ty=_D):
    if a is None:
        return None
    return a.ctypes.data_as(ty)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


# --------------------------------------------------------------------------
# quadrature, grids, pair interaction
# --------------------------------------------------------------------------
def gl_newton(n: int):
    x, w = np.zeros(n), np.zeros(n)
    assert lib().orc_gl_newton(n, _p(x), _p(w)) == OK
    return x, w


def gl_golub_welsch(n: int):
    x, w = np.zeros(n), np.zeros(n)
    assert lib().orc_gl_golub_welsch(n, _p(x), _p(w)) == OK
    return x, w


def jacobi_eigh(A):
    A = _f64(A).copy()
    n = A.shape[0]
    ev, V = np.zeros(n), np.zeros((n, n))
    assert lib().orc_jacobi_eigh(n, _p(A), _p(ev), _p(V)) == OK
    return ev, V


def tangent_edges(N: int, pmax: float):
    e = np.zeros(N + 1)
    lib().orc_tangent_edges(N, pmax, _p(e))
    return e


def sph_i_scaled(l: int, z: float) -> float:
    return lib().orc_sph_i_scaled(l, z)


def vl(l: int, p: float, pp: float, V, a) -> float:
    V, a = _f64(V), _f64(a)
    return lib().orc_vl(l, p, pp, len(V), _p(V), _p(a))


def pair(edges, n_nodes: int, l: int, V, a):
    """Free-packet potential matrix v, h1, eigenvalues eps, rotation O."""
    e, V, a = _f64(edges), _f64(V), _f64(a)
    N = len(e) - 1
    v, h, eps, O = np.zeros((N, N)), np.zeros((N, N)), np.zeros(N), np.zeros((N, N))
    st = lib().orc_pair(N, _p(e), n_nodes, l, len(V), _p(V), _p(a), _p(v), _p(h), _p(eps), _p(O))
    assert st == OK, st
    return v, h, eps, O


# --------------------------------------------------------------------------
# P0
# --------------------------------------------------------------------------
def n_pairs(n_ch: int) -> int:
    return lib().orc_n_pairs(n_ch)


def pair_list(n_ch: int):
    return [(l, lp) for l in range(n_ch) for lp in range(n_ch) if (l + lp) % 2 == 0]


def P0(pe, qe, n_p, n_q, n_x, n_ch, normalize=True, with_outgrid=False, with_abs=False):
    """Node-binned lattice P0 as block-CSR over cells.

    Returns dict(row_ptr int64[N*M+1], col int32[nnz], val f64[nnz, n_pairs],
    outgrid f64[N*M, n_pairs] (unnormalised, optional), absval f64[nnz,
    n_pairs] (sum over the element's nodes of W |P_l(y)|, the magnitude that
    bounds every node term, normalised like val, optional)).
    """
    pe, qe = _f64(pe), _f64(qe)
    N, M = len(pe) - 1, len(qe) - 1
    rp = np.zeros(N * M + 1, dtype=np.int64)
    nnz = lib().orc_P0_count(N, _p(pe), M, _p(qe), n_p, n_q, n_x, _p(rp, _I64))
    assert nnz >= 0, nnz
    npair = n_pairs(n_ch)
    col = np.zeros(max(nnz, 1), dtype=np.int32)
    val = np.zeros((max(nnz, 1), npair))
    og = np.zeros((N * M, npair)) if with_outgrid else None
    av = np.zeros((max(nnz, 1), npair)) if with_abs else None
    st = lib().orc_P0_fill(N, _p(pe), M, _p(qe), n_p, n_q, n_x, n_ch, _p(rp, _I64), _p(col, _I32),
                           _p(val), _p(og), _p(av))
    assert st == OK, st
    if normalize:
        lib().orc_P0_normalize(N, _p(pe), M, _p(qe), n_ch, _p(rp, _I64), _p(col, _I32), _p(val))
        if with_abs:
            lib().orc_P0_normalize(N, _p(pe), M, _p(qe), n_ch, _p(rp, _I64), _p(col, _I32), _p(av))
    out = dict(row_ptr=rp, col=col[:nnz], val=val[:nnz], N=N, M=M, n_ch=n_ch)
    if with_abs:
        out["absval"] = av[:nnz]
    if with_outgrid:
        out["outgrid"] = og
    return out


def P0_vl(pe, qe, n_p, n_q, n_x, n_ch, normalize=True, with_outgrid=False):
    """P0 with variable limits: for every (p, q) node of a source cell and
    every target cell, the y-interval on which p' and q' lie in the target's
    bins (limits where p'^2, q'^2, linear in y, equal squared bin edges),
    integrated by the n_x-point GL rule mapped onto it; block-CSR like P0()."""
    pe, qe = _f64(pe), _f64(qe)
    N, M = len(pe) - 1, len(qe) - 1
    rp = np.zeros(N * M + 1, dtype=np.int64)
    nnz = lib().orc_P0_vl_count(N, _p(pe), M, _p(qe), n_p, n_q, n_x, _p(rp, _I64))
    assert nnz >= 0, nnz
    npair = n_pairs(n_ch)
    col = np.zeros(max(nnz, 1), dtype=np.int32)
    val = np.zeros((max(nnz, 1), npair))
    og = np.zeros((N * M, npair)) if with_outgrid else None
    st = lib().orc_P0_vl_fill(N, _p(pe), M, _p(qe), n_p, n_q, n_x, n_ch, _p(rp, _I64), _p(col, _I32),
                              _p(val), _p(og))
    assert st == OK, st
    if normalize:
        lib().orc_P0_normalize(N, _p(pe), M, _p(qe), n_ch, _p(rp, _I64), _p(col, _I32), _p(val))
    out = dict(row_ptr=rp, col=col[:nnz], val=val[:nnz], N=N, M=M, n_ch=n_ch)
    if with_outgrid:
        out["outgrid"] = og
    return out


def P0_node_totals(pe, qe, n_p, n_q, n_x, n_ch):
    pe, qe = _f64(pe), _f64(qe)
    N, M = len(pe) - 1, len(qe) - 1
    tot = np.zeros((N * M, n_pairs(n_ch)))
    assert lib().orc_P0_node_totals(N, _p(pe), M, _p(qe), n_p, n_q, n_x, n_ch, _p(tot)) == OK
    return tot


def P0_dense(P):
    """Dense matrix [n_ch*N*M]^2 of a block-CSR P0 (small cases only)."""
    N, M, n_ch = P["N"], P["M"], P["n_ch"]
    nc = N * M
    D = np.zeros((n_ch * nc, n_ch * nc))
    rows = np.repeat(np.arange(nc), np.diff(P["row_ptr"]))
    for k, (l, lp) in enumerate(pair_list(n_ch)):
        np.add.at(D, (l * nc + rows, lp * nc + P["col"]), P["val"][:, k])
    return D


def bnorm(e):
    e = np.asarray(e, dtype=np.float64)
    lo, hi = e[:-1], e[1:]
    return (hi - lo) * (hi * hi + hi * lo + lo * lo) / 3.0


# --------------------------------------------------------------------------
# resolvent and solve
# --------------------------------------------------------------------------
def onshell(qe, E, eps_b):
    qe = _f64(qe)
    j0 = ctypes.c_int()
    Elo, Ehi, q0 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = lib().orc_onshell(len(qe) - 1, _p(qe), E, eps_b, ctypes.byref(j0), ctypes.byref(Elo),
                           ctypes.byref(Ehi), ctypes.byref(q0))
    if st != OK:
        raise ValueError(f"no on-shell bin for E={E} (status {st})")
    return j0.value, Elo.value, Ehi.value, q0.value


def G1(eps, qe, E, eps_b):
    """Channel resolvent as complex array [n_ch, N, M], plus j0 and D."""
    eps, qe = _f64(eps), _f64(qe)
    n_ch, N = eps.shape
    M = len(qe) - 1
    g = np.zeros(2 * n_ch * N * M)
    j0, D = ctypes.c_int(), ctypes.c_double()
    st = lib().orc_G1(n_ch, N, _p(eps), M, _p(qe), E, eps_b, _p(g), ctypes.byref(j0), ctypes.byref(D))
    if st != OK:
        raise ValueError(f"G1 failed for E={E} (status {st})")
    return g.view(np.complex128).reshape(n_ch, N, M), j0.value, D.value


class Problem:
    """Everything the solve needs, built by the oracle alone.

    desc keys: pe, qe (edges), n_p, n_q, n_x, n_ch, V, a (potential terms),
    n_pair_nodes.
    """

    def __init__(self, desc, P=None):
        self.desc = dict(desc)
        pe, qe = _f64(desc["pe"]), _f64(desc["qe"])
        self.pe, self.qe = pe, qe
        self.N, self.M, self.n_ch = len(pe) - 1, len(qe) - 1, int(desc["n_ch"])
        N, M, n_ch = self.N, self.M, self.n_ch
        self.v = np.zeros((n_ch, N, N))
        self.O = np.zeros((n_ch, N, N))
        self.eps = np.zeros((n_ch, N))
        for l in range(n_ch):
            v, _, eps, O = pair(pe, desc["n_pair_nodes"], l, desc["V"], desc["a"])
            self.v[l], self.O[l], self.eps[l] = v, O, eps
        # Vt = O^T V1 in the channel basis = v O^T per channel
        self.Vt = np.ascontiguousarray(np.einsum("lij,lkj->lik", self.v, self.O))
        self.eps_b = float(self.eps[0, 0])
        self.P = P if P is not None else P0(pe, qe, desc["n_p"], desc["n_q"], desc["n_x"], n_ch)
        self.dim = n_ch * N * M

    def _args(self):
        P = self.P
        return (self.n_ch, self.N, self.M, _p(self.O), _p(self.Vt), _p(P["row_ptr"], _I64),
                _p(np.ascontiguousarray(P["col"]), _I32), _p(np.ascontiguousarray(P["val"])))

    def G1(self, E):
        return G1(self.eps, self.qe, E, self.eps_b)

    def kapply(self, x, g=None):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        out = np.zeros(self.dim, dtype=np.complex128)
        gp = None if g is None else np.ascontiguousarray(g, dtype=np.complex128)
        lib().orc_kapply(*self._args(), None if gp is None else gp.ctypes.data_as(_D),
                         x.ctypes.data_as(_D), out.ctypes.data_as(_D))
        return out

    def r0(self, j0):
        return j0  # channel 0, k = 0 (bound state), q-bin j0

    def born(self, j0):
        e0 = np.zeros(self.dim, dtype=np.complex128)
        e0[self.r0(j0)] = 1.0
        return self.kapply(e0)

    def solve_wynn(self, E, min_iter=4, max_iter=100, tol=1e-12, return_c=False):
        g, j0, D = self.G1(E)
        gp = np.ascontiguousarray(g.reshape(-1))
        U = np.zeros(2)
        nt = ctypes.c_int()
        c = np.zeros(2 * max_iter)
        st = lib().orc_solve_wynn(*self._args(), gp.ctypes.data_as(_D), self.r0(j0), min_iter, max_iter,
                                  tol, _p(U), ctypes.byref(nt), _p(c))
        res = dict(U00=complex(U[0], U[1]), n_terms=nt.value, status=st, j0=j0, D=D)
        if return_c:
            res["c"] = c[: 2 * nt.value].view(np.complex128)
        return res

    def solve_gmres(self, E, b=None, u0=None, max_iter=200, tol=1e-10):
        g, j0, D = self.G1(E)
        gp = np.ascontiguousarray(g.reshape(-1))
        if b is None:
            b = self.born(j0)
        b = np.ascontiguousarray(b, dtype=np.complex128)
        u = np.zeros(self.dim, np.complex128) if u0 is None else np.array(u0, dtype=np.complex128)
        nk = ctypes.c_int()
        rr = ctypes.c_double()
        st = lib().orc_solve_gmres(*self._args(), gp.ctypes.data_as(_D), b.ctypes.data_as(_D),
                                   u.ctypes.data_as(_D), max_iter, tol, ctypes.byref(nk),
                                   ctypes.byref(rr))
        return dict(u=u, U00=complex(u[self.r0(j0)]), n_kapply=nk.value, relres=rr.value,
                    status=st, j0=j0, D=D)

    def amplitudes(self, E, U00):
        """S = 1 - 2 pi i U00 / D and the paper's A = (2/(3 q0)) U00 / dq_j0."""
        j0, Elo, Ehi, q0 = onshell(self.qe, E, self.eps_b)
        D = Ehi - Elo
        S = 1.0 - 2j * np.pi * U00 / D
        A = 2.0 / (3.0 * q0) * U00 / (self.qe[j0 + 1] - self.qe[j0])
        return S, A

    def dense_K(self, E):
        """Dense K = O P0 Vt G1 (small cases only; for the LU pin)."""
        N, M, n_ch = self.N, self.M, self.n_ch
        n = self.dim
        Ob = np.zeros((n, n))
        Vb = np.zeros((n, n))
        for ch in range(n_ch):
            for j in range(M):
                idx = ch * N * M + np.arange(N) * M + j
                Ob[np.ix_(idx, idx)] = self.O[ch]
                Vb[np.ix_(idx, idx)] = self.Vt[ch]
        g, j0, D = self.G1(E)
        Pd = P0_dense(self.P)
        K = Ob @ Pd @ Vb @ np.diag(g.reshape(-1))
        u0 = Ob @ Pd @ Vb[:, self.r0(j0)]
        return K, u0, j0, D


# --------------------------------------------------------------------------
# exact cell-overlap integral (brute force, tiny grids only)
# --------------------------------------------------------------------------
def exact_overlap(pe, qe, c, t, l, lp, n_y=48, epsrel=1e-11):
    """Exact unnormalised cell overlap
    int_{cell c} p^2 dp q^2 dq int_{-1}^{1} dy P_l(y) P_l'(y') theta(target t)
    (zero for l + l' odd), the quantity the node sum of ``P0(...,
    normalize=False)`` estimates.  A different route from the node binning:
    for fixed (p, q) the squared momenta p'^2 = Bp + A y and q'^2 = Dq - C y are
    linear in y, so the y that land in target t form one clipped interval,
    integrated with an n_y-point GL rule.  The (p, q) integral is nested
    adaptive quadrature (QUADPACK) with the kinks of the clipped interval
    passed as break points: they lie where a recoupled momentum reaches a
    target edge at y = +-1, |p/2 +- 3q/4| = e and |p -+ q/2| = f, and where the
    two constraints meet, which by energy conservation is
    p^2 + 3q^2/4 = e^2 + 3f^2/4 (e, f the target's p and q edges).
    """
    from numpy.polynomial import legendre as npl
    from scipy import integrate

    if (l + lp) % 2:
        return 0.0
    pe, qe = np.asarray(pe, float), np.asarray(qe, float)
    M = len(qe) - 1
    i, j = divmod(c, M)
    it, jt = divmod(t, M)
    ty, wy = npl.leggauss(n_y)
    cl = np.zeros(l + 1)
    cl[l] = 1
    clp = np.zeros(lp + 1)
    clp[lp] = 1
    plo, phi = pe[it], pe[it + 1]
    qlo, qhi = qe[jt], qe[jt + 1]
    pa, pb, qa, qb = pe[i], pe[i + 1], qe[j], qe[j + 1]
    E_edges = [plo, phi]
    F_edges = [qlo, qhi]

    def y_integral(p, q):
        A = 0.75 * p * q
        Bp = 0.25 * p * p + 0.5625 * q * q
        C = p * q
        Dq = p * p + 0.25 * q * q
        ya = max(-1.0, (plo * plo - Bp) / A, (Dq - qhi * qhi) / C)
        yb = min(1.0, (phi * phi - Bp) / A, (Dq - qlo * qlo) / C)
        if yb <= ya:
            return 0.0
        y = 0.5 * (yb - ya) * ty + 0.5 * (yb + ya)
        p2 = Bp + A * y
        q2 = Dq - C * y
        yp = np.clip((-0.5 * p * p - 0.5 * p * q * y + 0.375 * q * q) / np.sqrt(p2 * q2), -1, 1)
        f = npl.legval(y, cl) * npl.legval(yp, clp)
        return p * p * q * q * 0.5 * (yb - ya) * np.dot(wy, f)

    def q_kinks(p):
        pts = []
        for e in E_edges:
            pts += [4.0 / 3.0 * (e - p / 2), 4.0 / 3.0 * (p / 2 - e), 4.0 / 3.0 * (e + p / 2)]
            for f in F_edges:
                a2 = (e * e + 0.75 * f * f - p * p) / 0.75
                if a2 > 0:
                    pts.append(np.sqrt(a2))
        for f in F_edges:
            pts += [2.0 * (p - f), 2.0 * (f - p), 2.0 * (p + f)]
        return sorted(x for x in pts if qa < x < qb)

    def p_kinks():
        pts = []
        for q in (qa, qb):
            for e in E_edges:
                pts += [2 * e - 1.5 * q, 1.5 * q - 2 * e, 2 * e + 1.5 * q]
                for f in F_edges:
                    a2 = e * e + 0.75 * f * f - 0.75 * q * q
                    if a2 > 0:
                        pts.append(np.sqrt(a2))
            for f in F_edges:
                pts += [f + q / 2, f - q / 2, q / 2 - f]
        return sorted(x for x in pts if pa < x < pb)

    def outer(p):
        v, _ = integrate.quad(lambda q: y_integral(p, q), qa, qb, points=q_kinks(p) or None,
                              epsabs=0.0, epsrel=epsrel, limit=200)
        return v

    val, _ = integrate.quad(outer, pa, pb, points=p_kinks() or None, epsabs=0.0, epsrel=epsrel,
                            limit=200)
    return val
