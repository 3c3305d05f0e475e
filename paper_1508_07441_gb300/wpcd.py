"""Thin ctypes binding of the C ABI in include/wpcd.h (argument marshalling only).

Every computation happens in ``libwpcd.so`` (sm_103a CUDA kernels and the
library's host setup).  Loading fails loudly when the library is missing: there
is no CPU fallback.  Device buffers are torch tensors (``data_ptr()``); streams
are torch streams (``cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwpcd.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "wpcd.h")

WPCD_OK, WPCD_EINVAL, WPCD_ENOMEM, WPCD_ECUDA = 0, -1, -2, -3
WPCD_ENOCONV, WPCD_EBREAKDOWN, WPCD_ETIMEOUT, WPCD_ENOBOUND = -4, -5, -6, -7
WPCD_FP64, WPCD_FP32C, WPCD_FP64_VL = 0, 1, 2
WPCD_SUM_KRYLOV, WPCD_SUM_WYNN = 0, 1
WPCD_SOLVE_FP64, WPCD_SOLVE_MIXED, WPCD_SOLVE_MIXED_FP64 = 0, 1, 2
WPCD_GEMM_FP64, WPCD_GEMM_FP32, WPCD_GEMM_TF32X3, WPCD_GEMM_FF, WPCD_GEMM_DIGITS = 0, 1, 2, 3, 4
WPCD_SPMM_FP64, WPCD_SPMM_FP32, WPCD_SPMM_FF, WPCD_SPMM_FP32_BLOCKED = 0, 1, 2, 3

_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)
_F = ctypes.POINTER(ctypes.c_float)


class wpcd_problem_desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("p_edges", _D), ("q_edges", _D),
                ("n_p", ctypes.c_int), ("n_q", ctypes.c_int), ("n_x", ctypes.c_int),
                ("n_ch", ctypes.c_int), ("n_terms", ctypes.c_int), ("V", _D), ("a", _D),
                ("n_pair_nodes", ctypes.c_int), ("device", ctypes.c_int)]


class wpcd_grid_desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("p_edges", _D), ("q_edges", _D),
                ("n_p", ctypes.c_int), ("n_q", ctypes.c_int), ("n_x", ctypes.c_int), ("device", ctypes.c_int)]


class wpcd_pair_desc(ctypes.Structure):
    _fields_ = [("n_ch", ctypes.c_int), ("n_terms", ctypes.c_int), ("V", _D), ("a", _D),
                ("n_pair_nodes", ctypes.c_int)]


class wpcd_solve_opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("max_iter", ctypes.c_int), ("min_iter", ctypes.c_int),
                ("tol", ctypes.c_double), ("check_every", ctypes.c_int), ("precision", ctypes.c_int),
                ("batch", ctypes.c_int), ("inner_iter", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("u_init", _P), ("u_out", _P)]


class wpcd_solve_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n_kapply", ctypes.c_int), ("j0", ctypes.c_int),
                ("D", ctypes.c_double), ("relres", ctypes.c_double),
                ("U00", ctypes.c_double * 2), ("S", ctypes.c_double * 2), ("A", ctypes.c_double * 2),
                ("ms", ctypes.c_float), ("n_kapply32", ctypes.c_int), ("n_outer", ctypes.c_int),
                ("warm_fallback", ctypes.c_int)]


_SIGS = {
    "wpcd_last_error": (ctypes.c_char_p, []),
    "wpcd_version": (ctypes.c_int, []),
    "wpcd_launch_count": (ctypes.c_int64, []),
    "wpcd_debug_expire_first_wait": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "wpcd_set_allocator": (ctypes.c_int, [_P, _P, _P]),
    "wpcd_P_timing": (ctypes.c_int, [_P, _F]),
    "wpcd_P_work": (ctypes.c_int, [_P, _I64]),
    "wpcd_tangent_edges": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, _D]),
    "wpcd_problem_create": (ctypes.c_int, [ctypes.POINTER(wpcd_problem_desc), ctypes.POINTER(_P)]),
    "wpcd_problem_destroy": (None, [_P]),
    "wpcd_problem_info": (ctypes.c_int, [_P, _I, _I, _D]),
    "wpcd_problem_pair": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, _D]),
    "wpcd_assemble_P": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "wpcd_grid_create": (ctypes.c_int, [ctypes.POINTER(wpcd_grid_desc), ctypes.POINTER(_P)]),
    "wpcd_grid_destroy": (None, [_P]),
    "wpcd_pair_create": (ctypes.c_int, [_P, ctypes.POINTER(wpcd_pair_desc), ctypes.POINTER(_P)]),
    "wpcd_assemble_P_grid": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "wpcd_problem_grid": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "wpcd_P_destroy": (None, [_P]),
    "wpcd_P_info": (ctypes.c_int, [_P, _I64, _I, _I, _F]),
    "wpcd_P_export": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "wpcd_resolvent": (ctypes.c_int, [_P, _D, ctypes.c_int, _P, _I, _D, _P]),
    "wpcd_kapply": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "wpcd_solve": (ctypes.c_int, [_P, _P, _D, ctypes.c_int, ctypes.POINTER(wpcd_solve_opts), _D,
                                  ctypes.POINTER(wpcd_solve_stats), _P]),
    "wpcd_solve_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                        ctypes.POINTER(_D), _I, ctypes.POINTER(wpcd_solve_opts),
                                        ctypes.POINTER(_D), ctypes.POINTER(ctypes.POINTER(wpcd_solve_stats)),
                                        _P]),
    "wpcd_tune_spmm": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _P, _I, _I, _I]),
    "wpcd_channel_gemm": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P, ctypes.c_int, _F, _P]),
    "wpcd_spmm": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, ctypes.c_int, _F, _P]),
    "wpcd_born": (ctypes.c_int, [_P, _P, _D, ctypes.c_int, _P, _P]),
    "wpcd_kapply_noalloc": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "wpcd_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                       ctypes.c_int, ctypes.POINTER(_P)]),
    "wpcd_mlp_destroy": (None, [_P]),
    "wpcd_mlp_info": (ctypes.c_int, [_P, _I64, _I, _I, _I]),
    "wpcd_mlp_params": (ctypes.c_int, [_P, _P, _P]),
    "wpcd_mlp_set_affine": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "wpcd_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int, _P]),
    "wpcd_mlp_loss_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _F, _P, _P]),
    "wpcd_mlp_train": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_float, ctypes.c_uint64, _F, _P]),
    "wpcd_basis_project": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, _P]),
    "wpcd_basis_expand": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, _P]),
    "wpcd_basis_orthonormalize": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P]),
    "wpcd_warm_softmax": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "wpcd_warm_features": (ctypes.c_int, [_P, _D, ctypes.c_int, ctypes.c_double, ctypes.c_double, _P,
                                          ctypes.c_int, ctypes.c_int, _P, _P]),
    "wpcd_vec_axpy": (ctypes.c_int, [ctypes.c_double, _P, _P, ctypes.c_int64, _P]),
    "wpcd_complex_to_f32": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P]),
    "wpcd_split_f64": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P]),
}

_lib = None


class WpcdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"wpcd status {status}: {msg}")
        self.status = status


def lib():
    """Load libwpcd.so (raises if it has not been built: no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                               "(the CUDA library is required; there is no CPU path)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_functions():
    """Names of the functions declared in include/wpcd.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(wpcd_\w+)\s*\(", txt)))


def last_error() -> str:
    return lib().wpcd_last_error().decode()


def check(status: int, allow=()):
    if status != WPCD_OK and status not in allow:
        raise WpcdError(status, last_error())
    return status


def _dp(a):
    return a.ctypes.data_as(_D)


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _tensor_ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# same names as the C ABI
# ---------------------------------------------------------------------------
def wpcd_launch_count() -> int:
    return int(lib().wpcd_launch_count())


def wpcd_debug_expire_first_wait(kernel: int, role: int = 0):
    """Test knob: the first wait of `role` in every launch of tensor-core GEMM
    `kernel` (1 warp-specialised TF32x3, 2 digit-plane) runs out at once, so
    the operation returns WPCD_ETIMEOUT on valid input; kernel 0 clears it."""
    check(lib().wpcd_debug_expire_first_wait(kernel, role))


# device allocator callbacks: alloc(bytes, device, stream, user) -> pointer,
# free(pointer, stream, user)
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_hooks = None  # the installed callbacks, kept alive while installed


def wpcd_set_allocator(alloc=None, free=None):
    """Route every device allocation of the library through Python callables
    alloc(nbytes, device, stream) -> int pointer and free(pointer, stream)
    (stream: a cudaStream_t as int, 0 for the legacy default stream), or back
    to the library's own allocator with both None.  Set it before creating
    handles or after destroying them (the library refuses otherwise)."""
    global _hooks
    if alloc is None and free is None:
        check(lib().wpcd_set_allocator(None, None, None))
        _hooks = None
        return
    a = _ALLOC_FN(lambda n, dev, s, u: int(alloc(int(n), int(dev), int(s or 0))) or None)
    f = _FREE_FN(lambda p, s, u: free(int(p), int(s or 0)))
    check(lib().wpcd_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None))
    _hooks = (a, f)


def use_torch_allocator(enable=True):
    """Take the library's device memory from PyTorch's caching allocator on
    the stream of each request (enable=False: back to the library's own)."""
    if not enable:
        wpcd_set_allocator(None, None)
        return
    import torch

    def alloc(nbytes, device, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, device=device, stream=stream)

    def free(ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    wpcd_set_allocator(alloc, free)


def wpcd_solve_batch(problems, Ps, energies, max_iter=100, tol=1e-10, check_every=4,
                     precision=WPCD_SOLVE_FP64, inner_iter=0, max_outer=0, use_graph=1, stream=None,
                     allow=(WPCD_ENOCONV, WPCD_EBREAKDOWN)):
    """Grouped solve of several problems (uneven grids) in one iteration.
    problems, Ps: sequences of Problem / PMatrix; energies: sequence of
    arrays.  Returns (list of complex U00 arrays, list of stats lists, status)."""
    n = len(problems)
    if len(Ps) != n or len(energies) != n:
        raise ValueError("problems, Ps and energies must have the same length")
    Es = [np.ascontiguousarray(np.atleast_1d(e), dtype=np.float64) for e in energies]
    Us = [np.zeros(2 * len(e)) for e in Es]
    stats = [(wpcd_solve_stats * len(e))() for e in Es]
    hp = (_P * n)(*[p.handle for p in problems])
    hP = (_P * n)(*[P.handle for P in Ps])
    hE = (_D * n)(*[_dp(e) for e in Es])
    hU = (_D * n)(*[_dp(u) for u in Us])
    hS = (ctypes.POINTER(wpcd_solve_stats) * n)(
        *[ctypes.cast(st, ctypes.POINTER(wpcd_solve_stats)) for st in stats])
    nE = (ctypes.c_int * n)(*[len(e) for e in Es])
    opts = wpcd_solve_opts(WPCD_SUM_KRYLOV, max_iter, 4, tol, check_every, precision, 0,
                           inner_iter, max_outer, use_graph, None, None)
    st = lib().wpcd_solve_batch(n, hp, hP, hE, nE, ctypes.byref(opts), hU, hS, _stream_ptr(stream))
    check(st, allow=allow)
    return [u.view(np.complex128) for u in Us], [list(x) for x in stats], st


def wpcd_tangent_edges(n_bins: int, k_max: float) -> np.ndarray:
    e = np.zeros(n_bins + 1)
    check(lib().wpcd_tangent_edges(n_bins, k_max, _dp(e)))
    return e


class Grid:
    """Handle of wpcd_grid: the packet lattice and its quadrature tables,
    all that P0 depends on."""

    def __init__(self, p_edges, q_edges, n_p, n_q, n_x, device=0):
        self.pe = np.ascontiguousarray(p_edges, dtype=np.float64)
        self.qe = np.ascontiguousarray(q_edges, dtype=np.float64)
        self.N, self.M = len(self.pe) - 1, len(self.qe) - 1
        d = wpcd_grid_desc(self.N, self.M, _dp(self.pe), _dp(self.qe), n_p, n_q, n_x, device)
        h = _P()
        self._h = None
        check(lib().wpcd_grid_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None:
            lib().wpcd_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def wpcd_assemble_P(self, n_ch, prec=WPCD_FP64, stream=None) -> "PMatrix":
        """P0 of this lattice for n_ch channels, usable with every Problem made
        on the grid with n_ch channels."""
        h = _P()
        check(lib().wpcd_assemble_P_grid(self._h, n_ch, prec, _stream_ptr(stream), ctypes.byref(h)))
        return PMatrix(h, self)

    def wpcd_pair_create(self, V, a, n_ch, n_pair_nodes=8) -> "Problem":
        """A Problem (this grid + the pair setup of V(r) = sum V_k exp(-r^2/a_k))."""
        return Problem.on_grid(self, V, a, n_ch, n_pair_nodes)


class Problem:
    """Handle of wpcd_problem (step 1 of the scheme, done by the library)."""

    def __init__(self, p_edges, q_edges, n_p, n_q, n_x, n_ch, V, a, n_pair_nodes=8, device=0):
        self._keep = [np.ascontiguousarray(x, dtype=np.float64) for x in (p_edges, q_edges, V, a)]
        pe, qe, Vv, av = self._keep
        d = wpcd_problem_desc(len(pe) - 1, len(qe) - 1, _dp(pe), _dp(qe), n_p, n_q, n_x, n_ch,
                              len(Vv), _dp(Vv), _dp(av), n_pair_nodes, device)
        h = _P()
        self._h = None
        check(lib().wpcd_problem_create(ctypes.byref(d), ctypes.byref(h)))
        self._init(h, pe, qe, n_ch)

    @classmethod
    def on_grid(cls, grid, V, a, n_ch, n_pair_nodes=8):
        """The pair setup on an existing grid (wpcd_pair_create)."""
        self = cls.__new__(cls)
        self._keep = [np.ascontiguousarray(x, dtype=np.float64) for x in (V, a)]
        Vv, av = self._keep
        d = wpcd_pair_desc(n_ch, len(Vv), _dp(Vv), _dp(av), n_pair_nodes)
        h = _P()
        self._h = None
        check(lib().wpcd_pair_create(grid.handle, ctypes.byref(d), ctypes.byref(h)))
        self._init(h, grid.pe, grid.qe, n_ch)
        return self

    def _init(self, h, pe, qe, n_ch):
        self._h = h
        self.N, self.M, self.n_ch = len(pe) - 1, len(qe) - 1, n_ch
        self.pe, self.qe = pe, qe
        dim, npair, eb = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        check(lib().wpcd_problem_info(h, ctypes.byref(dim), ctypes.byref(npair), ctypes.byref(eb)))
        self.dim, self.n_pairs, self.eps_bound = dim.value, npair.value, eb.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None:
            lib().wpcd_problem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def wpcd_problem_pair(self, l: int):
        N = self.N
        eps, O, v = np.zeros(N), np.zeros((N, N)), np.zeros((N, N))
        check(lib().wpcd_problem_pair(self._h, l, _dp(eps), _dp(O), _dp(v)))
        return eps, O, v

    def wpcd_assemble_P(self, prec=WPCD_FP64, stream=None) -> "PMatrix":
        h = _P()
        check(lib().wpcd_assemble_P(self._h, prec, _stream_ptr(stream), ctypes.byref(h)))
        return PMatrix(h, self)

    def wpcd_resolvent(self, E, g, stream=None):
        """g: device tensor (float64) of >= 2 * len(E) * dim elements."""
        E = np.ascontiguousarray(np.atleast_1d(E), dtype=np.float64)
        j0 = np.zeros(len(E), dtype=np.int32)
        D = np.zeros(len(E))
        check(lib().wpcd_resolvent(self._h, _dp(E), len(E), _tensor_ptr(g),
                                   j0.ctypes.data_as(_I), _dp(D), _stream_ptr(stream)))
        return j0, D

    def wpcd_kapply(self, P, g, x, y, stream=None):
        check(lib().wpcd_kapply(self._h, P.handle, _tensor_ptr(g), _tensor_ptr(x), _tensor_ptr(y),
                                _stream_ptr(stream)))

    def wpcd_kapply_noalloc(self, P, g, x, y, stream=None):
        """K application with the library's fixed device scratch (no device
        allocation); enqueued, not synchronised."""
        check(lib().wpcd_kapply_noalloc(self._h, P.handle, _tensor_ptr(g), _tensor_ptr(x),
                                        _tensor_ptr(y), _stream_ptr(stream)))

    def wpcd_solve(self, P, E, method=WPCD_SUM_KRYLOV, max_iter=100, min_iter=4, tol=1e-10,
                   check_every=4, precision=WPCD_SOLVE_FP64, batch=0, inner_iter=0, max_outer=0,
                   use_graph=1, u_init=None, u_out=None, stream=None,
                   allow=(WPCD_ENOCONV, WPCD_EBREAKDOWN)):
        """U00 per energy (complex array), per-energy stats, status.  u_init /
        u_out: device float64 tensors of 2 * len(E) * dim (energy-major)."""
        E = np.ascontiguousarray(np.atleast_1d(E), dtype=np.float64)
        U = np.zeros(2 * len(E))
        stats = (wpcd_solve_stats * len(E))()
        opts = wpcd_solve_opts(method, max_iter, min_iter, tol, check_every, precision, batch,
                               inner_iter, max_outer, use_graph,
                               None if u_init is None else u_init.data_ptr(),
                               None if u_out is None else u_out.data_ptr())
        st = lib().wpcd_solve(self._h, P.handle, _dp(E), len(E), ctypes.byref(opts), _dp(U), stats,
                              _stream_ptr(stream))
        check(st, allow=allow)
        return U.view(np.complex128), list(stats), st

    def wpcd_spmm(self, P, y, z, n_rhs, mode=WPCD_SPMM_FP64, stream=None, timed=False):
        """z = P0 y for n_rhs vectors (device tensors, batched layout).
        With timed, returns the SpMM kernel's device milliseconds."""
        ms = ctypes.c_float()
        check(lib().wpcd_spmm(self._h, P.handle, mode, _tensor_ptr(y), _tensor_ptr(z), n_rhs,
                              ctypes.byref(ms) if timed else None, _stream_ptr(stream)))
        return ms.value if timed else None

    def wpcd_channel_gemm(self, which, mode, g, x, y, n_rhs, stream=None, timed=False):
        """y = A (g o x) per channel block, A = Vt (which 0) or O (which 1);
        g, x, y device tensors in the batched layout (g may be None).  With
        timed, returns the product kernel's device milliseconds."""
        ms = ctypes.c_float()
        check(lib().wpcd_channel_gemm(self._h, which, mode, _tensor_ptr(g), _tensor_ptr(x), _tensor_ptr(y),
                                      n_rhs, ctypes.byref(ms) if timed else None, _stream_ptr(stream)))
        return ms.value if timed else None

    def wpcd_born(self, P, E, b, stream=None):
        """Born terms into device tensor b (float64, 2 * len(E) * dim)."""
        E = np.ascontiguousarray(np.atleast_1d(E), dtype=np.float64)
        check(lib().wpcd_born(self._h, P.handle, _dp(E), len(E), _tensor_ptr(b), _stream_ptr(stream)))

    def wpcd_tune_spmm(self, P, n_rhs, fp32=False, stream=None, mode=None):
        """(rows_per_warp, energy_lanes, energies_per_lane) chosen by timing;
        mode: WPCD_SPMM_* (default: FP32 if fp32 else FP64)."""
        m = (WPCD_SPMM_FP32 if fp32 else WPCD_SPMM_FP64) if mode is None else mode
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().wpcd_tune_spmm(self._h, P.handle, n_rhs, m, _stream_ptr(stream),
                                   ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value


class PMatrix:
    """Handle of wpcd_P (block-CSR P0 on the device); `problem` is the Problem
    or Grid it was assembled from (for the lattice sizes)."""

    def __init__(self, h, problem):
        self._h = h
        self.problem = problem
        nnz, npair, prec, ms = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        check(lib().wpcd_P_info(h, ctypes.byref(nnz), ctypes.byref(npair), ctypes.byref(prec),
                                ctypes.byref(ms)))
        self.nnz, self.n_pairs, self.prec, self.ms = nnz.value, npair.value, prec.value, ms.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None:
            lib().wpcd_P_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def wpcd_P_work(self):
        """Quadrature points the assembly evaluated."""
        n = ctypes.c_int64()
        check(lib().wpcd_P_work(self._h, ctypes.byref(n)))
        return n.value

    def wpcd_P_timing(self):
        """(count, scan, fill) device milliseconds of this assembly."""
        ms = (ctypes.c_float * 3)()
        check(lib().wpcd_P_timing(self._h, ms))
        return tuple(ms)

    def wpcd_P_export(self):
        """Host copies: row_ptr int64[N*M+1], col int32[nnz], val f64[n_pairs, nnz]."""
        pr = self.problem
        rp = np.zeros(pr.N * pr.M + 1, dtype=np.int64)
        col = np.zeros(max(self.nnz, 1), dtype=np.int32)
        val = np.zeros((self.n_pairs, max(self.nnz, 1)))
        check(lib().wpcd_P_export(self._h, ctypes.c_void_p(rp.ctypes.data),
                                  ctypes.c_void_p(col.ctypes.data), ctypes.c_void_p(val.ctypes.data),
                                  None))
        return rp, col[: self.nnz], val[:, : self.nnz]


class MLP:
    """Handle of wpcd_mlp (3-layer tanh MLP; training and inference kernels
    in the library)."""

    def __init__(self, n_in, width, n_out, seed=2026, device=0):
        h = _P()
        self._h = None
        check(lib().wpcd_mlp_create(n_in, width, n_out, seed, device, ctypes.byref(h)))
        self._h = h
        n = ctypes.c_int64()
        check(lib().wpcd_mlp_info(h, ctypes.byref(n), None, None, None))
        self.n_params, self.n_in, self.width, self.n_out = n.value, n_in, width, n_out

    def close(self):
        if self._h is not None:
            lib().wpcd_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def wpcd_mlp_params(self, get=None, set=None):
        """get / set: numpy float32 arrays or torch tensors of n_params."""
        def ptr(a):
            if a is None:
                return None
            return ctypes.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)
        check(lib().wpcd_mlp_params(self._h, ptr(get), ptr(set)))

    def wpcd_mlp_set_affine(self, in_scale=None, in_shift=None, out_scale=None, out_shift=None):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float32)
                for a in (in_scale, in_shift, out_scale, out_shift)]
        check(lib().wpcd_mlp_set_affine(self._h, *[None if a is None else ctypes.c_void_p(a.ctypes.data)
                                                   for a in arrs]))

    def wpcd_mlp_forward(self, X, Y, bf16=False, stream=None):
        check(lib().wpcd_mlp_forward(self._h, _tensor_ptr(X), X.shape[0], _tensor_ptr(Y),
                                     1 if bf16 else 0, _stream_ptr(stream)))

    def wpcd_mlp_loss_grad(self, X, T, grad=None, stream=None):
        loss = ctypes.c_float()
        check(lib().wpcd_mlp_loss_grad(self._h, _tensor_ptr(X), _tensor_ptr(T), X.shape[0],
                                       ctypes.byref(loss), _tensor_ptr(grad), _stream_ptr(stream)))
        return loss.value

    def wpcd_mlp_train(self, X, T, epochs, batch, lr, seed=2026, stream=None):
        hist = np.zeros(epochs, dtype=np.float32)
        check(lib().wpcd_mlp_train(self._h, _tensor_ptr(X), _tensor_ptr(T), X.shape[0], epochs, batch,
                                   lr, seed, hist.ctypes.data_as(_F), _stream_ptr(stream)))
        return hist


def wpcd_basis_project(Phi, k, dim, U, n, C, stream=None):
    check(lib().wpcd_basis_project(_tensor_ptr(Phi), k, dim, _tensor_ptr(U), n, _tensor_ptr(C),
                                   _stream_ptr(stream)))


def wpcd_basis_expand(Phi, k, dim, C, n, U, stream=None):
    check(lib().wpcd_basis_expand(_tensor_ptr(Phi), k, dim, _tensor_ptr(C), n, _tensor_ptr(U),
                                  _stream_ptr(stream)))


def wpcd_basis_orthonormalize(Phi, k, dim, stream=None):
    check(lib().wpcd_basis_orthonormalize(_tensor_ptr(Phi), k, dim, _stream_ptr(stream)))


def wpcd_split_f64(x, hi, lo, stream=None):
    """Float-float split of device float64 tensor x into float32 tensors hi, lo."""
    check(lib().wpcd_split_f64(_tensor_ptr(x), x.numel(), _tensor_ptr(hi), _tensor_ptr(lo), _stream_ptr(stream)))


def wpcd_warm_softmax(logits, n, k, C, stream=None):
    check(lib().wpcd_warm_softmax(_tensor_ptr(logits), n, k, _tensor_ptr(C), _stream_ptr(stream)))


def wpcd_warm_features(problem, E, e_lo, e_hi, Cb, k, kf, X, stream=None):
    E = np.ascontiguousarray(np.atleast_1d(E), dtype=np.float64)
    check(lib().wpcd_warm_features(problem.handle, _dp(E), len(E), e_lo, e_hi, _tensor_ptr(Cb), k, kf,
                                   _tensor_ptr(X), _stream_ptr(stream)))


def wpcd_vec_axpy(alpha, x, y, stream=None):
    """y += alpha x (device float64 tensors of equal size)."""
    check(lib().wpcd_vec_axpy(float(alpha), _tensor_ptr(x), _tensor_ptr(y), y.numel(), _stream_ptr(stream)))


def wpcd_complex_to_f32(src, n, dst, stream=None):
    check(lib().wpcd_complex_to_f32(_tensor_ptr(src), n, _tensor_ptr(dst), _stream_ptr(stream)))
