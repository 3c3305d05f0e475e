"""The C ABI library (include/wpcd.h): it builds for sm_103a, loads, exports
every declared symbol, and rejects invalid input on the host before any
device work (no GPU needed for these)."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def W():
    from paper_1508_07441_gb300 import build, wpcd

    build.build()
    return wpcd


def test_exports_every_declared_symbol(W):
    L = W.lib()
    names = W.header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    assert L.wpcd_version() >= 100


def test_struct_layouts_match_header(W, tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's sizes."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "wpcd.h"\nint main(void){printf("%zu %zu %zu %zu %zu",'
                   'sizeof(wpcd_problem_desc), sizeof(wpcd_solve_opts), sizeof(wpcd_solve_stats),'
                   'sizeof(wpcd_grid_desc), sizeof(wpcd_pair_desc));}\n')
    exe = tmp_path / "sz"
    inc = W.HEADER.rsplit("/", 1)[0]
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    sizes = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert sizes == [ctypes.sizeof(W.wpcd_problem_desc), ctypes.sizeof(W.wpcd_solve_opts),
                     ctypes.sizeof(W.wpcd_solve_stats), ctypes.sizeof(W.wpcd_grid_desc),
                     ctypes.sizeof(W.wpcd_pair_desc)]


def _desc(W, N=4, M=4, **kw):
    pe = np.linspace(0, 3, N + 1)
    qe = np.linspace(0, 3, M + 1)
    args = dict(n_p=2, n_q=2, n_x=4, n_ch=1, V=np.array([-3.0]), a=np.array([1.0]), n_pair_nodes=4,
                device=0)
    args.update(kw)
    keep = [pe, qe, args["V"], args["a"]]
    d = W.wpcd_problem_desc(N, M, keep[0].ctypes.data_as(W._D), keep[1].ctypes.data_as(W._D),
                            args["n_p"], args["n_q"], args["n_x"], args["n_ch"], len(args["V"]),
                            keep[2].ctypes.data_as(W._D), keep[3].ctypes.data_as(W._D),
                            args["n_pair_nodes"], args["device"])
    return d, keep


@pytest.mark.parametrize("kw,needle", [
    (dict(n_ch=0), "n_ch"), (dict(n_ch=9), "n_ch"), (dict(n_p=0), "node"), (dict(n_x=300), "node"),
    (dict(a=np.array([-1.0])), "a_k"), (dict(V=np.array([np.nan])), "finite"),
    (dict(n_pair_nodes=0), "n_pair_nodes"),
])
def test_create_rejects_invalid_input(W, kw, needle):
    d, keep = _desc(W, **kw)
    h = ctypes.c_void_p()
    st = W.lib().wpcd_problem_create(ctypes.byref(d), ctypes.byref(h))
    assert st == W.WPCD_EINVAL
    assert needle in W.last_error()
    assert not h.value


def test_create_rejects_bad_edges(W):
    d, keep = _desc(W)
    keep[0][2] = keep[0][1]  # not strictly increasing
    h = ctypes.c_void_p()
    assert W.lib().wpcd_problem_create(ctypes.byref(d), ctypes.byref(h)) == W.WPCD_EINVAL
    assert "edges" in W.last_error()


def test_tangent_edges_host_call(W):
    e = W.wpcd_tangent_edges(30, 20.0)
    assert e[0] == 0 and e[-1] == 20.0 and np.all(np.diff(e) > 0)
    with pytest.raises(W.WpcdError):
        W.wpcd_tangent_edges(0, 20.0)


def test_null_handles_are_rejected(W):
    L = W.lib()
    assert L.wpcd_problem_info(None, None, None, None) == W.WPCD_EINVAL
    assert L.wpcd_P_info(None, None, None, None, None) == W.WPCD_EINVAL
    assert L.wpcd_solve(None, None, None, 0, None, None, None, None) == W.WPCD_EINVAL
    L.wpcd_problem_destroy(None)
    L.wpcd_P_destroy(None)


def test_set_allocator_argument_checks(W):
    """wpcd_set_allocator takes both callbacks or neither (host-only check);
    restoring the library's own allocator with nothing live succeeds."""
    L = W.lib()
    cb = W._ALLOC_FN(lambda n, dev, s, u: None)
    assert L.wpcd_set_allocator(ctypes.cast(cb, ctypes.c_void_p), None, None) == W.WPCD_EINVAL
    assert "both" in W.last_error()
    assert L.wpcd_set_allocator(None, None, None) == W.WPCD_OK


def test_wait_limit_knob_argument_checks(W):
    """the test knob of the tensor-core wait-limit path takes kernel 1 with
    roles 0-3, kernel 2 with role 0, and kernel 0 (clear); nothing else"""
    L = W.lib()
    for kernel, role in ((1, 4), (1, -1), (2, 1), (3, 0), (-1, 0)):
        assert L.wpcd_debug_expire_first_wait(kernel, role) == W.WPCD_EINVAL, (kernel, role)
    for kernel, role in ((1, 0), (1, 3), (2, 0), (0, 0)):
        assert L.wpcd_debug_expire_first_wait(kernel, role) == W.WPCD_OK, (kernel, role)


def test_warm_softmax_argument_checks(W):
    L = W.lib()
    for n, k in ((0, 4), (4, 0), (4, 1025)):
        assert L.wpcd_warm_softmax(None, n, k, None, None) == W.WPCD_EINVAL


def test_split_argument_checks(W):
    L = W.lib()
    assert L.wpcd_split_f64(None, 4, None, None, None) == W.WPCD_EINVAL
    assert L.wpcd_split_f64(1, -1, 1, 1, None) == W.WPCD_EINVAL
    assert L.wpcd_split_f64(1, 0, 1, 1, None) == W.WPCD_OK  # nothing to do, nothing launched


def test_no_cpu_fallback_when_library_missing(W, monkeypatch, tmp_path):
    monkeypatch.setattr(W, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(W, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU path"):
        W.lib()


def test_grid_and_pair_reject_invalid_input(W):
    """wpcd_grid_create, wpcd_pair_create and wpcd_assemble_P_grid validate
    their arguments on the host (EINVAL) before any device call."""
    L = W.lib()
    h = ctypes.c_void_p()
    pe = np.array([0.0, 1.0, 0.5])  # not increasing
    qe = np.linspace(0, 3, 5)
    d = W.wpcd_grid_desc(2, 4, pe.ctypes.data_as(W._D), qe.ctypes.data_as(W._D), 2, 2, 4, 0)
    assert L.wpcd_grid_create(ctypes.byref(d), ctypes.byref(h)) == W.WPCD_EINVAL
    assert "edges" in W.last_error()
    d = W.wpcd_grid_desc(4, 4, qe.ctypes.data_as(W._D), qe.ctypes.data_as(W._D), 0, 2, 4, 0)
    assert L.wpcd_grid_create(ctypes.byref(d), ctypes.byref(h)) == W.WPCD_EINVAL
    V, a = np.array([-3.0]), np.array([1.0])
    pd = W.wpcd_pair_desc(3, 1, V.ctypes.data_as(W._D), a.ctypes.data_as(W._D), 8)
    assert L.wpcd_pair_create(None, ctypes.byref(pd), ctypes.byref(h)) == W.WPCD_EINVAL
    assert L.wpcd_assemble_P_grid(None, 3, W.WPCD_FP64, None, ctypes.byref(h)) == W.WPCD_EINVAL
