"""Build of the in-tree CUDA library ``libwpcd.so`` (sm_103a only).

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into a shared library next to this file.  No cmake, no torch
extension machinery: the library is a plain C ABI (include/wpcd.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwpcd.so")
SOURCES = ["capi.cpp", "setup.cpp", "assemble.cu", "solve.cu", "group.cu", "tc_gemm.cu", "df.cu", "mlp.cu",
           "kapply_noalloc.cu", "spmm_tile.cu", "oz_gemm.cu", "spmv.cu",
           "assemble_vl.cu", "pair.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwpcd")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src, os.path.join(CSRC, "wpcd_internal.h"), os.path.join(CSRC, "common.cuh"),
            os.path.join(CSRC, "df_common.cuh"), os.path.join(CSRC, "tc_ptx.cuh"), os.path.join(CSRC, "bessel.h"),
            os.path.join(ROOT, "include", "wpcd.h"), os.path.abspath(__file__)]  # flags live here
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OUT_DIR, s + ".o")
        if force or _stale(obj, src):
            cmd = [cc] + _flags() + ["-c", src, "-o", obj]
            if s.endswith(".cu"):
                cmd += ["-Xptxas", "-warn-spills"]
            else:  # host setup: OpenMP over the pair-matrix rows
                cmd += ["-Xcompiler", "-fopenmp"]
            jobs.append((s, cmd))
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        futs = {ex.submit(subprocess.run, cmd, capture_output=True, text=True): s for s, cmd in jobs}
        for f in cf.as_completed(futs):
            r = f.result()
            if verbose or r.returncode != 0:
                print(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {futs[f]}")
    objs = [os.path.join(OUT_DIR, s + ".o") for s in SOURCES]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-Xcompiler", "-fopenmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            print(r.stdout + r.stderr)
            raise RuntimeError("link of libwpcd.so failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
