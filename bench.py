#!/usr/bin/env python
"""Benchmark of the WPCD Faddeev hot path on GB300.

One step = one pass of the whole hot path over the 3-channel workload
(three identical bosons, V = -3 exp(-r^2), l = lambda <= 2 coupled to L = 0,
N = M = 200 packet bins, 8 x 8 p,q nodes and 32 y nodes per cell, dimension
120 000): assemble P0 in FP64 (count, scan, fill), build G1 for a batch of
128 energies uniform in [-0.9 |E_d|, 5], and solve the matrix Faddeev
equation for all of them in one batched iteration (FP32 inner Krylov cycles
replayed from a CUDA graph inside an FP64 refinement loop, relative residual
1e-10).  The plain FP64 single-energy solve, the comparison baseline, is
timed separately on the same P0.  Inputs are resident in HBM before the timed
region; L2 is flushed before every timed step, outside its events: a 512 MB
write, then a 256 MB read of another buffer, so that L2 holds clean lines and
the timed work pays no write-back of the flush's dirty lines.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "P assembly Gnodes/s; energies solved/s vs plain FP64 GPU at rel 1e-6"
WORKLOAD_DESC = ("3 identical bosons, V=-3exp(-r^2), l=lambda<=2 -> L=0 (3 channels), N=M=200 "
                 "tangent bins to 20, GL 8x8 p,q + 32 y nodes per cell (81.9M nodes), dim 120000")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="bosons3_200")
    ap.add_argument("--n-energies", type=int, default=128)
    ap.add_argument("--plain-energy", type=float, default=0.5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true")
    ap.add_argument("--no-warm-start", action="store_true")
    ap.add_argument("--warm-train", type=int, default=2000)
    ap.add_argument("--warm-test", type=int, default=512)
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-precision-stress", action="store_true")
    ap.add_argument("--kernel", choices=["spmv32", "spmv64", "spmm32", "spmm64", "asm64", "asm32c", "asmvl"],
                    default=None,
                    help="time one kernel of the path alone on the workload's lattice (for profiling)")
    ap.add_argument("--kernel-reps", type=int, default=5)
    return ap.parse_args()


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# GB300: 152 SMs; FP64 issue rate 2 DFMA per SM per clock (about 1.25 TFLOP/s
# at 2.07 GHz), FP32 128 FMA per SM per clock.
N_SM = 152
FP64_FMA_PER_SM_CLK = 2
FP32_FMA_PER_SM_CLK = 128


def fill_flops_per_node(n_ch: int, n_pairs: int) -> int:
    """FP64 operations of one node in the fill pass (algorithmic count):
    recoupled momenta 2 FMA, y' 1 FMA + 2 MUL + rsqrt (counted as 4),
    Legendre recurrence 3 per order above 1, and per (l, l') pair two
    products and one accumulation."""
    return 4 + (2 + 2 + 4) + 3 * max(n_ch - 2, 0) + 3 * n_pairs


# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture
# of the kernel as it stands (profiles/ names the capture); None where no
# capture of the current kernel exists
NCU_TRAFFIC = {
    "fill_kernel<FP64,3>": 435.8e6,
    "spmm_tile_kernel<FP32>": 333.6e6,
    "tc_gemm_kernel<TF32x3> (Vt, G1)": 329.0e6,
    "tc_gemm_kernel<TF32x3> (O)": 331.7e6,
    "spmm_df_kernel": 954.4e6,  # the tuner's 4-energies-per-lane shape
    "oz_gemm_kernel (digit planes)": 323.7e6,
    "gemm_df_kernel": 903.6e6,
}


class L2Flush:
    """Clears L2 (129 MB on GB300) between timed runs: fill_() writes a
    512 MB buffer and then reads a 256 MB one, leaving L2 full of clean lines
    (a write alone would leave ~129 MB of dirty lines for the timed kernel's
    misses to write back)."""

    def __init__(self):
        import torch

        self.w = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
        self.r = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
        self.sink = None

    def fill_(self, v):
        self.w.fill_(v)
        self.sink = self.r.sum()


def bench_precision_stress(args, W, inputs, stream, flush, device):
    """Precision stress: 5 channels, 300 x 300 lattice (dimension 450 000),
    V = -6 exp(-r^2/0.5) + 2 exp(-r^2/0.1).  Assembly in FP64 and FP32C, and
    the amplitude at E = 0.5 from the plain FP64 solve and from the mixed
    solve on FP64 and on FP32C values, each against the FP64 oracle."""
    import torch

    w = inputs.workload("stress5_300")
    pr = W.Problem(w["p_edges"], w["q_edges"], *w["nodes"], w["n_ch"], w["V"], w["a"], device=device)
    n_nodes = w["N"] * w["M"] * w["nodes"][0] * w["nodes"][1] * w["nodes"][2]
    out = {"workload": "3 bosons, V=-6exp(-r^2/0.5)+2exp(-r^2/0.1), 5 channels, N=M=300, GL 8x8x32 "
                       "nodes per cell (184M nodes), dim 450000"}
    Ps = {}
    for name, prec in (("fp64", W.WPCD_FP64), ("fp32c", W.WPCD_FP32C)):
        ts = []
        for it in range(3):
            flush.fill_(1)
            torch.cuda.synchronize()
            P = pr.wpcd_assemble_P(prec, stream=stream)
            if it > 0:
                ts.append(P.ms)
            if it < 2:
                P.close()
        Ps[name] = P
        ms = statistics.mean(ts)
        out[f"assembly_{name}"] = {"value": n_nodes / (ms * 1e-3) / 1e9, "unit": "Gnodes/s", "ms": ms,
                                    "nnz_cells": P.nnz}
    E = 0.5
    U64, _, _ = pr.wpcd_solve(Ps["fp64"], [E], tol=1e-10, max_iter=300, batch=1, stream=stream)
    Um64, _, _ = pr.wpcd_solve(Ps["fp64"], [E], tol=1e-10, precision=W.WPCD_SOLVE_MIXED, batch=1, stream=stream)
    Um32, _, _ = pr.wpcd_solve(Ps["fp32c"], [E], tol=1e-10, precision=W.WPCD_SOLVE_MIXED, batch=1,
                               stream=stream)
    U = {"fp64": U64[0], "mixed_fp64_values": Um64[0], "mixed_fp32c_values": Um32[0]}
    out["energy"] = E
    out["U00"] = {k: [v.real, v.imag] for k, v in U.items()}
    if not args.no_oracle_check:
        import oracle

        oracle.build()
        t0 = time.perf_counter()
        opr = oracle.Problem(dict(pe=w["p_edges"], qe=w["q_edges"], n_p=w["nodes"][0], n_q=w["nodes"][1],
                                  n_x=w["nodes"][2], n_ch=w["n_ch"], V=list(w["V"]), a=list(w["a"]),
                                  n_pair_nodes=8))
        ref = opr.solve_gmres(E, tol=1e-12, max_iter=400)["U00"]
        out["rel_err_vs_oracle"] = {k: abs(v - ref) / abs(ref) for k, v in U.items()}
        out["oracle_s"] = time.perf_counter() - t0
    for P in Ps.values():
        P.close()
    pr.close()
    return out


def check_all_bins(opr, energies, U, j0_gpu, tol=1e-6):
    """Every energy's U00 against the FP64 oracle.  G1 and the Born term
    depend on an energy only through its on-shell q-bin j0 (the average over
    that energy bin, Sec. 2.3), so the oracle's U00 is the same for all
    energies of one bin: one oracle solve per distinct bin (at the bin's
    first energy) serves every energy of it.  The bins are the oracle's own
    (its on-shell search), and each energy's GPU bin must agree."""
    import oracle

    t0 = time.perf_counter()
    bins = {}
    jo = [oracle.onshell(opr.qe, float(E), opr.eps_b)[0] for E in energies]
    for k, j in enumerate(jo):
        bins.setdefault(j, k)
    ref = {j: opr.solve_gmres(float(energies[k]), tol=1e-12, max_iter=300)["U00"] for j, k in bins.items()}
    errs = [abs(U[k] - ref[j]) / abs(ref[j]) for k, j in enumerate(jo)]
    ok = [e <= tol and int(j0_gpu[k]) == jo[k] for k, e in enumerate(errs)]
    return {"n_energies": len(energies), "n_bins": len(bins), "n_oracle_solves": len(bins),
            "n_checked": len(errs), "within_1e-6": int(sum(ok)), "max_rel_err_U00": max(errs),
            "bins_agree": all(int(j0_gpu[k]) == jo[k] for k in range(len(jo))),
            "oracle_s": time.perf_counter() - t0}


def fp32c_element_stats(val, ref, absref, row_ptr, n_ch, rel=1e-5, ab=1e-6):
    """Per-element error of FP32C P0 values against the oracle's FP64 ones.
    measure = |d| / max(|ref|, 1e-12 rowmax), rowmax the largest |ref| of the
    element's matrix row (l, c); and the bar the tests apply,
    |d| <= rel |ref| + ab S (S = sum_nodes W |P_l(y)|, the magnitude bounding
    every node term): elements that meet the bar only through its absolute
    term are counted."""
    import numpy as np

    pairs = [(l, lp) for l in range(n_ch) for lp in range(n_ch) if (l + lp) % 2 == 0]
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    d = np.abs(val - ref)
    rowmax = np.zeros((len(row_ptr) - 1, n_ch))
    for k, (l, _) in enumerate(pairs):
        np.maximum.at(rowmax[:, l], rows, np.abs(ref[:, k]))
    rm = np.stack([rowmax[rows, l] for l, _ in pairs], axis=1)
    meas = d / np.maximum(np.abs(ref), 1e-12 * rm)
    within_bar = d <= rel * np.abs(ref) + ab * absref
    rel_only = meas <= rel
    return {"n_elements": int(d.size), "max_measure": float(meas.max()),
            "n_measure_above_1e-5": int((~rel_only).sum()),
            "n_within_bar": int(within_bar.sum()),
            "n_abs_term_only": int((within_bar & ~rel_only).sum()),
            "measure": "|d| / max(|ref|, 1e-12 rowmax); bar |d| <= 1e-5 |ref| + 1e-6 sum_nodes W |P_l(y)|"}


def max_over_ranks(x, dist=None, device="cuda"):
    """The largest of the ranks' values of x (every rank gets it); x itself
    on one process.  The step time of a replicated run is the slowest
    rank's."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, seconds, world):
    """Whole-job throughput of a weak-scaling run: every rank processes the
    same number of independent units (energies, lattices) in the slowest
    rank's time; no data moves between ranks."""
    return world * units_per_rank / seconds


def _time_kernel(stream, flush, fn, reps=3):
    """Mean device time (ms) of the kernel fn() times (it returns the
    library's own event timing of that kernel alone), L2 flushed before each
    launch; the first launch (tuning, operand packing) is not counted."""
    import torch

    ts = []
    for _ in range(reps + 1):
        flush.fill_(1)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ts.append(fn())
    return statistics.mean(ts[1:])


# FP32 instructions per float-float multiply-add (TwoProduct by FMA with the
# two cross terms: 4; TwoSum into the accumulator: 6; the error terms: 2)
FF_INSTR_PER_FMA = 12


def kernel_rooflines(W, pr, w, phases, n_nodes, n_e, stream, flush, peaks, f_sm, n32, n64):
    """Achieved vs peak for the kernels that make up the step, each timed on
    its own (the library's CUDA events around that kernel, on the bench
    stream) in the launch configuration the step uses.  n32, n64: the FP32
    and float-float K applications of one step (the Born term takes one
    SpMM and one O product, every residual one SpMM and two products)."""
    import torch

    N, M, n_ch = w["N"], w["M"], w["n_ch"]
    dim = n_ch * N * M
    hbm = peaks.get("hbm_gbs", 6800.0)
    fp64 = 2 * FP64_FMA_PER_SM_CLK * N_SM * f_sm / 1e12
    fp32 = 2 * FP32_FMA_PER_SM_CLK * N_SM * f_sm / 1e12
    ff = 2 * FP32_FMA_PER_SM_CLK * N_SM * f_sm / FF_INSTR_PER_FMA / 1e12
    clk = f"{f_sm / 1e6:.0f} MHz"
    src64 = f"FP64 pipe: {FP64_FMA_PER_SM_CLK} DFMA/SM/clk x {N_SM} SMs x {clk}"
    src32 = f"FP32 pipe: {FP32_FMA_PER_SM_CLK} FMA/SM/clk x {N_SM} SMs x {clk}"
    srcff = (f"float-float on the FP32 pipe: {FP32_FMA_PER_SM_CLK} instr/SM/clk x {N_SM} SMs x {clk} / "
             f"{FF_INSTR_PER_FMA} instr per multiply-add (FP64-equivalent flops)")
    out = []

    def entry(kernel, bound, achieved, peak, unit, ms, per_step, what, peak_source):
        out.append({"kernel": kernel, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                    "frac": achieved / peak, "traffic": NCU_TRAFFIC.get(kernel), "ms_per_launch": ms,
                    "launches_per_step": per_step, "ms_per_step": ms * per_step, "work": what,
                    "peak_source": peak_source})

    fpn = fill_flops_per_node(n_ch, pr.n_pairs)
    entry("fill_kernel<FP64,3>", "alu", n_nodes * fpn / (phases[2] * 1e-3) / 1e12, fp64, "TFLOP/s", phases[2], 1,
          f"{fpn} FP64 flops per node x {n_nodes} nodes", src64)
    # variable-limit assembly (WPCD_FP64_VL) of the same lattice: its value
    # kernel evaluates n_x GL points on every (node, target) y-interval
    grid = W.Grid(w["p_edges"], w["q_edges"], *w["nodes"], device=torch.cuda.current_device())
    vl_ms = []
    for _ in range(2):
        flush.fill_(1)
        torch.cuda.synchronize()
        Pvl = grid.wpcd_assemble_P(n_ch, W.WPCD_FP64_VL, stream=stream)
        vl_ms.append(Pvl.wpcd_P_timing())
        vl_points, vl_nnz = Pvl.wpcd_P_work(), Pvl.nnz
        Pvl.close()
    grid.close()
    ph = vl_ms[-1]
    entry("vl_value_kernel<FP64> (variable limits)", "alu", vl_points * fpn / (ph[2] * 1e-3) / 1e12, fp64, "TFLOP/s",
          ph[2], 0, f"{fpn} FP64 flops per y point x {vl_points} points (n_x per (node, target) interval; "
          f"{vl_nnz} nonzeros; rows pass {ph[0]:.2f} ms, columns and values {ph[2]:.2f} ms)", src64)
    P = pr.wpcd_assemble_P(W.WPCD_FP64, stream=stream)
    x64 = torch.randn(2 * dim * n_e, dtype=torch.float64, device="cuda")
    g64 = torch.randn_like(x64)
    y64 = torch.empty_like(x64)
    x32 = torch.randn(2 * dim * n_e, dtype=torch.float32, device="cuda")
    g32 = torch.randn_like(x32)
    y32 = torch.empty_like(x32)
    gemm_flops = 2.0 * N * N * (2 * M * n_e) * n_ch
    spmm_flops = 4.0 * pr.n_pairs * P.nnz * n_e
    # FP32 inner cycles: P0 SpMM and the two tensor-core channel products
    ms = _time_kernel(stream, flush, lambda: pr.wpcd_spmm(P, x32, y32, n_e, mode=W.WPCD_SPMM_FP32, stream=stream,
                                                           timed=True))
    entry("spmm_tile_kernel<FP32>", "alu", spmm_flops / (ms * 1e-3) / 1e12, fp32, "TFLOP/s", ms, n32,
          f"4 n_pairs nnz B = {spmm_flops:.3e} FP32 flops (one real-by-complex multiply-add per block entry and "
          "energy)", src32)
    tc_bytes = 3.0 * 8 * dim * n_e
    ms = _time_kernel(stream, flush, lambda: pr.wpcd_channel_gemm(0, W.WPCD_GEMM_TF32X3, g32, x32, y32, n_e,
                                                                   stream=stream, timed=True))
    entry("tc_gemm_kernel<TF32x3> (Vt, G1)", "hbm", tc_bytes / (ms * 1e-3) / 1e9, hbm, "GB/s", ms, n32,
          f"X + G1 read, Y written (FP32 complex): {tc_bytes:.3e} B; {3 * gemm_flops:.3e} TF32 MMA flops",
          "measured HBM copy (hbm_gbs)")
    o_bytes = 2.0 * 8 * dim * n_e
    ms = _time_kernel(stream, flush, lambda: pr.wpcd_channel_gemm(1, W.WPCD_GEMM_TF32X3, None, x32, y32, n_e,
                                                                   stream=stream, timed=True))
    entry("tc_gemm_kernel<TF32x3> (O)", "hbm", o_bytes / (ms * 1e-3) / 1e9, hbm, "GB/s", ms, n32,
          f"Z read, Y written (FP32 complex): {o_bytes:.3e} B (the solve's O step also reads S)",
          "measured HBM copy (hbm_gbs)")
    # refinement residual and Born term: float-float SpMM and channel products
    ms = _time_kernel(stream, flush, lambda: pr.wpcd_spmm(P, x64, y64, n_e, mode=W.WPCD_SPMM_FF, stream=stream,
                                                           timed=True))
    # per step at the full batch: the refinement residuals (n64 - 1 of them);
    # the Born term runs once per distinct on-shell bin, in smaller launches
    entry("spmm_df_kernel", "alu", spmm_flops / (ms * 1e-3) / 1e12, ff, "TFLOP/s", ms, n64 - 1,
          f"4 n_pairs nnz B = {spmm_flops:.3e} FP64-equivalent flops in float-float", srcff)
    # channel products of the residual: bf16 digit planes on the tensor cores
    # when N <= 256 (the solve's path), else float-float SIMT
    digits = N <= 256
    if digits:
        ms = _time_kernel(stream, flush, lambda: pr.wpcd_channel_gemm(1, W.WPCD_GEMM_DIGITS, None, x64, y64, n_e,
                                                                       stream=stream, timed=True))
        dflops = 36 * gemm_flops
        entry("oz_gemm_kernel (digit planes)", "tensor", dflops / (ms * 1e-3) / 1e12,
              peaks.get("bf16_tflops", 1900.0), "TFLOP/s", ms, 2 * (n64 - 1),
              f"36 bf16 digit-plane products x 2 N^2 (2 M B) n_ch = {dflops:.3e} bf16 MMA flops "
              f"(FP64-class result: {gemm_flops / (ms * 1e-3) / 1e12:.2f} FP64-equivalent TFLOP/s)",
              "measured cuBLAS bf16 burst (bf16_tflops)")
    ms = _time_kernel(stream, flush, lambda: pr.wpcd_channel_gemm(1, W.WPCD_GEMM_FF, None, x64, y64, n_e,
                                                                   stream=stream, timed=True))
    entry("gemm_df_kernel", "alu", gemm_flops / (ms * 1e-3) / 1e12, ff, "TFLOP/s", ms,
          0 if digits else 2 * (n64 - 1),
          f"2 N^2 (2 M B) n_ch = {gemm_flops:.3e} FP64-equivalent flops in float-float", srcff)
    # the plain FP64 iteration's kernels (the comparison baseline), one energy
    x1 = torch.randn(2 * dim, dtype=torch.float64, device="cuda")
    y1 = torch.empty_like(x1)
    ms = _time_kernel(stream, flush, lambda: pr.wpcd_spmm(P, x1, y1, 1, mode=W.WPCD_SPMM_FP64, stream=stream,
                                                           timed=True))
    spmv_bytes = P.nnz * (4 + 8 * pr.n_pairs) + 8 * (N * M + 1) + 2 * 16 * dim
    spmv_flops = 4.0 * pr.n_pairs * P.nnz
    entry("spmv_kernel<FP64> (1 RHS)", "alu", spmv_flops / (ms * 1e-3) / 1e12, fp64, "TFLOP/s", ms, 0,
          f"{spmv_flops:.3e} FP64 flops, {spmv_bytes:.3e} B (HBM fraction "
          f"{spmv_bytes / (ms * 1e-3) / 1e9 / hbm:.3f}): at 0.45 flop/B it sits above GB300's FP64 ridge "
          f"({fp64 * 1e3 / hbm:.2f} flop/B), so the FP64 pipe, not HBM, bounds it", src64)
    # the FP32-valued one-right-hand-side SpMV (the mixed single-energy inner
    # loop): HBM-bound, 4 B column + 4 n_pairs B values per nonzero
    x1f = torch.randn(2 * dim, dtype=torch.float32, device="cuda")
    y1f = torch.empty_like(x1f)
    ms = _time_kernel(stream, flush, lambda: pr.wpcd_spmm(P, x1f, y1f, 1, mode=W.WPCD_SPMM_FP32, stream=stream,
                                                           timed=True), reps=5)
    spmv32_bytes = P.nnz * (4 + 4 * pr.n_pairs) + 8 * (N * M + 1) + 2 * 8 * dim
    entry("spmv_kernel<FP32> (1 RHS)", "hbm", spmv32_bytes / (ms * 1e-3) / 1e9, hbm, "GB/s", ms, 0,
          f"{spmv32_bytes:.3e} B: columns and FP32 values read once, row pointers, y read and z written "
          "once (FP32 complex)", "measured HBM copy (hbm_gbs)")
    ms = _time_kernel(stream, flush, lambda: pr.wpcd_channel_gemm(1, W.WPCD_GEMM_FP64, None, x1, y1, 1,
                                                                   stream=stream, timed=True))
    g1 = 2.0 * N * N * (2 * M) * n_ch
    entry("gemm_kernel<double> (1 RHS)", "alu", g1 / (ms * 1e-3) / 1e12, fp64, "TFLOP/s", ms, 0,
          f"2 N^2 (2 M) n_ch = {g1:.3e} FP64 flops", src64)
    P.close()
    return out


def run_reference(args):
    """The oracle (FP64 C, OpenMP) on the host cores: the same workload and
    metric; each step assembles P0 for the full lattice."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401

    import oracle
    from paper_1508_07441_gb300 import inputs

    oracle.build()
    w = inputs.workload(args.workload)
    nodes = w["N"] * w["M"] * int(np.prod(w["nodes"]))
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        P = oracle.P0(w["p_edges"], w["q_edges"], *w["nodes"], w["n_ch"])
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
        del P
    ms = 1e3 * statistics.mean(times)
    value = nodes / (ms * 1e-3) / 1e9
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gnodes/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "step": "oracle P0 assembly (count + fill), full lattice"},
        "cpu_baseline": {"value": value, "unit": "Gnodes/s", "cores": cores, "kind": "oracle",
                         "sample": "full 200x200 lattice, all 81.9M nodes, per step"},
        "e2e": {"value": value, "unit": "Gnodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _timed(stream, fn):
    """Device milliseconds of fn() on stream (CUDA events), and its result."""
    import torch

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    out = fn()
    ev1.record(stream)
    ev1.synchronize()
    return ev0.elapsed_time(ev1), out


def bench_batching(args, W, inputs, stream, flush, device, maxr_fn=None):
    """Batching workload (150 x 150 lattice, 3 channels, 8x8x32 nodes):
    128 energies in one batched mixed solve, and 16 uneven-grid problems
    (N = M from [40, 160], seed 1234; 8 seeded energies each) in one grouped
    mixed solve against one solve per problem; a sample checked against the
    oracle."""
    import numpy as np
    import torch

    w = inputs.workload("bosons3_150")
    pr = W.Problem(w["p_edges"], w["q_edges"], *w["nodes"], w["n_ch"], w["V"], w["a"], device=device)
    P = pr.wpcd_assemble_P(W.WPCD_FP64, stream=stream)
    Eb = [float(x) for x in inputs.batch_energies(pr.eps_bound, 128)]
    kw = dict(precision=W.WPCD_SOLVE_MIXED, tol=1e-10, stream=stream)
    t128 = []
    for it in range(4):
        flush.fill_(1)
        torch.cuda.synchronize()
        ms, (U128, s128, _) = _timed(stream, lambda: pr.wpcd_solve(P, Eb, batch=len(Eb), **kw))
        if it > 0:
            t128.append(ms)
    tp = []
    for it in range(3):
        flush.fill_(1)
        torch.cuda.synchronize()
        ms, (Up, sp, _) = _timed(stream, lambda: pr.wpcd_solve(P, [Eb[64]], tol=1e-10, max_iter=200,
                                                                  batch=1, stream=stream))
        if it > 0:
            tp.append(ms)
    # uneven group
    sizes = [int(n) for n in inputs.uneven_sizes(16, 40, 160, 1234)]
    probs, Ps, Es = [], [], []
    for g, n in enumerate(sizes):
        e = inputs.tangent_edges(n, w["k_max"])
        q = W.Problem(e, e, *w["nodes"], w["n_ch"], w["V"], w["a"], device=device)
        probs.append(q)
        Ps.append(q.wpcd_assemble_P(W.WPCD_FP64, stream=stream))
        Es.append(inputs.random_energies(q.eps_bound, 8, 5000 + g))
    n_sys = sum(len(e) for e in Es)
    tg, ts = [], []
    for it in range(4):
        flush.fill_(1)
        torch.cuda.synchronize()
        ms, (Ug, sg, stg) = _timed(stream, lambda: W.wpcd_solve_batch(probs, Ps, Es, **kw))
        if it > 0:
            tg.append(ms)
        flush.fill_(1)
        torch.cuda.synchronize()

        def seq():
            return [q.wpcd_solve(Pq, E, batch=len(E), **kw) for q, Pq, E in zip(probs, Ps, Es)]

        ms, outs = _timed(stream, seq)
        if it > 0:
            ts.append(ms)
    Useq = [o[0] for o in outs]
    diff = max(float(np.max(np.abs(a - b) / np.abs(b))) for a, b in zip(Ug, Useq))
    acc = None
    if not args.no_oracle_check:
        import oracle

        oracle.build()
        errs = []
        t0 = time.perf_counter()
        for g, (n, E) in enumerate(zip(sizes, Es)):
            e = inputs.tangent_edges(n, w["k_max"])
            opr = oracle.Problem(dict(pe=e, qe=e, n_p=w["nodes"][0], n_q=w["nodes"][1], n_x=w["nodes"][2],
                                      n_ch=w["n_ch"], V=list(w["V"]), a=list(w["a"]), n_pair_nodes=8))
            k = g % len(E)
            ref = opr.solve_gmres(float(E[k]), tol=1e-12, max_iter=300)["U00"]
            errs.append(abs(Ug[g][k] - ref) / abs(ref))
        opr = oracle.Problem(dict(pe=w["p_edges"], qe=w["q_edges"], n_p=w["nodes"][0], n_q=w["nodes"][1],
                                  n_x=w["nodes"][2], n_ch=w["n_ch"], V=list(w["V"]), a=list(w["a"]),
                                  n_pair_nodes=8))
        chk = check_all_bins(opr, Eb, U128, [st_.j0 for st_ in s128])
        acc = {"group_max_rel_err_U00": max(errs), "group_within_1e-6": int(sum(x < 1e-6 for x in errs)),
               "group_n_checked": len(errs), "batch128": chk, "oracle_s": time.perf_counter() - t0}
    b128 = statistics.mean(t128)
    bp = statistics.mean(tp)
    g_ms, s_ms = statistics.mean(tg), statistics.mean(ts)
    # only energies within 1e-6 of the oracle count (all of them unchecked
    # when the oracle check is switched off)
    n_ok = acc["batch128"]["within_1e-6"] if acc else 128
    res = {
        "workload": "3 bosons, V=-3exp(-r^2), 3 channels, GL 8x8x32 nodes per cell",
        "batch128": {"value": n_ok / (b128 * 1e-3), "unit": "energies/s", "ms": b128, "N": w["N"],
                     "energies_counted": n_ok,
                     "fp32_k_applications": s128[0].n_kapply32, "fp64_k_applications": s128[0].n_kapply,
                     "max_rel_residual": max(s.relres for s in s128),
                     "plain_fp64": {"value": 1e3 / bp, "unit": "energies/s", "ms": bp, "energy": Eb[64],
                                    "k_applications": sp[0].n_kapply},
                     "speedup_vs_plain_fp64": (n_ok / (b128 * 1e-3)) / (1e3 / bp)},
        "uneven_group": {"value": n_sys / (g_ms * 1e-3), "unit": "energies/s", "ms": g_ms,
                         "sizes": sizes, "energies_per_problem": 8, "status": stg,
                         "max_rel_residual": max(s.relres for sl in sg for s in sl),
                         "fp32_k_applications": sg[0][0].n_kapply32,
                         "one_solve_per_problem": {"value": n_sys / (s_ms * 1e-3), "unit": "energies/s",
                                                   "ms": s_ms},
                         "speedup_vs_per_problem": s_ms / g_ms,
                         "max_rel_diff_vs_per_problem": diff},
        "accuracy_vs_oracle": acc,
    }
    for Pq in Ps:
        Pq.close()
    for q in probs:
        q.close()
    P.close()
    pr.close()
    return res


def run_kernel(args):
    """One kernel of the path on the workload's lattice (FP64 assembly, then
    the kernel's tuning, then --kernel-reps timed launches, each after an L2
    flush): spmv32 / spmv64 the one-right-hand-side SpMV with FP32 / FP64
    values and vectors, spmm32 / spmm64 the SpMM over --n-energies energies;
    asm64 / asm32c / asmvl --kernel-reps assemblies of P0 (node-binned FP64
    and FP32C, variable-limit FP64), each after an L2 flush, with the device
    time of each phase."""
    import numpy as np
    import torch

    from paper_1508_07441_gb300 import inputs
    from paper_1508_07441_gb300 import wpcd as W

    torch.cuda.set_device(0)
    w = inputs.workload(args.workload)
    pr = W.Problem(w["p_edges"], w["q_edges"], *w["nodes"], w["n_ch"], w["V"], w["a"], n_pair_nodes=8)
    if args.kernel.startswith("asm"):
        prec = {"asm64": W.WPCD_FP64, "asm32c": W.WPCD_FP32C, "asmvl": W.WPCD_FP64_VL}[args.kernel]
        flush = L2Flush()
        phases = []
        for _ in range(args.kernel_reps):
            flush.fill_(1)
            torch.cuda.synchronize()
            Pk = pr.wpcd_assemble_P(prec)
            phases.append(Pk.wpcd_P_timing())
            Pk.close()
        print(json.dumps({"kernel": args.kernel, "phases_ms": phases, "nnz": pr.wpcd_assemble_P(prec).nnz}))
        return 0
    P = pr.wpcd_assemble_P(W.WPCD_FP64)
    B = 1 if args.kernel.startswith("spmv") else args.n_energies
    fp32 = args.kernel.endswith("32")
    dt = torch.float32 if fp32 else torch.float64
    y = torch.randn(2 * pr.dim * B, dtype=dt, device="cuda")
    z = torch.empty_like(y)
    flush = L2Flush()
    mode = W.WPCD_SPMM_FP32 if fp32 else W.WPCD_SPMM_FP64
    pr.wpcd_spmm(P, y, z, B, mode=mode)  # tuning (and the FP32 value copy)
    shape = pr.wpcd_tune_spmm(P, B, fp32=fp32)  # the cached choice, before the timed launches
    ms = []
    for _ in range(args.kernel_reps):
        flush.fill_(1)
        torch.cuda.synchronize()
        ms.append(pr.wpcd_spmm(P, y, z, B, mode=mode, timed=True))
    s_val = 4 if fp32 else 8
    nbytes = P.nnz * (4 + s_val * pr.n_pairs) + 8 * (pr.N * pr.M + 1) + 2 * 2 * s_val * pr.dim * B
    print(json.dumps({"kernel": args.kernel, "n_rhs": B, "ms": ms, "ms_mean": float(np.mean(ms[1:] or ms)),
                      "bytes": nbytes, "GB_per_s": nbytes / (float(np.mean(ms[1:] or ms)) * 1e-3) / 1e9,
                      "flops": 4.0 * pr.n_pairs * P.nnz * B, "shape": shape}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel:
        return run_kernel(args)

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1508_07441_gb300 import inputs
    from paper_1508_07441_gb300 import wpcd as W

    w = inputs.workload(args.workload)
    n_nodes = w["N"] * w["M"] * int(np.prod(w["nodes"]))
    stream = torch.cuda.Stream()
    pr = W.Problem(w["p_edges"], w["q_edges"], *w["nodes"], w["n_ch"], w["V"], w["a"],
                   n_pair_nodes=8, device=local)
    energies = [float(x) for x in inputs.batch_energies(pr.eps_bound, args.n_energies)]
    flush = L2Flush()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def one_step():
        with torch.cuda.stream(stream):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            P = pr.wpcd_assemble_P(W.WPCD_FP64, stream=stream)
            U, stats, st = pr.wpcd_solve(P, energies, precision=W.WPCD_SOLVE_MIXED, tol=1e-10,
                                         batch=len(energies), stream=stream)
            ev1.record(stream)
            ev1.synchronize()
            rec = dict(step_ms=ev0.elapsed_time(ev1), asm_ms=P.ms, phases=P.wpcd_P_timing(),
                       solve_ms=stats[0].ms * len(energies), U=U.copy(), nnz=P.nnz,
                       j0=[s_.j0 for s_ in stats],
                       n64=stats[0].n_kapply, n32=stats[0].n_kapply32, n_outer=stats[0].n_outer,
                       relres=max(s.relres for s in stats), status=st)
            P.close()
            return rec

    for _ in range(args.warmup):
        one_step()
    recs = []
    barrier()
    l0 = W.wpcd_launch_count()
    t_wall = time.perf_counter()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)  # L2 flush, outside the step's events
            torch.cuda.synchronize()
            recs.append(one_step())
        barrier()
    wall = time.perf_counter() - t_wall
    launches = W.wpcd_launch_count() - l0

    def maxr(x):
        return max_over_ranks(x, dist, "cuda")

    step_ms = maxr(statistics.mean(r["step_ms"] for r in recs))
    asm_ms = maxr(statistics.mean(r["asm_ms"] for r in recs))
    solve_ms = maxr(statistics.mean(r["solve_ms"] for r in recs))
    phases = [statistics.mean(r["phases"][k] for r in recs) for k in range(3)]
    value = job_throughput(n_nodes, asm_ms * 1e-3, world) / 1e9
    energies_per_s = job_throughput(len(energies), solve_ms * 1e-3, world)

    # ---- FP32C assembly (FP64 binning, FP32 node values), same lattice ----
    f32 = []
    for it in range(max(args.steps, 2) + 1):
        flush.fill_(1)
        torch.cuda.synchronize()
        P3 = pr.wpcd_assemble_P(W.WPCD_FP32C, stream=stream)
        if it > 0:
            f32.append((P3.ms, P3.wpcd_P_timing()))
        P3.close()
    f32_ms = maxr(statistics.mean(m for m, _ in f32))
    f32_phases = [statistics.mean(ph[k] for _, ph in f32) for k in range(3)]

    # ---- plain FP64 single-energy solve (the comparison baseline) ---------
    P4 = pr.wpcd_assemble_P(W.WPCD_FP64, stream=stream)
    plain = []
    for it in range(4):
        flush.fill_(1)
        torch.cuda.synchronize()
        Up, sp, _ = pr.wpcd_solve(P4, [args.plain_energy], tol=1e-10, max_iter=200, batch=1,
                                  stream=stream)
        if it > 0:
            plain.append((sp[0].ms, sp[0].n_kapply, Up[0]))
    plain_ms = maxr(statistics.mean(m for m, _, _ in plain))
    # ---- the same batch with an FP64 refinement residual (FP32 inner
    # cycles, FP64 SpMM and block products for the residual and Born term)
    mf = []
    for it in range(3):
        flush.fill_(1)
        torch.cuda.synchronize()
        Uf, sf, stf = pr.wpcd_solve(P4, energies, precision=W.WPCD_SOLVE_MIXED_FP64, tol=1e-10,
                                    batch=len(energies), stream=stream)
        if it > 0:
            mf.append((sf[0].ms * len(energies), stf, sf[0].n_kapply, sf[0].n_kapply32))
    mixed_fp64_ms = maxr(statistics.mean(m for m, _, _, _ in mf))
    U_ref = recs[-1]["U"]
    mixed_fp64 = {"value": len(energies) / (mixed_fp64_ms * 1e-3), "unit": "energies/s", "ms": mixed_fp64_ms,
                  "status": int(mf[-1][1]), "fp64_k_applications": mf[-1][2], "fp32_k_applications": mf[-1][3],
                  "max_rel_diff_U00_vs_float_float_residual":
                      float(np.max(np.abs(Uf - U_ref) / np.abs(U_ref))),
                  "what": "128 energies, FP32 inner cycles, FP64 residual and Born term, rel residual 1e-10"}
    P4.close()

    # ---- batching workload: 128 energies on the 150 x 150 lattice, and 16
    # problems of uneven grids (N = M drawn from [40, 160], seed 1234, 8
    # seeded energies each) in one grouped iteration vs one solve per problem
    batching = None
    if not args.no_batching:
        batching = bench_batching(args, W, inputs, stream, flush, local, maxr_fn=None)

    # ---- precision stress: 5 channels, 300 x 300 (dimension 450 000) ------
    stress = None
    if not args.no_precision_stress and world == 1:
        stress = bench_precision_stress(args, W, inputs, stream, flush, local)

    # ---- end to end through the public API with host buffers -------------
    barrier()
    n_e2e = 4
    e2e_each = []
    for _ in range(n_e2e):
        t0 = time.perf_counter()
        pr2 = W.Problem(w["p_edges"], w["q_edges"], *w["nodes"], w["n_ch"], w["V"], w["a"],
                        n_pair_nodes=8, device=local)
        P2 = pr2.wpcd_assemble_P(W.WPCD_FP64, stream=stream)
        U2, st2, _ = pr2.wpcd_solve(P2, energies, precision=W.WPCD_SOLVE_MIXED, tol=1e-10,
                                    batch=len(energies), stream=stream)
        P2.close()
        pr2.close()
        torch.cuda.synchronize()
        e2e_each.append(time.perf_counter() - t0)
    e2e_s = maxr(statistics.mean(e2e_each))
    N, M, n_ch = w["N"], w["M"], w["n_ch"]
    nn = w["nodes"]
    h2d = 8 * ((N + 1) + (M + 1) + N * nn[0] * 2 + M * nn[1] * 2 + nn[2] * 2 + N * M + (M + 1)
               + n_ch * N + 2 * n_ch * N * N) + 8 * (2 * len(energies) + 64)
    d2h = 8 + 48 * len(energies) + 16 * len(energies) * (st2[0].n_outer + 2)

    # ---- learned warm start: iterations to rel residual 1e-8, warm vs cold --
    warm = None
    if not args.no_warm_start:
        from paper_1508_07441_gb300.warmstart import WarmStart

        t0 = time.perf_counter()
        P5 = pr.wpcd_assemble_P(W.WPCD_FP64, stream=stream)
        ws = WarmStart(pr, P5, k=64, kf=16, width=256, seed=2026, device=local, stream=stream)
        lo, hi = -0.9 * abs(pr.eps_bound), 5.0
        ws.e_lo, ws.e_hi = lo, hi
        ws.build_basis(ws.snapshot_energies(lo, hi))
        Xtr, Ttr = ws.dataset(inputs.random_energies(pr.eps_bound, args.warm_train, seed=2026))
        t_data = time.perf_counter() - t0
        t1 = time.perf_counter()
        hist = ws.fit(Xtr, Ttr, epochs=600, batch=256, lr=2e-3, decay=(0.1, 0.01, 0.001))
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t1
        Ete = inputs.random_energies(pr.eps_bound, args.warm_test, seed=2027)
        cold, rc, _, Uc = ws.iterations(Ete, tol=1e-8, batch=64, max_iter=60)
        t2 = time.perf_counter()
        ug = ws.predict(Ete)
        torch.cuda.synchronize()
        t_pred = time.perf_counter() - t2
        wit, rw, fb, Uw = ws.iterations(Ete, u_init=ug, tol=1e-8, batch=64, max_iter=60)
        # accuracy of the warm start itself: |u_g - u| / |u| per energy, BF16
        # inference (the one used) and FP32 inference of the same network
        ut = ws.solve_vectors(Ete, batch=128).view(len(Ete), -1)
        torch.cuda.synchronize()
        nrm = torch.linalg.vector_norm(ut, dim=1)
        err_bf16 = (torch.linalg.vector_norm(ug.view(len(Ete), -1) - ut, dim=1) / nrm).cpu().numpy()
        ug32 = ws.predict(Ete, bf16=False).view(len(Ete), -1)
        torch.cuda.synchronize()  # predict runs on the bench stream
        err_fp32 = (torch.linalg.vector_norm(ug32 - ut, dim=1) / nrm).cpu().numpy()
        del ut
        wit32, _, fb32, _ = ws.iterations(Ete, u_init=ug32.view(-1), tol=1e-8, batch=64, max_iter=60)
        del ug32
        warm = {"what": "3-layer MLP (width 256, FP32 train by the library's kernels, BF16 inference) "
                        "predicting mixture weights (softmax of 64 logits) over a 64-vector basis of "
                        "the method's own solutions beyond the Born term, at the 64 on-shell bins "
                        "that carry most of the energy range; FP64 Krylov to rel residual 1e-8 from "
                        "the warm start vs from zero; K applications include the Born term and, "
                        "warm, the warm start's residual",
                "train_energies": args.warm_train, "test_energies": args.warm_test,
                "basis": ws.k, "train_loss_first_last": [float(hist[0]), float(hist[-1])],
                "k_applications_cold_mean": float(cold.mean()),
                "k_applications_warm_mean": float(wit.mean()),
                "saved_fraction": float(1.0 - wit.mean() / cold.mean()),
                "max_rel_residual_cold": float(rc.max()), "max_rel_residual_warm": float(rw.max()),
                "fallbacks": int(fb.sum()),
                "warm_rel_error_median_bf16": float(np.median(err_bf16)),
                "warm_rel_error_median_fp32_inference": float(np.median(err_fp32)),
                "k_applications_warm_fp32_inference_mean": float(wit32.mean()),
                "saved_fraction_fp32_inference": float(1.0 - wit32.mean() / cold.mean()),
                "max_rel_diff_U00_warm_vs_cold": float(np.max(np.abs(Uw - Uc) / np.abs(Uc))),
                "s_data": t_data, "s_train": t_train, "s_predict": t_pred}
        P5.close()
        del ws

    # ---- rooflines of the step's kernels, timed live (CUDA events on the
    # bench stream, L2 flushed before every timed launch); the dominant
    # kernel (largest per-step time) becomes `roofline`
    peaks, peak_src = measured_peaks()
    clocks = clk.summary()
    f_sm = (clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)) * 1e6
    rl = kernel_rooflines(W, pr, w, phases, n_nodes, len(energies), stream, flush, peaks, f_sm,
                          recs[-1]["n32"], recs[-1]["n64"])
    dom = max(rl, key=lambda r: r["ms_per_step"])  # the kernel with the largest share of the step
    roofline = {k: dom[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "traffic")}
    roofline["peak_source"] = dom["peak_source"]

    # ---- accuracy against the oracle and the CPU baseline -----------------
    cpu = None
    acc = None
    fp32c_stats = None
    if rank == 0 and world == 1 and not (args.no_cpu_baseline and args.no_oracle_check):
        import oracle

        oracle.build()
        t0 = time.perf_counter()
        Pref = oracle.P0(w["p_edges"], w["q_edges"], *w["nodes"], n_ch)
        t_asm = time.perf_counter() - t0
        cpu = {"value": n_nodes / t_asm / 1e9, "unit": "Gnodes/s", "cores": oracle.num_threads(),
               "kind": "oracle",
               "sample": "P0 assembly (count + fill) of the full 200x200 lattice, 81.9M nodes, once"}
        # one core (the paper's CPU convention), on the lattice of the first
        # 100 x 100 bins of the same edges (a quarter of the nodes)
        n_all = oracle.num_threads()
        oracle.set_threads(1)
        t0 = time.perf_counter()
        oracle.P0(w["p_edges"][:101], w["q_edges"][:101], *w["nodes"], n_ch)
        t1c = time.perf_counter() - t0
        oracle.set_threads(n_all)
        cpu["single_core"] = {"value": 100 * 100 * int(np.prod(w["nodes"])) / t1c / 1e9, "unit": "Gnodes/s",
                              "cores": 1, "s": t1c,
                              "sample": "P0 assembly of the first 100 x 100 bins of the same edges (20.5M nodes)"}
        if not args.no_oracle_check:
            opr = oracle.Problem(dict(pe=w["p_edges"], qe=w["q_edges"], n_p=nn[0], n_q=nn[1],
                                      n_x=nn[2], n_ch=n_ch, V=list(w["V"]), a=list(w["a"]),
                                      n_pair_nodes=8), P=Pref)
            acc = check_all_bins(opr, energies, recs[-1]["U"], recs[-1]["j0"])
            cpu["solve_energies_per_s"] = acc["n_oracle_solves"] / acc["oracle_s"]
            cpu["solve_sample"] = (f"one FP64 Krylov solve (rel residual 1e-12) per distinct on-shell bin of "
                                   f"the {len(energies)} energies ({acc['n_bins']} bins)")
            pref = opr.solve_gmres(args.plain_energy, tol=1e-12, max_iter=300)["U00"]
            acc["plain_fp64_rel_err"] = abs(plain[-1][2] - pref) / abs(pref)
            # FP32C values of the full lattice, element by element
            Pabs = oracle.P0(w["p_edges"], w["q_edges"], *w["nodes"], n_ch, with_abs=True)
            P3 = pr.wpcd_assemble_P(W.WPCD_FP32C, stream=stream)
            rp3, col3, val3 = P3.wpcd_P_export()
            P3.close()
            if np.array_equal(rp3, Pabs["row_ptr"]) and np.array_equal(col3, Pabs["col"]):
                fp32c_stats = fp32c_element_stats(val3.T, Pabs["val"], Pabs["absval"], Pabs["row_ptr"], n_ch)
            else:
                fp32c_stats = {"pattern_mismatch": True}
            del Pabs

    if rank != 0:
        return 0
    # only energies within 1e-6 of the oracle count into the solve rate
    n_ok = acc["within_1e-6"] if acc else len(energies)
    solve_value = energies_per_s * n_ok / len(energies)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "Gnodes/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC,
                   "energies": f"{len(energies)} uniform in [-0.9|E_d|, 5] (E_d = {pr.eps_bound:.6f})",
                   "assembly": "FP64",
                   "solve": "batched (all energies in one iteration), FP32 inner Krylov cycles "
                            "of 10 steps (tensor-core TF32x3 block products, CUDA graph) + float-float "
                            "refinement residual to rel residual 1e-10",
                   "l2": "flushed (512 MB write, then a 256 MB read) before every timed step and every "
                         "timed kernel launch",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "assembly": {"ms": asm_ms, "count_ms": phases[0], "scan_ms": phases[1], "fill_ms": phases[2],
                     "nnz_cells": recs[-1]["nnz"]},
        "assembly_fp32c": {"value": world * n_nodes / (f32_ms * 1e-3) / 1e9, "unit": "Gnodes/s",
                           "ms": f32_ms, "count_ms": f32_phases[0], "scan_ms": f32_phases[1],
                           "fill_ms": f32_phases[2], "vs_oracle": fp32c_stats},
        "solve": {"value": solve_value, "unit": "energies/s", "ms": solve_ms,
                  "n_energies": len(energies), "energies_counted": n_ok,
                  "fp64_k_applications": recs[-1]["n64"],
                  "fp32_k_applications": recs[-1]["n32"], "refinement_cycles": recs[-1]["n_outer"],
                  "max_rel_residual": recs[-1]["relres"],
                  "plain_fp64": {"value": 1e3 / plain_ms, "unit": "energies/s", "ms": plain_ms,
                                 "energy": args.plain_energy, "k_applications": plain[-1][1],
                                 "what": "one energy, FP64 Krylov, rel residual 1e-10"},
                  "speedup_vs_plain_fp64": solve_value / (1e3 / plain_ms),
                  "mixed_fp64_residual": mixed_fp64,
                  "accuracy_vs_oracle": acc},
        "warm_start": warm,
        "batching": batching,
        "precision_stress": stress,
        "roofline": roofline,
        "roofline_peak_source": peak_src,
        "kernel_rooflines": rl,
        "cpu_baseline": cpu,
        "e2e": {"value": world * n_nodes / e2e_s / 1e9, "unit": "Gnodes/s",
                "s_per_step": e2e_s, "s_each": [round(x, 5) for x in e2e_each],
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "what": "Problem create (host setup + uploads) + assemble + solve with host "
                        "energies and host U00, per step"},
        # headline numbers as flat scalars
        "solve_energies_per_s": solve_value,
        "solve_energies_checked": acc["n_checked"] if acc else 0,
        "solve_energies_within_1e-6": n_ok if acc else 0,
        "solve_max_rel_err_U00": acc["max_rel_err_U00"] if acc else None,
        "plain_fp64_energies_per_s": 1e3 / plain_ms,
        "solve_speedup_vs_plain_fp64": solve_value / (1e3 / plain_ms),
        "solve_mixed_fp64_residual_energies_per_s": mixed_fp64["value"],
        "assembly_fp32c_gnodes_per_s": world * n_nodes / (f32_ms * 1e-3) / 1e9,
        "assembly_fp32c_max_measure": fp32c_stats.get("max_measure") if fp32c_stats else None,
        "assembly_fp32c_n_abs_term_only": fp32c_stats.get("n_abs_term_only") if fp32c_stats else None,
        "batch150_energies_per_s": batching["batch128"]["value"] if batching else None,
        "uneven_group_energies_per_s": batching["uneven_group"]["value"] if batching else None,
        "stress_U00_rel_err_mixed_fp32c": (stress or {}).get("rel_err_vs_oracle", {}).get("mixed_fp32c_values"),
        "warm_start_saved_fraction": warm["saved_fraction"] if warm else None,
        "gpu_launches": launches // max(args.steps, 1) * args.steps,
        "gpu_launches_per_step": launches / max(args.steps, 1),
        "clocks": clocks,
        "wall_s_timed": wall,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
