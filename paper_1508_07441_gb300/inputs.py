"""Seeded synthetic workloads (inputs only: no arithmetic of the method).

Both the CUDA path and the oracle take their inputs from here: packet-grid
edges, node counts, channel counts, pair-potential terms and energies.  The
workloads are the three-boson Gaussian systems the benchmarks are quoted on;
the paper's own potentials (Malfliet-Tjon, Nijmegen I) and comparison data are
not used.
"""
from __future__ import annotations

import math

import numpy as np


def tangent_edges(n_bins: int, k_max: float) -> np.ndarray:
    """Edges k_n = s tan(pi n / (2 (n_bins + 1))), k_0 = 0, k_{n_bins} = k_max."""
    n = np.arange(n_bins + 1, dtype=np.float64)
    ang = np.pi * n / (2.0 * (n_bins + 1))
    s = k_max / math.tan(np.pi * n_bins / (2.0 * (n_bins + 1)))
    e = s * np.tan(ang)
    e[0] = 0.0
    e[-1] = k_max
    return e


def jittered_edges(n_bins: int, k_max: float, seed: int, frac: float = 0.1) -> np.ndarray:
    """Tangent edges with each interior edge moved by up to +-frac of its
    smaller neighbouring bin (seeded), for robustness tests."""
    e = tangent_edges(n_bins, k_max)
    rng = np.random.default_rng(seed)
    w = np.diff(e)
    for k in range(1, n_bins):
        e[k] += frac * min(w[k - 1], w[k]) * rng.uniform(-1.0, 1.0)
    return e


# Workloads: (N = M, nodes (n_p, n_q, n_x), channels, potential terms)
WORKLOADS = {
    # s-wave, V = -3 exp(-r^2), 50 x 50 lattice, 4x4x16 nodes; one energy E = 0.5
    "swave_50": dict(N=50, M=50, k_max=20.0, nodes=(4, 4, 16), n_ch=1, V=(-3.0,), a=(1.0,),
                 energies=(0.5,)),
    # l = lambda <= 2 (3 channels), 200 x 200 lattice, 8x8x32 nodes (dimension 120 000)
    "bosons3_200": dict(N=200, M=200, k_max=20.0, nodes=(8, 8, 32), n_ch=3, V=(-3.0,), a=(1.0,),
                 energies=(0.5,)),
    # batching: 150 x 150, 3 channels, 128 energies in [-0.9 |E_d|, 5]
    "bosons3_150": dict(N=150, M=150, k_max=20.0, nodes=(8, 8, 32), n_ch=3, V=(-3.0,), a=(1.0,),
                 energies=None),
    # precision stress: short-range repulsion, 5 channels, 300 x 300 (dimension 450 000)
    "stress5_300": dict(N=300, M=300, k_max=20.0, nodes=(8, 8, 32), n_ch=5, V=(-6.0, 2.0), a=(0.5, 0.1),
                 energies=(0.5,)),
}


def workload(name: str) -> dict:
    w = dict(WORKLOADS[name])
    w["p_edges"] = tangent_edges(w["N"], w["k_max"])
    w["q_edges"] = tangent_edges(w["M"], w["k_max"])
    return w


def batch_energies(eps_dimer: float, n: int = 128, hi: float = 5.0) -> np.ndarray:
    """n energies uniform in [-0.9 |E_d|, hi] (inclusive grid)."""
    return np.linspace(-0.9 * abs(eps_dimer), hi, n)


def random_energies(eps_dimer: float, n: int, seed: int, hi: float = 5.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.9 * abs(eps_dimer), hi, n)


def uneven_sizes(n: int = 16, lo: int = 40, hi: int = 160, seed: int = 1234) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, n)


def random_complex(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)
