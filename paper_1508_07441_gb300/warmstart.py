"""Learned warm start for the Faddeev iteration (argument marshalling around
the library's kernels).

G1 depends on the energy only through its on-shell bin, so u(E) is constant
across a bin and its source u0 (the Born term, the first iterate) is specific
to the bin.  The network therefore predicts the part of the solution beyond
the first iterate, u - u0, in a basis built from that part.

Pipeline, every arithmetic step in libwpcd:
  1. snapshots: u(E) - u0(E) at the centres of the k on-shell bins that
     carry the most of the energy range (batched mixed solves),
     orthonormalised on the GPU into a projected basis Phi;
  2. data: for each training energy the target is Phi^H (u - u0) (k complex
     = 2k reals) and the features are the scaled centre of the on-shell bin
     and the first kf coefficients Phi^H u0 of the first iterate;
  3. the MLP is trained by the library's FP32 forward / backward / Adam
     kernels and inferred with BF16 weights;
  4. warm start u_g = u0 + Phi c_hat; the solve starts from u_g and falls
     back to u = 0 for any energy whose warm residual is not below |u0|; the
     plain iteration's FP64 residual judges convergence.
"""
from __future__ import annotations

import numpy as np

from . import wpcd as W


class WarmStart:
    def __init__(self, pr, P, k=64, kf=16, width=256, seed=2026, device=0, stream=None):
        import torch

        self.torch = torch
        self.pr, self.P, self.k, self.kf, self.width = pr, P, k, kf, width
        self.seed, self.device, self.stream = seed, device, stream
        self.dim = pr.dim
        self.Phi = None
        self.mlp = None
        self.e_lo = self.e_hi = None

    def _dev(self, n, dtype):
        return self.torch.zeros(n, dtype=dtype, device=f"cuda:{self.device}")

    def solve_vectors(self, E, batch=128, tol=1e-10):
        """Solutions u(E) (device float64 [len(E)][2 dim]) by batched mixed solves."""
        E = np.asarray(E, dtype=np.float64)
        U = self._dev(2 * len(E) * self.dim, self.torch.float64)
        self.pr.wpcd_solve(self.P, E, precision=W.WPCD_SOLVE_MIXED, batch=batch, tol=tol, u_out=U,
                           stream=self.stream)
        return U

    def born(self, E):
        E = np.asarray(E, dtype=np.float64)
        b = self._dev(2 * len(E) * self.dim, self.torch.float64)
        self.pr.wpcd_born(self.P, E, b, stream=self.stream)
        return b

    def snapshot_energies(self, e_lo, e_hi):
        """k energies at the centres of the on-shell bins that carry the most
        of [e_lo, e_hi] in energy (a bin q in [q_j, q_j+1) spans eps_d + 3/4 q^2
        over its edges): u depends on E only through the bin, so a basis that
        holds the solutions of those bins holds the exact solution for every
        energy that falls in one of them."""
        qe, eb = self.pr.qe, self.pr.eps_bound
        Eq = eb + 0.75 * np.asarray(qe) ** 2
        meas = np.clip(np.minimum(Eq[1:], e_hi) - np.maximum(Eq[:-1], e_lo), 0.0, None)
        js = np.sort(np.argsort(-meas, kind="stable")[:self.k])
        js = js[meas[js] > 0]
        E = eb + 0.75 * (0.5 * (qe[js] + qe[js + 1])) ** 2
        return np.clip(E, e_lo, e_hi)  # fewer than k when the range has fewer bins

    def build_basis(self, E_snap, batch=128):
        E_snap = np.asarray(E_snap, dtype=np.float64)
        self.k = len(E_snap)
        U = self.solve_vectors(E_snap, batch=batch)
        W.wpcd_vec_axpy(-1.0, self.born(E_snap), U, stream=self.stream)  # u - u0
        W.wpcd_basis_orthonormalize(U, self.k, self.dim, stream=self.stream)
        self.Phi = U
        return U

    def coefficients(self, U, n):
        C = self._dev(2 * n * self.k, self.torch.float64)
        W.wpcd_basis_project(self.Phi, self.k, self.dim, U, n, C, stream=self.stream)
        return C

    def features(self, E, b=None):
        """X [n][1 + 2 kf] (device float32) from the on-shell bin and the
        Born term."""
        E = np.asarray(E, dtype=np.float64)
        n = len(E)
        if b is None:
            b = self.born(E)
        Cb = self.coefficients(b, n)
        X = self._dev(n * (1 + 2 * self.kf), self.torch.float32)
        W.wpcd_warm_features(self.pr, E, self.e_lo, self.e_hi, Cb, self.k, self.kf, X, stream=self.stream)
        return X.view(n, 1 + 2 * self.kf)

    def dataset(self, E, batch=128):
        """(X, T): features and target coefficients, device float32."""
        E = np.asarray(E, dtype=np.float64)
        Xs, Ts = [], []
        for i in range(0, len(E), batch):
            Eb = E[i:i + batch]
            U = self.solve_vectors(Eb, batch=batch)
            b = self.born(Eb)
            W.wpcd_vec_axpy(-1.0, b, U, stream=self.stream)  # u - u0
            C = self.coefficients(U, len(Eb))
            T = self._dev(2 * len(Eb) * self.k, self.torch.float32)
            W.wpcd_complex_to_f32(C, len(Eb) * self.k, T, stream=self.stream)
            Xs.append(self.features(Eb, b))
            Ts.append(T.view(len(Eb), 2 * self.k))
            del U
        return self.torch.cat(Xs), self.torch.cat(Ts)

    def fit(self, X, T, epochs=300, batch=256, lr=1e-3, decay=()):
        """Train for epochs at lr, then epochs more at each lr * f for f in
        decay (a step schedule); the loss history of all phases."""
        n_in, n_out = X.shape[1], T.shape[1]
        self.mlp = W.MLP(n_in, self.width, n_out, seed=self.seed, device=self.device)
        # affine maps from the training statistics (setup of the network, host)
        Xh, Th = X.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)
        xs = Xh.std(axis=0)
        xs[xs == 0] = 1.0
        ts = Th.std(axis=0)
        ts[ts == 0] = 1.0
        self.mlp.wpcd_mlp_set_affine(1.0 / xs, -Xh.mean(axis=0) / xs, ts, Th.mean(axis=0))
        hist = [self.mlp.wpcd_mlp_train(X.contiguous(), T.contiguous(), epochs, batch, lr, seed=self.seed,
                                        stream=self.stream)]
        for i, f in enumerate(decay):
            hist.append(self.mlp.wpcd_mlp_train(X.contiguous(), T.contiguous(), epochs, batch, lr * f,
                                                seed=self.seed + 1 + i, stream=self.stream))
        return np.concatenate(hist)

    def predict(self, E, bf16=True):
        """Warm starts u_g = u0 + Phi c_hat (device float64 [len(E)][2 dim])."""
        E = np.asarray(E, dtype=np.float64)
        n = len(E)
        b = self.born(E)
        X = self.features(E, b)
        Y = self._dev(n * 2 * self.k, self.torch.float32)
        self.mlp.wpcd_mlp_forward(X.contiguous(), Y, bf16=bf16, stream=self.stream)
        U = self._dev(2 * n * self.dim, self.torch.float64)
        W.wpcd_basis_expand(self.Phi, self.k, self.dim, Y, n, U, stream=self.stream)
        W.wpcd_vec_axpy(1.0, b, U, stream=self.stream)
        return U

    def iterations(self, E, u_init=None, tol=1e-8, batch=64, max_iter=200):
        """Per-energy FP64 K applications to the relative residual tol, the
        achieved residuals and the fallback flags."""
        E = np.asarray(E, dtype=np.float64)
        its, res, fb, amps = [], [], [], []
        for i in range(0, len(E), batch):
            Eb = E[i:i + batch]
            ui = None
            if u_init is not None:
                ui = u_init[2 * i * self.dim:2 * (i + len(Eb)) * self.dim]
            U, stats, st = self.pr.wpcd_solve(self.P, Eb, tol=tol, max_iter=max_iter, batch=batch,
                                              check_every=1, u_init=ui, stream=self.stream)
            its += [s.n_kapply for s in stats]
            res += [s.relres for s in stats]
            fb += [s.warm_fallback for s in stats]
            amps += list(U)
        return np.array(its), np.array(res), np.array(fb), np.array(amps)
