"""Learned warm start for the Faddeev iteration (argument marshalling around
the library's kernels).

G1 depends on the energy only through its on-shell bin, so u(E) is constant
across a bin and its source u0 (the Born term, the first iterate) is specific
to the bin.  The network therefore predicts the part of the solution beyond
the first iterate, u - u0, in a basis of the method's own solutions.

Pipeline, every arithmetic step in libwpcd:
  1. snapshots: d_j = u(E_j) - u0(E_j) at the centres of the k on-shell bins
     that carry the most of the energy range (batched mixed solves); D =
     [d_1 .. d_k] is the basis, and an orthonormalised copy Phi serves the
     features;
  2. data: each training energy is solved; its label is the snapshot nearest
     to its u - u0 (least |d - d_j|, from the inner products <d_j, d>); the
     target is a logit vector, L at the label and 0 elsewhere; the features
     are the scaled centre of the on-shell bin and the first kf coefficients
     Phi^H u0 of the first iterate;
  3. the MLP is trained by the library's FP32 forward / backward / Adam
     kernels and inferred with BF16 weights;
  4. warm start u_g = u0 + D w with w = softmax(logits): mixture weights over
     the snapshots.  The weights are insensitive to the BF16 rounding of the
     logits (an error of 1e-3 L in a logit changes a weight by that relative
     amount, while the weight of a wrong snapshot stays near exp(-L)), so an
     energy in a snapshot's bin gets that snapshot's solution almost exactly.
     The solve starts from u_g and falls back to u = 0 for any energy whose
     warm residual is not below |u0|; the plain iteration's FP64 residual
     judges convergence.
"""
from __future__ import annotations

import numpy as np

from . import wpcd as W


class WarmStart:
    def __init__(self, pr, P, k=64, kf=16, width=256, seed=2026, device=0, stream=None, logit=24.0):
        import torch

        self.torch = torch
        self.pr, self.P, self.k, self.kf, self.width = pr, P, k, kf, width
        self.seed, self.device, self.stream = seed, device, stream
        self.logit = logit
        self.dim = pr.dim
        self.D = None    # snapshots u - u0 [k][2 dim], the mixture basis
        self.Phi = None  # its orthonormalised copy (features)
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
        with self.torch.cuda.stream(self._torch_stream()):
            self.D = U.clone()
        W.wpcd_basis_orthonormalize(U, self.k, self.dim, stream=self.stream)
        self.Phi = U
        # |d_j|^2 for the labels: the diagonal of D^H D
        G = self._dev(2 * self.k * self.k, self.torch.float64)
        W.wpcd_basis_project(self.D, self.k, self.dim, self.D, self.k, G, stream=self.stream)
        self._sync()
        g = G.cpu().numpy().view(np.complex128).reshape(self.k, self.k)
        self.dnorm2 = np.real(np.diag(g)).copy()
        return U

    def _torch_stream(self):
        if self.stream is None:
            return self.torch.cuda.current_stream(self.device)
        return self.stream

    def _sync(self):
        self.torch.cuda.synchronize(self.device)

    def coefficients(self, U, n, basis=None):
        """C [n][k] complex FP64 (device): <b_j, U_e> for the basis b (Phi by
        default)."""
        C = self._dev(2 * n * self.k, self.torch.float64)
        W.wpcd_basis_project(self.Phi if basis is None else basis, self.k, self.dim, U, n, C,
                             stream=self.stream)
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

    def labels(self, Ud, n):
        """The snapshot nearest to each of the n vectors Ud (u - u0):
        argmin_j |d_j|^2 - 2 Re <d_j, d>."""
        C = self.coefficients(Ud, n, basis=self.D)
        self._sync()
        c = C.cpu().numpy().view(np.complex128).reshape(n, self.k)
        return np.argmin(self.dnorm2[None, :] - 2.0 * c.real, axis=1)

    def dataset(self, E, batch=128):
        """(X, T): features and logit targets (L at the label, 0 elsewhere),
        device float32; the labels come from the solutions of the energies."""
        E = np.asarray(E, dtype=np.float64)
        Xs, Ts = [], []
        self.train_labels = []
        for i in range(0, len(E), batch):
            Eb = E[i:i + batch]
            U = self.solve_vectors(Eb, batch=batch)
            b = self.born(Eb)
            W.wpcd_vec_axpy(-1.0, b, U, stream=self.stream)  # u - u0
            lab = self.labels(U, len(Eb))
            self.train_labels.append(lab)
            T = np.zeros((len(Eb), self.k), dtype=np.float32)
            T[np.arange(len(Eb)), lab] = self.logit
            Xs.append(self.features(Eb, b))
            Ts.append(self.torch.from_numpy(T).to(f"cuda:{self.device}"))
            del U
        self.train_labels = np.concatenate(self.train_labels)
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
        """Warm starts u_g = u0 + D softmax(logits) (device float64 [len(E)][2 dim])."""
        E = np.asarray(E, dtype=np.float64)
        n = len(E)
        b = self.born(E)
        X = self.features(E, b)
        Y = self._dev(n * self.k, self.torch.float32)
        self.mlp.wpcd_mlp_forward(X.contiguous(), Y, bf16=bf16, stream=self.stream)
        C = self._dev(n * 2 * self.k, self.torch.float32)
        W.wpcd_warm_softmax(Y, n, self.k, C, stream=self.stream)
        U = self._dev(2 * n * self.dim, self.torch.float64)
        W.wpcd_basis_expand(self.D, self.k, self.dim, C, n, U, stream=self.stream)
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
