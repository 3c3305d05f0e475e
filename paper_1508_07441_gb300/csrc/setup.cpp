// Host mathematics of step 1 of the numerical scheme (Sec. 3.3): packet
// grids, Gauss-Legendre tables, the pair potential in the free-packet basis
// (Sec. 2.2 Eq. vpot) and the diagonalisation of h1 (Eq. exp_z).  FP64,
// negligible time; everything here feeds the device kernels.
#include <algorithm>
#include <cmath>
#include <vector>

#include "wpcd_internal.h"

namespace wpcd {

// Gauss-Legendre nodes (ascending) and weights on [-1, 1]: Newton's method on
// P_n with the derivative from P_n' = n (x P_n - P_{n-1}) / (x^2 - 1), started
// from Tricomi's asymptotic node estimate, iterated in long double and
// rounded once.
void gauss_legendre(int n, double *t, double *w) {
  const long double pi = 3.14159265358979323846264338327950288L;
  for (int k = 1; k <= n; ++k) {
    long double th = pi * (4.0L * k - 1.0L) / (4.0L * n + 2.0L);
    long double x = (1.0L - (n - 1.0L) / (8.0L * n * n * n)) * cosl(th);
    long double d = 0.0L;
    for (int it = 0; it < 64; ++it) {
      long double pm1 = 1.0L, p = x;  // P_0, P_1
      for (int m = 2; m <= n; ++m) {
        long double pn = ((2.0L * m - 1.0L) * x * p - (m - 1.0L) * pm1) / m;
        pm1 = p;
        p = pn;
      }
      if (n == 1) { p = x; pm1 = 1.0L; }
      d = n * (x * p - pm1) / (x * x - 1.0L);
      long double step = p / d;
      x -= step;
      if (fabsl(step) < 1e-28L) break;
    }
    long double pm1 = 1.0L, p = x;
    for (int m = 2; m <= n; ++m) {
      long double pn = ((2.0L * m - 1.0L) * x * p - (m - 1.0L) * pm1) / m;
      pm1 = p;
      p = pn;
    }
    if (n == 1) { p = x; pm1 = 1.0L; }
    d = n * (x * p - pm1) / (x * x - 1.0L);
    // k = 1 is the largest node
    t[n - k] = (double)x;
    w[n - k] = (double)(2.0L / ((1.0L - x * x) * d * d));
  }
}

// Symmetric eigenproblem: Householder reduction to tridiagonal form, then
// implicit symmetric QR steps with Wilkinson shifts on the tridiagonal,
// accumulating the orthogonal transformations.
bool sym_eig(int n, std::vector<double> A, std::vector<double> &evals, std::vector<double> &rows) {
  auto a = [&](int i, int j) -> double & { return A[(size_t)i * n + j]; };
  // Householder: zero column k below the subdiagonal, A <- H_k A H_k with
  // H_k = 1 - beta_k u_k u_k^T; the u_k are kept for Q = H_0 H_1 .. H_{n-3}
  std::vector<double> Us((size_t)n * n, 0.0), betas(n, 0.0), pvec(n), kvec(n);
  for (int k = 0; k + 2 < n; ++k) {
    double *u = &Us[(size_t)k * n];
    double alpha = 0.0;
    for (int i = k + 1; i < n; ++i) alpha += a(i, k) * a(i, k);
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    if (a(k + 1, k) > 0) alpha = -alpha;
    u[k + 1] = a(k + 1, k) - alpha;
    for (int i = k + 2; i < n; ++i) u[i] = a(i, k);
    double unorm2 = 0.0;
    for (int i = k + 1; i < n; ++i) unorm2 += u[i] * u[i];
    if (unorm2 == 0.0) continue;
    const double beta = 2.0 / unorm2;
    betas[k] = beta;
    // p = beta A u ; K = p - (beta/2)(u.p) u ; A <- A - u K^T - K u^T.
    // A is symmetric, so A u is a sum of the rows a(j, .) weighted by u[j],
    // four rows per pass: independent lanes over i, a quarter of the stores
    std::fill(pvec.begin() + k, pvec.end(), 0.0);
    int j = k + 1;
    for (; j + 3 < n; j += 4) {
      const double u0 = u[j], u1 = u[j + 1], u2 = u[j + 2], u3 = u[j + 3];
      const double *a0 = &a(j, 0), *a1 = &a(j + 1, 0), *a2 = &a(j + 2, 0), *a3 = &a(j + 3, 0);
      for (int i = k; i < n; ++i) pvec[i] += (a0[i] * u0 + a1[i] * u1) + (a2[i] * u2 + a3[i] * u3);
    }
    for (; j < n; ++j) {
      const double uj = u[j], *aj = &a(j, 0);
      for (int i = k; i < n; ++i) pvec[i] += aj[i] * uj;
    }
    for (int i = k; i < n; ++i) pvec[i] *= beta;
    double up = 0.0;
    for (int i = k + 1; i < n; ++i) up += u[i] * pvec[i];
    for (int i = k; i < n; ++i) kvec[i] = pvec[i] - 0.5 * beta * up * u[i];
    // the rank-2 update on the upper triangle, mirrored: A stays exactly
    // symmetric
    for (int i = k; i < n; ++i) {
      const double ui = u[i], ki = kvec[i];
      for (int c = i; c < n; ++c) a(i, c) -= ui * kvec[c] + ki * u[c];
    }
    for (int i = k; i < n; ++i)
      for (int c = i + 1; c < n; ++c) a(c, i) = a(i, c);
  }
  // Q by backward accumulation: Q <- H_k Q for k = n-3 .. 0, starting from
  // the identity.  H_{k+1} .. H_{n-3} touch only indices above k + 1, so
  // each step works on the trailing block of rows and columns k + 1 .. n-1:
  // t = u_k^T Q (a sum of rows of Q), then Q <- Q - beta_k u_k t
  std::vector<double> Q((size_t)n * n, 0.0), t(n);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  for (int k = n - 3; k >= 0; --k) {
    const double beta = betas[k];
    if (beta == 0.0) continue;
    const double *u = &Us[(size_t)k * n];
    std::fill(t.begin() + k + 1, t.end(), 0.0);
    for (int i = k + 1; i < n; ++i) {
      const double ui = u[i], *qi = &Q[(size_t)i * n];
      for (int c = k + 1; c < n; ++c) t[c] += ui * qi[c];
    }
    for (int c = k + 1; c < n; ++c) t[c] *= beta;
    for (int i = k + 1; i < n; ++i) {
      const double ui = u[i];
      double *qi = &Q[(size_t)i * n];
      for (int c = k + 1; c < n; ++c) qi[c] -= ui * t[c];
    }
  }
  // the QR steps rotate pairs of columns of Q: keep Q transposed so that
  // each rotation runs over two contiguous rows
  std::vector<double> QT((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < n; ++c) QT[(size_t)c * n + i] = Q[(size_t)i * n + c];
  auto qt = [&](int k, int i) -> double & { return QT[(size_t)k * n + i]; };
  std::vector<double> d(n), e(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = a(i, i);
  for (int i = 0; i + 1 < n; ++i) e[i] = a(i + 1, i);
  // implicit symmetric QR on (d, e), deflating from the bottom
  auto small = [&](int i) { return std::fabs(e[i]) <= 2.3e-16 * (std::fabs(d[i]) + std::fabs(d[i + 1])); };
  int hi = n - 1, iters = 0;
  while (hi > 0) {
    if (small(hi - 1)) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int st = hi - 1;
    while (st > 0 && !small(st - 1)) --st;
    if (st > 0) e[st - 1] = 0.0;
    if (++iters > 100 * n) return false;
    // Wilkinson shift from the trailing 2x2 block
    double dd = 0.5 * (d[hi - 1] - d[hi]);
    double ee = e[hi - 1];
    double mu = d[hi] - ee * ee / (dd + (dd >= 0 ? 1.0 : -1.0) * std::hypot(dd, ee));
    double x = d[st] - mu, z = e[st];
    for (int k = st; k < hi; ++k) {
      double r = std::hypot(x, z);
      double c = r == 0.0 ? 1.0 : x / r, s = r == 0.0 ? 0.0 : z / r;
      if (k > st) e[k - 1] = r;
      double d0 = d[k], d1 = d[k + 1], e0 = e[k];
      d[k] = c * c * d0 + 2 * c * s * e0 + s * s * d1;
      d[k + 1] = s * s * d0 - 2 * c * s * e0 + c * c * d1;
      e[k] = c * s * (d1 - d0) + (c * c - s * s) * e0;
      if (k + 1 < hi) {
        x = e[k];
        z = s * e[k + 1];
        e[k + 1] *= c;
      }
      double *r0 = &qt(k, 0), *r1 = &qt(k + 1, 0);
      for (int i = 0; i < n; ++i) {
        const double qk = r0[i], qk1 = r1[i];
        r0[i] = c * qk + s * qk1;
        r1[i] = -s * qk + c * qk1;
      }
    }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return d[x] < d[y]; });
  evals.assign(n, 0.0);
  rows.assign((size_t)n * n, 0.0);
  for (int k = 0; k < n; ++k) {
    int c = order[k];
    evals[k] = d[c];
    int imax = 0;
    double big = -1.0;
    for (int i = 0; i < n; ++i)
      if (std::fabs(qt(c, i)) > big) { big = std::fabs(qt(c, i)); imax = i; }
    double sg = qt(c, imax) < 0 ? -1.0 : 1.0;
    for (int i = 0; i < n; ++i) rows[(size_t)k * n + i] = sg * qt(c, i);
  }
  return true;
}

// Node tables of the pair matrices (Sec. 2.2 Eq. vpot with unit weight
// functions in the p^2 dp measure): n_nodes GL nodes per p bin, their
// weights times p^2, and 1/sqrt(bin volume).  The matrices themselves are
// formed on the device (pair.cu).
void pair_nodes(int N, const double *edges, int n_nodes, std::vector<double> &pn, std::vector<double> &pw,
                std::vector<double> &rsB) {
  std::vector<double> t(n_nodes), w(n_nodes);
  gauss_legendre(n_nodes, t.data(), w.data());
  pn.assign((size_t)N * n_nodes, 0.0);
  pw.assign((size_t)N * n_nodes, 0.0);
  rsB.assign(N, 0.0);
  for (int i = 0; i < N; ++i) {
    const double lo = edges[i], hi = edges[i + 1];
    const double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
    for (int a_ = 0; a_ < n_nodes; ++a_) {
      const double p = mid + half * t[a_];
      pn[(size_t)i * n_nodes + a_] = p;
      pw[(size_t)i * n_nodes + a_] = half * w[a_] * p * p;
    }
    rsB[i] = 1.0 / std::sqrt(shell_volume(lo, hi));
  }
}

// h1 = diag(<p^2>) + v of every channel, <p^2> the bin average of p^2 in the
// p^2 dp measure
void pair_h(int N, const double *edges, int n_ch, const std::vector<std::vector<double>> &v,
            std::vector<std::vector<double>> &h) {
  h = v;
  for (int l = 0; l < n_ch; ++l)
    for (int i = 0; i < N; ++i) {
      const double lo = edges[i], hi = edges[i + 1];
      const double lo2 = lo * lo, hi2 = hi * hi;
      const double p5 = (hi - lo) * (hi2 * hi2 + hi2 * hi * lo + hi2 * lo2 + hi * lo * lo2 + lo2 * lo2) / 5.0;
      h[l][(size_t)i * N + i] += p5 / shell_volume(lo, hi);
    }
}

// eps, O (eigenvectors as rows) of h1; empty on failure
void pair_eig(int N, const std::vector<double> &h, std::vector<double> &eps, std::vector<double> &O) {
  if (!sym_eig(N, h, eps, O)) {
    eps.clear();
    O.clear();
  }
}

}  // namespace wpcd
