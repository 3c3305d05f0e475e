/*
 * wpcd_oracle.c -- plain, slow FP64 CPU oracle for the wave-packet continuum
 * discretisation (WPCD) Faddeev method of Pomerantsev, Kukulin, Rubtsova and
 * Sakhiev, "Fast GPU-based calculations in few-body quantum scattering"
 * (arXiv:1508.07441).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library in
 * paper_1508_07441_gb300/; the two are written independently and compared.
 *
 * Every function follows the passage of the paper named in its comment.
 * Where the paper defers a formula to its references, the reading used here
 * is stated in the comment (units hbar = m = 1, three identical spinless
 * bosons, total orbital momentum L = 0, channels alpha = (l, lambda = l)).
 *
 * Conventions shared with the CUDA path (interface conventions, each written
 * out independently on both sides):
 *   - cell index c = i*M + j (p-bin i, q-bin j); vector index
 *     r = ch*N*M + k*M + j; complex vectors stored as interleaved (re, im).
 *   - GL node inside [lo, hi]:  mid + half*t, with half = 0.5*(hi-lo),
 *     mid = 0.5*(hi+lo), each operation rounded separately.
 *   - recoupled squared momenta (canonical FMA order):
 *       p'^2 = fma((0.75*p)*q, y, (p*p)*0.25 + (q*q)*0.5625)
 *       q'^2 = fma(-(p*q),     y, (p*p) + (q*q)*0.25)
 *   - binning against squared edges e2[k] = e[k]*e[k]: bin k holds
 *     [e2[k], e2[k+1]), the last bin also holds e2[N]; values above e2[N]
 *     leave the grid.
 *   - (l, l') pair order: l ascending, then l' ascending, l + l' even.
 *
 * Parity status: the node-binned P0 is an approximation (the method's own
 * quadrature); it is pinned by the l = 0 sum rule, by convergence to the
 * exact cell-overlap integral and by the symmetry of the exact overlap.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zdouble;

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_ENOCONV -4
#define ORC_EBREAKDOWN -5
#define ORC_ENOBOUND -7

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rules.  The paper integrates every matrix element with     */
/* Gaussian quadratures (Sec. 4.2, item c; the 48-point rule of Eq. Agau).   */
/* Two independent algorithms are kept so that each can pin the other.      */
/* ------------------------------------------------------------------------ */

/* Algorithm 1: Newton iteration on the three-term Legendre recurrence,
 * carried out in long double and rounded once.  Nodes ascending. */
int orc_gl_newton(int n, double *x, double *w) {
  if (n < 1) return ORC_EINVAL;
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    long double z = cosl(pi * ((long double)i + 0.75L) / ((long double)n + 0.5L));
    long double pn = 0.0L, pm = 0.0L, dp = 1.0L;
    for (int it = 0; it < 100; ++it) {
      /* P_n(z) and P_{n-1}(z) by the three-term recurrence */
      long double p0 = 1.0L, p1 = z;
      for (int k = 1; k < n; ++k) {
        long double p2 = ((2.0L * k + 1.0L) * z * p1 - (long double)k * p0) / (k + 1.0L);
        p0 = p1;
        p1 = p2;
      }
      pn = (n == 1) ? z : p1;
      pm = (n == 1) ? 1.0L : p0;
      dp = (long double)n * (z * pn - pm) / (z * z - 1.0L);
      long double dz = pn / dp;
      z -= dz;
      if (fabsl(dz) <= 1e-30L * (1.0L + fabsl(z))) break;
    }
    {
      long double p0 = 1.0L, p1 = z;
      for (int k = 1; k < n; ++k) {
        long double p2 = ((2.0L * k + 1.0L) * z * p1 - (long double)k * p0) / (k + 1.0L);
        p0 = p1;
        p1 = p2;
      }
      pn = (n == 1) ? z : p1;
      pm = (n == 1) ? 1.0L : p0;
      dp = (long double)n * (z * pn - pm) / (z * z - 1.0L);
    }
    /* i = 0 gives the largest node; store ascending */
    x[n - 1 - i] = (double)z;
    w[n - 1 - i] = (double)(2.0L / ((1.0L - z * z) * dp * dp));
  }
  return ORC_OK;
}

/* Cyclic Jacobi eigenvalue algorithm for a real symmetric n x n matrix
 * (row-major, destroyed).  On return evals ascending and evecs[k*n + i] is
 * component i of eigenvector k, normalised, with its largest-magnitude
 * component positive (sign convention of the rotation matrix O). */
int orc_jacobi_eigh(int n, double *A, double *evals, double *evecs) {
  if (n < 1) return ORC_EINVAL;
  double *V = (double *)malloc(sizeof(double) * (size_t)n * n);
  if (!V) return ORC_ENOMEM;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double a = A[(size_t)i * n + j];
        tot += a * a;
        if (i != j) off += a * a;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) { /* columns p, q */
          double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) { /* rows p, q */
          double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) { /* accumulate rotations: columns of V */
          double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  /* sort ascending (selection sort: n <= a few hundred) */
  int *idx = (int *)malloc(sizeof(int) * n);
  if (!idx) { free(V); return ORC_ENOMEM; }
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 0; i < n; ++i) {
    int best = i;
    for (int j = i + 1; j < n; ++j)
      if (A[(size_t)idx[j] * n + idx[j]] < A[(size_t)idx[best] * n + idx[best]]) best = j;
    int t = idx[i]; idx[i] = idx[best]; idx[best] = t;
  }
  for (int k = 0; k < n; ++k) {
    int col = idx[k];
    evals[k] = A[(size_t)col * n + col];
    double big = 0.0; int im = 0;
    for (int i = 0; i < n; ++i)
      if (fabs(V[(size_t)i * n + col]) > big) { big = fabs(V[(size_t)i * n + col]); im = i; }
    double sg = V[(size_t)im * n + col] < 0 ? -1.0 : 1.0;
    for (int i = 0; i < n; ++i) evecs[(size_t)k * n + i] = sg * V[(size_t)i * n + col];
  }
  free(idx);
  free(V);
  return ORC_OK;
}

/* Algorithm 2 (Golub-Welsch): nodes are the eigenvalues of the symmetric
 * tridiagonal Jacobi matrix of the Legendre recurrence, weights are twice the
 * squared first components of its eigenvectors. */
int orc_gl_golub_welsch(int n, double *x, double *w) {
  if (n < 1) return ORC_EINVAL;
  double *J = (double *)calloc((size_t)n * n, sizeof(double));
  double *ev = (double *)malloc(sizeof(double) * (size_t)n * n);
  if (!J || !ev) { free(J); free(ev); return ORC_ENOMEM; }
  for (int k = 1; k < n; ++k) {
    double b = k / sqrt(4.0 * k * k - 1.0);
    J[(size_t)(k - 1) * n + k] = b;
    J[(size_t)k * n + (k - 1)] = b;
  }
  int st = orc_jacobi_eigh(n, J, x, ev);
  if (st == ORC_OK)
    for (int k = 0; k < n; ++k) w[k] = 2.0 * ev[(size_t)k * n + 0] * ev[(size_t)k * n + 0];
  free(J);
  free(ev);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Packet grids (Sec. 2.2, Eq. ip and Eq. theta_p; Sec. 2.4, Eq. xij).       */
/* The paper fixes no mapping; the tangent map p_k = s tan(pi k/(2(N+1))),   */
/* s chosen so that p_N = p_max, is the reading used here.                   */
/* ------------------------------------------------------------------------ */
void orc_tangent_edges(int N, double pmax, double *e) {
  const double pi = 3.14159265358979323846;
  double s = pmax / tan(pi * N / (2.0 * (N + 1)));
  for (int k = 0; k <= N; ++k) e[k] = s * tan(pi * k / (2.0 * (N + 1)));
  e[0] = 0.0;
  e[N] = pmax;
}

/* Normalisation of a unit-weight packet in the p^2 dp measure (Eq. ip with
 * f = 1): B_i = (p_{i+1}^3 - p_i^3)/3. */
static double bnorm(double lo, double hi) { return (hi - lo) * (hi * hi + hi * lo + lo * lo) / 3.0; }

/* ------------------------------------------------------------------------ */
/* Pair interaction (Sec. 2.2, Eq. vpot).  Reading: V(r) = sum_k V_k        */
/* exp(-r^2/a_k), partial-wave momentum states normalised to delta(p-p')/p^2,*/
/*   v_l(p,p') = (2/pi) int r^2 j_l(pr) V(r) j_l(p'r) dr                     */
/*             = sum_k V_k/(2 sqrt(pi) alpha_k^{3/2})                        */
/*               * exp(-(p-p')^2/(4 alpha_k)) * [exp(-z) i_l(z)],            */
/* alpha_k = 1/a_k, z = p p'/(2 alpha_k), i_l the modified spherical Bessel. */
/* ------------------------------------------------------------------------ */

/* exp(-z) i_l(z), z >= 0.  Power series (all terms positive) for z <= 30;
 * the terminating expansion of i_l in powers of 1/z above. */
double orc_sph_i_scaled(int l, double z) {
  if (z < 0) return NAN;
  if (z <= 30.0) {
    /* i_l(z) = z^l sum_k (z^2/2)^k / (k! (2l+2k+1)!!) */
    double dfac = 1.0; /* (2l+1)!! */
    for (int m = 1; m <= 2 * l + 1; m += 2) dfac *= m;
    double term = 1.0 / dfac, sum = term, h = 0.5 * z * z;
    for (int k = 1; k < 400; ++k) {
      term *= h / ((double)k * (2.0 * l + 2.0 * k + 1.0));
      sum += term;
      if (term < 1e-18 * sum) break;
    }
    return pow(z, l) * sum * exp(-z);
  }
  /* exp(-z) i_l(z) = (1/2z) [ sum_k (-1)^k c_k (2z)^-k
   *                           + (-1)^(l+1) exp(-2z) sum_k c_k (2z)^-k ],
   * c_k = (l+k)! / (k! (l-k)!). */
  double s1 = 0.0, s2 = 0.0, x = 1.0 / (2.0 * z), pw = 1.0;
  for (int k = 0; k <= l; ++k) {
    double ck = 1.0;
    for (int m = l - k + 1; m <= l + k; ++m) ck *= m; /* (l+k)!/(l-k)! */
    for (int m = 2; m <= k; ++m) ck /= m;           /* / k! */
    s1 += ((k & 1) ? -1.0 : 1.0) * ck * pw;
    s2 += ck * pw;
    pw *= x;
  }
  double sg = ((l + 1) & 1) ? -1.0 : 1.0;
  return (s1 + sg * exp(-2.0 * z) * s2) / (2.0 * z);
}

double orc_vl(int l, double p, double pp, int nt, const double *Vk, const double *ak) {
  const double pi = 3.14159265358979323846;
  double v = 0.0;
  for (int t = 0; t < nt; ++t) {
    double al = 1.0 / ak[t];
    double z = p * pp / (2.0 * al);
    v += Vk[t] / (2.0 * sqrt(pi) * al * sqrt(al)) * exp(-(p - pp) * (p - pp) / (4.0 * al)) *
         orc_sph_i_scaled(l, z);
  }
  return v;
}

/* Free-packet matrix of v (Eq. vpot, double bin integral with n_nodes GL
 * points per bin and f = 1 in the p^2 dp measure), the pair Hamiltonian
 * h1 = diag(<p^2>_i) + v, and its diagonalisation (Eq. exp_z): eps ascending
 * and O[k*N + i] = <x_i|z_k>.  The lowest negative eps are bound states. */
int orc_pair(int N, const double *e, int n_nodes, int l, int nt, const double *Vk,
             const double *ak, double *v, double *h, double *eps, double *O) {
  if (N < 1 || n_nodes < 1) return ORC_EINVAL;
  double *t = (double *)malloc(sizeof(double) * n_nodes);
  double *wt = (double *)malloc(sizeof(double) * n_nodes);
  double *P = (double *)malloc(sizeof(double) * (size_t)N * n_nodes);
  double *W = (double *)malloc(sizeof(double) * (size_t)N * n_nodes);
  double *H = (double *)malloc(sizeof(double) * (size_t)N * N);
  if (!t || !wt || !P || !W || !H) { free(t); free(wt); free(P); free(W); free(H); return ORC_ENOMEM; }
  orc_gl_newton(n_nodes, t, wt);
  for (int i = 0; i < N; ++i) {
    double lo = e[i], hi = e[i + 1], half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
    for (int a = 0; a < n_nodes; ++a) {
      double p = mid + half * t[a];
      P[(size_t)i * n_nodes + a] = p;
      W[(size_t)i * n_nodes + a] = half * wt[a] * p * p;
    }
  }
  for (int i = 0; i < N; ++i) {
    double Bi = bnorm(e[i], e[i + 1]);
    for (int ip = 0; ip < N; ++ip) {
      double Bip = bnorm(e[ip], e[ip + 1]);
      double s = 0.0;
      for (int a = 0; a < n_nodes; ++a)
        for (int b = 0; b < n_nodes; ++b)
          s += W[(size_t)i * n_nodes + a] * W[(size_t)ip * n_nodes + b] *
               orc_vl(l, P[(size_t)i * n_nodes + a], P[(size_t)ip * n_nodes + b], nt, Vk, ak);
      v[(size_t)i * N + ip] = s / sqrt(Bi * Bip);
    }
  }
  for (int i = 0; i < N; ++i)
    for (int ip = 0; ip < N; ++ip) {
      double x = v[(size_t)i * N + ip];
      if (i == ip) {
        double lo = e[i], hi = e[i + 1];
        /* <p^2>_i = int p^4 dp / B_i = (hi^5 - lo^5) / (5 B_i) */
        double p5 = (hi - lo) * (hi * hi * hi * hi + hi * hi * hi * lo + hi * hi * lo * lo +
                                 hi * lo * lo * lo + lo * lo * lo * lo) / 5.0;
        x += p5 / bnorm(lo, hi);
      }
      H[(size_t)i * N + ip] = x;
      if (h) h[(size_t)i * N + ip] = x;
    }
  /* symmetrise against quadrature round-off before diagonalising */
  for (int i = 0; i < N; ++i)
    for (int ip = i + 1; ip < N; ++ip) {
      double m = 0.5 * (H[(size_t)i * N + ip] + H[(size_t)ip * N + i]);
      H[(size_t)i * N + ip] = H[(size_t)ip * N + i] = m;
    }
  int st = orc_jacobi_eigh(N, H, eps, O);
  free(t); free(wt); free(P); free(W); free(H);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Lattice permutation matrix P0 (Sec. 3.2, Eqs. perm_z, perm and gal).      */
/* Reading for spinless bosons, L = 0: with y = p^.q^ the set-2 momenta are  */
/* p' = -(p/2 + 3q/4), q' = p - q/2, and summing both cyclic permutations    */
/*  P0[(l,c),(l',c')] = delta_{l+l' even} sqrt((2l+1)(2l'+1))                */
/*       / sqrt(B_i Bq_j B_i' Bq_j')                                         */
/*       * int_{cell c} p^2 dp q^2 dq int_{-1}^{1} dy P_l(y) P_l'(y')        */
/*         theta(p' in bin i') theta(q' in bin j').                          */
/* The integral is replaced by the GL node sum over (p, q, y), each node     */
/* binned into its target cell (the node-binning estimate).                  */
/* ------------------------------------------------------------------------ */

int orc_n_pairs(int n_ch) {
  int n = 0;
  for (int l = 0; l < n_ch; ++l)
    for (int lp = 0; lp < n_ch; ++lp)
      if (((l + lp) & 1) == 0) ++n;
  return n;
}

static void pair_list(int n_ch, int *pl, int *plp) {
  int n = 0;
  for (int l = 0; l < n_ch; ++l)
    for (int lp = 0; lp < n_ch; ++lp)
      if (((l + lp) & 1) == 0) { pl[n] = l; plp[n] = lp; ++n; }
}

/* bin of a squared momentum: number of interior squared edges <= x2; -1 when
 * x2 lies above the last squared edge (outside the grid). */
static int bin_of(double x2, const double *e2, int n) {
  if (x2 > e2[n]) return -1;
  int k = 0;
  while (k + 1 < n && e2[k + 1] <= x2) ++k;
  return k;
}

static void legendre(int lmax, double y, double *P) {
  P[0] = 1.0;
  if (lmax >= 1) P[1] = y;
  for (int n = 1; n < lmax; ++n) P[n + 1] = ((2.0 * n + 1.0) * y * P[n] - n * P[n - 1]) / (n + 1.0);
}

typedef struct {
  int N, M, np_, nq, nx;
  double *pn, *wpn, *qn, *wqn, *yn, *wyn; /* nodes and weights incl. p^2, q^2 */
  double *pe2, *qe2;
} lattice;

static int lattice_init(lattice *L, int N, const double *pe, int M, const double *qe, int np_,
                        int nq, int nx) {
  memset(L, 0, sizeof(*L));
  L->N = N; L->M = M; L->np_ = np_; L->nq = nq; L->nx = nx;
  double *tp = malloc(sizeof(double) * np_), *wp = malloc(sizeof(double) * np_);
  double *tq = malloc(sizeof(double) * nq), *wq = malloc(sizeof(double) * nq);
  L->pn = malloc(sizeof(double) * (size_t)N * np_); L->wpn = malloc(sizeof(double) * (size_t)N * np_);
  L->qn = malloc(sizeof(double) * (size_t)M * nq); L->wqn = malloc(sizeof(double) * (size_t)M * nq);
  L->yn = malloc(sizeof(double) * nx); L->wyn = malloc(sizeof(double) * nx);
  L->pe2 = malloc(sizeof(double) * (N + 1)); L->qe2 = malloc(sizeof(double) * (M + 1));
  if (!tp || !wp || !tq || !wq || !L->pn || !L->wpn || !L->qn || !L->wqn || !L->yn || !L->wyn ||
      !L->pe2 || !L->qe2) {
    free(tp); free(wp); free(tq); free(wq);
    return ORC_ENOMEM;
  }
  orc_gl_newton(np_, tp, wp);
  orc_gl_newton(nq, tq, wq);
  orc_gl_newton(nx, L->yn, L->wyn);
  for (int i = 0; i < N; ++i) {
    double half = 0.5 * (pe[i + 1] - pe[i]), mid = 0.5 * (pe[i + 1] + pe[i]);
    for (int a = 0; a < np_; ++a) {
      double p = mid + half * tp[a];
      L->pn[(size_t)i * np_ + a] = p;
      L->wpn[(size_t)i * np_ + a] = half * wp[a] * p * p;
    }
  }
  for (int j = 0; j < M; ++j) {
    double half = 0.5 * (qe[j + 1] - qe[j]), mid = 0.5 * (qe[j + 1] + qe[j]);
    for (int b = 0; b < nq; ++b) {
      double q = mid + half * tq[b];
      L->qn[(size_t)j * nq + b] = q;
      L->wqn[(size_t)j * nq + b] = half * wq[b] * q * q;
    }
  }
  for (int k = 0; k <= N; ++k) L->pe2[k] = pe[k] * pe[k];
  for (int k = 0; k <= M; ++k) L->qe2[k] = qe[k] * qe[k];
  free(tp); free(wp); free(tq); free(wq);
  return ORC_OK;
}

static void lattice_free(lattice *L) {
  free(L->pn); free(L->wpn); free(L->qn); free(L->wqn); free(L->yn); free(L->wyn);
  free(L->pe2); free(L->qe2);
}

/* Map one node (p, q, y) to its target cell; -1 if it leaves the grid.
 * Also returns y' = p'^.q'^ (clamped to [-1, 1]). */
static int map_node(const lattice *L, double p, double q, double y, double *yp) {
  double A = (0.75 * p) * q;
  double Bp = (p * p) * 0.25 + (q * q) * 0.5625;
  double Cq = -(p * q);
  double Dq = (p * p) + (q * q) * 0.25;
  double p2 = fma(A, y, Bp);
  double q2 = fma(Cq, y, Dq);
  /* p'.q' = -p^2/2 - p q y / 2 + 3 q^2 / 8 */
  double num = -0.5 * p * p - 0.5 * p * q * y + 0.375 * q * q;
  double den = sqrt(fmax(p2, 0.0) * fmax(q2, 0.0));
  double c = den > 0.0 ? num / den : 0.0;
  if (c > 1.0) c = 1.0;
  if (c < -1.0) c = -1.0;
  *yp = c;
  int ip = bin_of(p2, L->pe2, L->N);
  int jq = bin_of(q2, L->qe2, L->M);
  if (ip < 0 || jq < 0) return -1;
  return ip * L->M + jq;
}

/* Step 2a (pre-selection, Sec. 3.3 and Sec. 4.2 item d): for every source
 * cell, the number of distinct target cells hit by at least one node.
 * row_ptr has N*M+1 entries.  Returns nnz (number of cell pairs) or < 0. */
int64_t orc_P0_count(int N, const double *pe, int M, const double *qe, int np_, int nq, int nx,
                     int64_t *row_ptr) {
  lattice L;
  if (lattice_init(&L, N, pe, M, qe, np_, nq, nx) != ORC_OK) return ORC_ENOMEM;
  int ncell = N * M;
  int err = 0;
#pragma omp parallel
  {
    unsigned char *seen = calloc((size_t)ncell, 1);
    int *touched = malloc(sizeof(int) * (size_t)np_ * nq * nx);
    if (!seen || !touched) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 8)
    for (int c = 0; c < ncell; ++c) {
      if (!seen || !touched) continue;
      int i = c / M, j = c % M, nt = 0;
      for (int a = 0; a < np_; ++a)
        for (int b = 0; b < nq; ++b)
          for (int x = 0; x < nx; ++x) {
            double yp;
            int t = map_node(&L, L.pn[(size_t)i * np_ + a], L.qn[(size_t)j * nq + b], L.yn[x], &yp);
            if (t >= 0 && !seen[t]) { seen[t] = 1; touched[nt++] = t; }
          }
      row_ptr[c + 1] = nt;
      for (int k = 0; k < nt; ++k) seen[touched[k]] = 0;
    }
    free(seen);
    free(touched);
  }
  lattice_free(&L);
  if (err) return ORC_ENOMEM;
  row_ptr[0] = 0;
  for (int c = 0; c < ncell; ++c) row_ptr[c + 1] += row_ptr[c];
  return row_ptr[ncell];
}

static int cmp_int(const void *a, const void *b) {
  int x = *(const int *)a, y = *(const int *)b;
  return (x > y) - (x < y);
}

/* Step 2b: node-binned values, unnormalised (the bare node sums), columns
 * ascending within each row; val is [nnz][n_pairs].  outgrid (optional,
 * [N*M][n_pairs]) receives the weight of nodes that leave the grid.  absval
 * (optional, [nnz][n_pairs]) receives sum_nodes W |P_l(y)|, the magnitude
 * that bounds every node term (|P_l'| <= 1) and so sets the scale of the
 * rounding error of each element: elements whose terms cancel exactly (e.g.
 * l' = 0 with the GL rule integrating P_l(y) to zero) are rounding noise of
 * that size, and a node evaluated in FP32 carries an absolute error of order
 * eps_32 times its W |P_l(y)| even where P_l'(y') passes through zero. */
int orc_P0_fill(int N, const double *pe, int M, const double *qe, int np_, int nq, int nx,
                int n_ch, const int64_t *row_ptr, int32_t *col, double *val, double *outgrid,
                double *absval) {
  lattice L;
  if (n_ch < 1) return ORC_EINVAL;
  if (lattice_init(&L, N, pe, M, qe, np_, nq, nx) != ORC_OK) return ORC_ENOMEM;
  int npair = orc_n_pairs(n_ch);
  int pl[64], plp[64];
  pair_list(n_ch, pl, plp);
  int ncell = N * M;
  int err = 0;
#pragma omp parallel
  {
    double *acc = calloc((size_t)ncell * npair, sizeof(double));
    double *aacc = absval ? calloc((size_t)ncell * npair, sizeof(double)) : NULL;
    unsigned char *seen = calloc((size_t)ncell, 1);
    int *touched = malloc(sizeof(int) * (size_t)np_ * nq * nx);
    double Py[32], Pyp[32], og[64];
    if (!acc || !seen || !touched || (absval && !aacc)) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 8)
    for (int c = 0; c < ncell; ++c) {
      if (!acc || !seen || !touched || (absval && !aacc)) continue;
      int i = c / M, j = c % M, nt = 0;
      for (int k = 0; k < npair; ++k) og[k] = 0.0;
      for (int a = 0; a < np_; ++a)
        for (int b = 0; b < nq; ++b)
          for (int x = 0; x < nx; ++x) {
            double p = L.pn[(size_t)i * np_ + a], q = L.qn[(size_t)j * nq + b], y = L.yn[x];
            double W = L.wpn[(size_t)i * np_ + a] * L.wqn[(size_t)j * nq + b] * L.wyn[x];
            double yp;
            int t = map_node(&L, p, q, y, &yp);
            legendre(n_ch - 1, y, Py);
            legendre(n_ch - 1, yp, Pyp);
            if (t < 0) {
              for (int k = 0; k < npair; ++k) og[k] += W * Py[pl[k]] * Pyp[plp[k]];
              continue;
            }
            if (!seen[t]) { seen[t] = 1; touched[nt++] = t; }
            for (int k = 0; k < npair; ++k) {
              double term = W * Py[pl[k]] * Pyp[plp[k]];
              acc[(size_t)t * npair + k] += term;
              if (aacc) aacc[(size_t)t * npair + k] += W * fabs(Py[pl[k]]);
            }
          }
      if (row_ptr[c + 1] - row_ptr[c] != nt) {
#pragma omp atomic write
        err = 2;
      }
      qsort(touched, nt, sizeof(int), cmp_int);
      int64_t o = row_ptr[c];
      for (int k = 0; k < nt && o + k < row_ptr[c + 1]; ++k) {
        int t = touched[k];
        col[o + k] = t;
        for (int m = 0; m < npair; ++m) {
          val[(o + k) * npair + m] = acc[(size_t)t * npair + m];
          acc[(size_t)t * npair + m] = 0.0;
          if (aacc) {
            absval[(o + k) * npair + m] = aacc[(size_t)t * npair + m];
            aacc[(size_t)t * npair + m] = 0.0;
          }
        }
        seen[t] = 0;
      }
      if (outgrid)
        for (int k = 0; k < npair; ++k) outgrid[(size_t)c * npair + k] = og[k];
    }
    free(acc);
    free(aacc);
    free(seen);
    free(touched);
  }
  lattice_free(&L);
  return err == 1 ? ORC_ENOMEM : (err == 2 ? ORC_EINVAL : ORC_OK);
}

/* Un-binned node sums per source cell: sum over all nodes of
 * W P_l(y) P_l'(y'), whether or not the node stays inside the grid.  This is
 * the right-hand side of the sum rule. */
int orc_P0_node_totals(int N, const double *pe, int M, const double *qe, int np_, int nq, int nx,
                       int n_ch, double *tot) {
  lattice L;
  if (lattice_init(&L, N, pe, M, qe, np_, nq, nx) != ORC_OK) return ORC_ENOMEM;
  int npair = orc_n_pairs(n_ch);
  int pl[64], plp[64];
  pair_list(n_ch, pl, plp);
#pragma omp parallel for schedule(dynamic, 8)
  for (int c = 0; c < N * M; ++c) {
    int i = c / M, j = c % M;
    double Py[32], Pyp[32], s[64];
    for (int k = 0; k < npair; ++k) s[k] = 0.0;
    for (int a = 0; a < np_; ++a)
      for (int b = 0; b < nq; ++b)
        for (int x = 0; x < nx; ++x) {
          double p = L.pn[(size_t)i * np_ + a], q = L.qn[(size_t)j * nq + b], y = L.yn[x];
          double W = L.wpn[(size_t)i * np_ + a] * L.wqn[(size_t)j * nq + b] * L.wyn[x];
          double yp;
          (void)map_node(&L, p, q, y, &yp);
          legendre(n_ch - 1, y, Py);
          legendre(n_ch - 1, yp, Pyp);
          for (int k = 0; k < npair; ++k) s[k] += W * Py[pl[k]] * Pyp[plp[k]];
        }
    for (int k = 0; k < npair; ++k) tot[(size_t)c * npair + k] = s[k];
  }
  lattice_free(&L);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* P0 with variable limits (Sec. 3.2, after Eq. gal: the cell overlap as an */
/* integral with variable limits).  For a GL node (p, q) of the source cell */
/* the recoupled squares are linear in y = p.q/(|p||q|):                    */
/*   p'^2 = A y + Bp,  A = 3 p q / 4 > 0,   q'^2 = C y + Dq,  C = -p q < 0,  */
/* so theta(p' in bin i') theta(q' in bin j') of Eq. perm holds on one      */
/* y-interval, its limits where p'^2 or q'^2 equals the bins' squared edges:*/
/*   p-bin i': y in [(e_i'^2 - Bp)/A, (e_i'+1^2 - Bp)/A]                     */
/*   q-bin j': y in [(f_j'+1^2 - Dq)/C, (f_j'^2 - Dq)/C]                     */
/* intersected with [-1, 1].  P_l(y) P_l'(y') is integrated over it with    */
/* the n_x-point GL rule mapped onto it; the p and q integrals keep the     */
/* cell's GL rule.  Neighbouring targets share the same computed limit, so  */
/* the intervals of one node tile [-1, 1] (those beyond the last edges      */
/* leave the grid).                                                         */
/* ------------------------------------------------------------------------ */

/* the y-interval [ya, yb] of node (p, q) for target (it, jt); returns 1 if
   it is not empty */
static int vl_interval(const lattice *L, double p, double q, int it, int jt, double *ya, double *yb) {
  double A = (0.75 * p) * q, Bp = (p * p) * 0.25 + (q * q) * 0.5625;
  double C = -(p * q), Dq = (p * p) + (q * q) * 0.25;
  double lo = -1.0, hi = 1.0;
  double plo = (L->pe2[it] - Bp) / A, phi = (L->pe2[it + 1] - Bp) / A;
  double qlo = (L->qe2[jt + 1] - Dq) / C, qhi = (L->qe2[jt] - Dq) / C;
  if (plo > lo) lo = plo;
  if (qlo > lo) lo = qlo;
  if (phi < hi) hi = phi;
  if (qhi < hi) hi = qhi;
  *ya = lo;
  *yb = hi;
  return hi > lo;
}

/* y' of the node (p, q) at y, as in the node-binned P0 */
static double vl_yprime(double p, double q, double y) {
  double A = (0.75 * p) * q, Bp = (p * p) * 0.25 + (q * q) * 0.5625;
  double C = -(p * q), Dq = (p * p) + (q * q) * 0.25;
  double p2 = fma(A, y, Bp), q2 = fma(C, y, Dq);
  double num = -0.5 * p * p - 0.5 * p * q * y + 0.375 * q * q;
  double den = sqrt(fmax(p2, 0.0) * fmax(q2, 0.0));
  double c = den > 0.0 ? num / den : 0.0;
  return c > 1.0 ? 1.0 : (c < -1.0 ? -1.0 : c);
}

/* the p-bins and q-bins a node can reach (a superset: the bins whose
   squared-momentum range meets [min, max] of p'^2 and q'^2 over y) */
static void vl_range(const lattice *L, double p, double q, int *i0, int *i1, int *j0, int *j1) {
  double pmin = fabs(0.5 * p - 0.75 * q), pmax = 0.5 * p + 0.75 * q;
  double qmin = fabs(p - 0.5 * q), qmax = p + 0.5 * q;
  *i0 = 0;
  while (*i0 + 1 < L->N && L->pe2[*i0 + 1] <= pmin * pmin * (1.0 - 1e-12)) ++*i0;
  *i1 = *i0;
  while (*i1 + 1 < L->N && L->pe2[*i1 + 1] < pmax * pmax * (1.0 + 1e-12)) ++*i1;
  *j0 = 0;
  while (*j0 + 1 < L->M && L->qe2[*j0 + 1] <= qmin * qmin * (1.0 - 1e-12)) ++*j0;
  *j1 = *j0;
  while (*j1 + 1 < L->M && L->qe2[*j1 + 1] < qmax * qmax * (1.0 + 1e-12)) ++*j1;
}

/* row lengths of the variable-limit P0 (distinct target cells per source
   cell); returns nnz or < 0 */
int64_t orc_P0_vl_count(int N, const double *pe, int M, const double *qe, int np_, int nq, int nx,
                        int64_t *row_ptr) {
  lattice L;
  if (lattice_init(&L, N, pe, M, qe, np_, nq, nx) != ORC_OK) return ORC_ENOMEM;
  int ncell = N * M, err = 0;
#pragma omp parallel
  {
    unsigned char *seen = calloc((size_t)ncell, 1);
    int *touched = malloc(sizeof(int) * (size_t)ncell);
    if (!seen || !touched) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 8)
    for (int c = 0; c < ncell; ++c) {
      if (!seen || !touched) continue;
      int i = c / M, j = c % M, nt = 0;
      for (int a = 0; a < np_; ++a)
        for (int b = 0; b < nq; ++b) {
          double p = L.pn[(size_t)i * np_ + a], q = L.qn[(size_t)j * nq + b], ya, yb;
          int i0, i1, j0, j1;
          vl_range(&L, p, q, &i0, &i1, &j0, &j1);
          for (int it = i0; it <= i1; ++it)
            for (int jt = j0; jt <= j1; ++jt) {
              int t = it * M + jt;
              if (!seen[t] && vl_interval(&L, p, q, it, jt, &ya, &yb)) { seen[t] = 1; touched[nt++] = t; }
            }
        }
      row_ptr[c + 1] = nt;
      for (int k = 0; k < nt; ++k) seen[touched[k]] = 0;
    }
    free(seen);
    free(touched);
  }
  lattice_free(&L);
  if (err) return ORC_ENOMEM;
  row_ptr[0] = 0;
  for (int c = 0; c < ncell; ++c) row_ptr[c + 1] += row_ptr[c];
  return row_ptr[ncell];
}

/* values of the variable-limit P0, unnormalised, in the layout of
   orc_P0_fill (val [nnz][n_pairs], columns ascending); outgrid (optional,
   [N*M][n_pairs]) receives the integral over the y that leave the grid */
int orc_P0_vl_fill(int N, const double *pe, int M, const double *qe, int np_, int nq, int nx, int n_ch,
                   const int64_t *row_ptr, int32_t *col, double *val, double *outgrid) {
  lattice L;
  if (n_ch < 1) return ORC_EINVAL;
  if (lattice_init(&L, N, pe, M, qe, np_, nq, nx) != ORC_OK) return ORC_ENOMEM;
  int npair = orc_n_pairs(n_ch);
  int pl[64], plp[64];
  pair_list(n_ch, pl, plp);
  int ncell = N * M, err = 0;
#pragma omp parallel
  {
    double *acc = calloc((size_t)ncell * npair, sizeof(double));
    unsigned char *seen = calloc((size_t)ncell, 1);
    int *touched = malloc(sizeof(int) * (size_t)ncell);
    double Py[32], Pyp[32], og[64];
    if (!acc || !seen || !touched) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 8)
    for (int c = 0; c < ncell; ++c) {
      if (!acc || !seen || !touched) continue;
      int i = c / M, j = c % M, nt = 0;
      for (int k = 0; k < npair; ++k) og[k] = 0.0;
      for (int a = 0; a < np_; ++a)
        for (int b = 0; b < nq; ++b) {
          double p = L.pn[(size_t)i * np_ + a], q = L.qn[(size_t)j * nq + b], ya, yb;
          double Wpq = L.wpn[(size_t)i * np_ + a] * L.wqn[(size_t)j * nq + b];
          int i0, i1, j0, j1;
          vl_range(&L, p, q, &i0, &i1, &j0, &j1);
          for (int it = i0; it <= i1; ++it)
            for (int jt = j0; jt <= j1; ++jt) {
              if (!vl_interval(&L, p, q, it, jt, &ya, &yb)) continue;
              int t = it * M + jt;
              if (!seen[t]) { seen[t] = 1; touched[nt++] = t; }
              double half = 0.5 * (yb - ya), mid = 0.5 * (ya + yb);
              for (int x = 0; x < nx; ++x) {
                double y = mid + half * L.yn[x];
                double W = Wpq * (half * L.wyn[x]);
                legendre(n_ch - 1, y, Py);
                legendre(n_ch - 1, vl_yprime(p, q, y), Pyp);
                for (int k = 0; k < npair; ++k) {
                  double term = W * Py[pl[k]] * Pyp[plp[k]];
                  acc[(size_t)t * npair + k] += term;
                }
              }
            }
          /* outside the grid: p'^2 above the last p edge (y > yp) or q'^2
             above the last q edge (y < yq); both pieces by the GL rule */
          {
            double A = (0.75 * p) * q, Bp = (p * p) * 0.25 + (q * q) * 0.5625;
            double C = -(p * q), Dq = (p * p) + (q * q) * 0.25;
            double yp = (L.pe2[N] - Bp) / A, yq = (L.qe2[M] - Dq) / C;
            double lo[2], hi[2];
            int npc = 0;
            if (yq >= yp) { lo[0] = -1.0; hi[0] = 1.0; npc = 1; } /* no y inside the grid */
            else {
              if (yq > -1.0) { lo[npc] = -1.0; hi[npc] = yq < 1.0 ? yq : 1.0; ++npc; }
              if (yp < 1.0) { lo[npc] = yp > -1.0 ? yp : -1.0; hi[npc] = 1.0; ++npc; }
            }
            for (int s2 = 0; s2 < npc; ++s2) {
              double half = 0.5 * (hi[s2] - lo[s2]), mid = 0.5 * (hi[s2] + lo[s2]);
              for (int x = 0; x < nx; ++x) {
                double y = mid + half * L.yn[x];
                legendre(n_ch - 1, y, Py);
                legendre(n_ch - 1, vl_yprime(p, q, y), Pyp);
                for (int k = 0; k < npair; ++k) og[k] += Wpq * (half * L.wyn[x]) * Py[pl[k]] * Pyp[plp[k]];
              }
            }
          }
        }
      if (row_ptr[c + 1] - row_ptr[c] != nt) {
#pragma omp atomic write
        err = 2;
      }
      qsort(touched, nt, sizeof(int), cmp_int);
      int64_t o = row_ptr[c];
      for (int k = 0; k < nt && o + k < row_ptr[c + 1]; ++k) {
        int t = touched[k];
        col[o + k] = t;
        for (int m = 0; m < npair; ++m) {
          val[(o + k) * npair + m] = acc[(size_t)t * npair + m];
          acc[(size_t)t * npair + m] = 0.0;
        }
        seen[t] = 0;
      }
      if (outgrid)
        for (int k = 0; k < npair; ++k) outgrid[(size_t)c * npair + k] = og[k];
    }
    free(acc);
    free(seen);
    free(touched);
  }
  lattice_free(&L);
  return err == 1 ? ORC_ENOMEM : (err == 2 ? ORC_EINVAL : ORC_OK);
}

/* Normalisation of Eq. perm: sqrt((2l+1)(2l'+1)) / sqrt(B_i Bq_j B_i' Bq_j'). */
void orc_P0_normalize(int N, const double *pe, int M, const double *qe, int n_ch,
                      const int64_t *row_ptr, const int32_t *col, double *val) {
  int npair = orc_n_pairs(n_ch);
  int pl[64], plp[64];
  pair_list(n_ch, pl, plp);
  for (int c = 0; c < N * M; ++c) {
    int i = c / M, j = c % M;
    double Bc = bnorm(pe[i], pe[i + 1]) * bnorm(qe[j], qe[j + 1]);
    for (int64_t o = row_ptr[c]; o < row_ptr[c + 1]; ++o) {
      int t = col[o], it = t / M, jt = t % M;
      double Bt = bnorm(pe[it], pe[it + 1]) * bnorm(qe[jt], qe[jt + 1]);
      for (int k = 0; k < npair; ++k)
        val[o * npair + k] *= sqrt((2.0 * pl[k] + 1.0) * (2.0 * plp[k] + 1.0)) / sqrt(Bc * Bt);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Channel resolvent G1 (Sec. 2.1 Eq. g_tot; Sec. 2.3 energy averaging;      */
/* Sec. 2.4 channel basis Z_kj).  Reading: every channel state Z_kj has      */
/*   g_kj(E) = (1/Bq_j) int_{bin j} q^2 dq / (E - eps_k - 3q^2/4 + i0),      */
/* eps_k the bound energy or pseudostate eigenvalue, averaged over the       */
/* on-shell energy bin [E_lo, E_hi] = eps_b + 3/4 [q_j0^2, q_j0+1^2] that    */
/* contains E:                                                               */
/*   Re = [Phi_j(E_hi - eps_k) - Phi_j(E_lo - eps_k)] / (D Bq_j),            */
/*   Im = -pi/(D Bq_j) int_{bin j} q^2 dq theta(E_lo < eps_k+3q^2/4 < E_hi), */
/* Phi_j(a) = int_{bin j} q^2 ln|a - 3q^2/4| dq, D = E_hi - E_lo.            */
/* ------------------------------------------------------------------------ */

/* antiderivative of q^2 ln|q + sg*s| (s > 0); the x ln|x| limit is 0 */
static double F_log_lin(double q, double s, double sg) {
  double d = q + sg * s;
  /* q^3 + sg s^3 = (q + sg s)(q^2 - sg q s + s^2) */
  double c = d * (q * q - sg * q * s + s * s) / 3.0;
  double L = (d == 0.0) ? 0.0 : c * log(fabs(d));
  return L - (q * q * q / 9.0 - sg * s * q * q / 6.0 + s * s * q / 3.0);
}

/* closed form of Phi over [qa, qb] */
static double Phi_closed(double qa, double qb, double a) {
  double base = log(0.75) * bnorm(qa, qb);
  if (a > 0.0) {
    double s = sqrt(a / 0.75);
    return (F_log_lin(qb, s, 1.0) + F_log_lin(qb, s, -1.0)) -
           (F_log_lin(qa, s, 1.0) + F_log_lin(qa, s, -1.0)) + base;
  } else if (a < 0.0) {
    double t = sqrt(-a / 0.75);
#define FNEG(q) ((q) * (q) * (q) / 3.0 * log((q) * (q) + t * t) - \
                 2.0 / 3.0 * ((q) * (q) * (q) / 3.0 - t * t * (q) + t * t * t * atan((q) / t)))
    return FNEG(qb) - FNEG(qa) + base;
#undef FNEG
  } else {
#define FZ(q) ((q) > 0.0 ? 2.0 * ((q) * (q) * (q) / 3.0 * log(q) - (q) * (q) * (q) / 9.0) : 0.0)
    return FZ(qb) - FZ(qa) + base;
#undef FZ
  }
}

/* Re part; when neither log argument changes sign across the bin and the
 * on-shell width is small against the distance to the singularity, the
 * difference of logs is integrated directly (log1p) with a 32-point GL rule
 * to avoid cancelling two nearly equal closed forms. */
static double re_g(double qa, double qb, double Elo, double Ehi, double ek, const double *t,
                   const double *w) {
  double D = Ehi - Elo;
  double alo_a = Elo - ek - 0.75 * qa * qa, alo_b = Elo - ek - 0.75 * qb * qb;
  double ahi_a = Ehi - ek - 0.75 * qa * qa, ahi_b = Ehi - ek - 0.75 * qb * qb;
  int same = (alo_a > 0) == (alo_b > 0) && (ahi_a > 0) == (ahi_b > 0) && (alo_a > 0) == (ahi_a > 0) &&
             alo_a != 0 && alo_b != 0 && ahi_a != 0 && ahi_b != 0;
  double mind = fmin(fabs(alo_a), fabs(alo_b));
  if (same && fabs(D) < 0.05 * mind) {
    double half = 0.5 * (qb - qa), mid = 0.5 * (qb + qa), s = 0.0;
    for (int k = 0; k < 32; ++k) {
      double q = mid + half * t[k];
      double den = Elo - ek - 0.75 * q * q;
      s += half * w[k] * q * q * log1p(D / den);
    }
    return s;
  }
  return Phi_closed(qa, qb, Ehi - ek) - Phi_closed(qa, qb, Elo - ek);
}

/* On-shell bin of energy E for bound energy eps_b: j0 with
 * q0 = sqrt(4(E - eps_b)/3) in [q_j0, q_j0+1). */
int orc_onshell(int M, const double *qe, double E, double eps_b, int *j0, double *Elo,
                double *Ehi, double *q0) {
  if (!(E > eps_b)) return ORC_ENOBOUND;
  double q = sqrt((E - eps_b) / 0.75);
  if (!(q < qe[M])) return ORC_EINVAL;
  int j = 0;
  while (j + 1 < M && qe[j + 1] <= q) ++j;
  *j0 = j;
  *Elo = eps_b + 0.75 * qe[j] * qe[j];
  *Ehi = eps_b + 0.75 * qe[j + 1] * qe[j + 1];
  if (q0) *q0 = q;
  return ORC_OK;
}

/* g[(ch*N + k)*M + j] as interleaved complex; eps is [n_ch][N]. */
int orc_G1(int n_ch, int N, const double *eps, int M, const double *qe, double E, double eps_b,
           double *g, int *j0_out, double *D_out) {
  const double pi = 3.14159265358979323846;
  int j0;
  double Elo, Ehi;
  int st = orc_onshell(M, qe, E, eps_b, &j0, &Elo, &Ehi, NULL);
  if (st != ORC_OK) return st;
  double D = Ehi - Elo;
  double t32[32], w32[32];
  orc_gl_newton(32, t32, w32);
#pragma omp parallel for collapse(2)
  for (int ch = 0; ch < n_ch; ++ch)
    for (int k = 0; k < N; ++k) {
      double ek = eps[ch * N + k];
      for (int j = 0; j < M; ++j) {
        double qa = qe[j], qb = qe[j + 1], Bq = bnorm(qa, qb);
        double re = re_g(qa, qb, Elo, Ehi, ek, t32, w32) / (D * Bq);
        double im = 0.0;
        if (Ehi - ek > 0.0) {
          double lo2 = (Elo - ek) / 0.75, hi2 = (Ehi - ek) / 0.75;
          double a = fmax(qa, sqrt(fmax(lo2, 0.0))), b = fmin(qb, sqrt(hi2));
          if (b > a) im = -pi * bnorm(a, b) / (D * Bq);
        }
        size_t r = ((size_t)ch * N + k) * M + j;
        g[2 * r] = re;
        g[2 * r + 1] = im;
      }
    }
  *j0_out = j0;
  *D_out = D;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Kernel of the matrix Faddeev equation (Sec. 3.3, Eq. kernel):             */
/*   K = O P0 Vt G1,  Vt = O^T V1 = v O^T per channel (block N x N, the same */
/* for every q-bin j), O block N x N per channel, G1 diagonal.               */
/* x_out = O P0 Vt (g o x_in); g == NULL means G1 = identity.                */
/* O, Vt are [n_ch][N][N] row-major; vectors are interleaved complex.        */
/* ------------------------------------------------------------------------ */
void orc_kapply(int n_ch, int N, int M, const double *O, const double *Vt, const int64_t *row_ptr,
                const int32_t *col, const double *val, const double *g, const double *x_in,
                double *x_out) {
  size_t n = (size_t)n_ch * N * M;
  int npair = orc_n_pairs(n_ch);
  int pl[64], plp[64];
  pair_list(n_ch, pl, plp);
  zdouble *a = malloc(sizeof(zdouble) * n), *b = malloc(sizeof(zdouble) * n);
  /* a = G1 x */
  for (size_t r = 0; r < n; ++r) {
    zdouble xv = x_in[2 * r] + I * x_in[2 * r + 1];
    zdouble gv = g ? g[2 * r] + I * g[2 * r + 1] : 1.0;
    a[r] = gv * xv;
  }
  /* b = Vt a  (per channel and q-bin) */
#pragma omp parallel for collapse(2)
  for (int ch = 0; ch < n_ch; ++ch)
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < M; ++j) {
        zdouble s = 0.0;
        for (int k = 0; k < N; ++k)
          s += Vt[((size_t)ch * N + i) * N + k] * a[((size_t)ch * N + k) * M + j];
        b[((size_t)ch * N + i) * M + j] = s;
      }
  /* a = P0 b  (cell rows, channel pairs) */
#pragma omp parallel for
  for (int c = 0; c < N * M; ++c) {
    zdouble s[32];
    for (int ch = 0; ch < n_ch; ++ch) s[ch] = 0.0;
    for (int64_t o = row_ptr[c]; o < row_ptr[c + 1]; ++o) {
      int t = col[o];
      for (int k = 0; k < npair; ++k)
        s[pl[k]] += val[o * npair + k] * b[(size_t)plp[k] * N * M + t];
    }
    for (int ch = 0; ch < n_ch; ++ch) a[(size_t)ch * N * M + c] = s[ch];
  }
  /* x_out = O a */
#pragma omp parallel for collapse(2)
  for (int ch = 0; ch < n_ch; ++ch)
    for (int k = 0; k < N; ++k)
      for (int j = 0; j < M; ++j) {
        zdouble s = 0.0;
        for (int i = 0; i < N; ++i)
          s += O[((size_t)ch * N + k) * N + i] * a[((size_t)ch * N + i) * M + j];
        size_t r = ((size_t)ch * N + k) * M + j;
        x_out[2 * r] = creal(s);
        x_out[2 * r + 1] = cimag(s);
      }
  free(a);
  free(b);
}

/* ------------------------------------------------------------------------ */
/* Pade summation of the iterates (Sec. 3.3): c_n = e0^T K^n u0, U00 = sum   */
/* c_n summed by Pade approximants.  Reading: Wynn's epsilon algorithm on    */
/* the partial sums S_n gives the [n+k/k] Pade values at lambda = 1; the     */
/* estimate after S_0..S_m is the deepest even column of the table.          */
/* ------------------------------------------------------------------------ */

/* Full epsilon table for S[0..m] (complex interleaved).  Returns 0, or
 * ORC_EBREAKDOWN when a difference in the table is exactly zero. */
int orc_wynn(int m1, const double *S, double *est) {
  if (m1 < 1) return ORC_EINVAL;
  zdouble *block = calloc(3 * ((size_t)m1 + 1), sizeof(zdouble));
  if (!block) return ORC_ENOMEM;
  zdouble *prev = block, *cur = block + (m1 + 1), *nxt = block + 2 * (m1 + 1);
  int len = m1, k = 0, st = ORC_OK;
  for (int n = 0; n < m1; ++n) cur[n] = S[2 * n] + I * S[2 * n + 1];
  zdouble best = cur[m1 - 1];
  while (len > 1) {
    for (int n = 0; n + 1 < len; ++n) {
      zdouble d = cur[n + 1] - cur[n];
      if (d == 0.0) { st = ORC_EBREAKDOWN; break; }
      nxt[n] = prev[n + 1] + 1.0 / d;
    }
    if (st != ORC_OK) break;
    zdouble *t = prev; prev = cur; cur = nxt; nxt = t;
    --len;
    ++k;
    if ((k & 1) == 0) best = cur[len - 1];
  }
  est[0] = creal(best);
  est[1] = cimag(best);
  free(block);
  return st;
}

/* The paper's solve: u0 = O P0 Vt e0 (Born term), iterate x_{n+1} = K x_n,
 * record c_n = x_n[r0], and sum by Wynn-epsilon.  Stops when two successive
 * estimates agree to rel tol (after min_iter terms).  Otherwise, after
 * max_iter terms, returns ORC_ENOCONV with the estimate that changed least
 * from its predecessor (the partial sums grow like rho(K)^n when K has
 * eigenvalues outside the unit circle, so later estimates lose digits).
 * c_out (optional) receives the c_n. */
int orc_solve_wynn(int n_ch, int N, int M, const double *O, const double *Vt,
                   const int64_t *row_ptr, const int32_t *col, const double *val, const double *g,
                   int r0, int min_iter, int max_iter, double tol, double *U00, int *n_terms,
                   double *c_out) {
  size_t n = (size_t)n_ch * N * M;
  double *x = calloc(2 * n, sizeof(double)), *y = malloc(sizeof(double) * 2 * n);
  double *S = malloc(sizeof(double) * 2 * (size_t)(max_iter + 1));
  double *e0 = calloc(2 * n, sizeof(double));
  if (!x || !y || !S || !e0) { free(x); free(y); free(S); free(e0); return ORC_ENOMEM; }
  e0[2 * (size_t)r0] = 1.0;
  orc_kapply(n_ch, N, M, O, Vt, row_ptr, col, val, NULL, e0, x);
  free(e0);
  zdouble sum = 0.0, last = 0.0, best = 0.0;
  double best_d = INFINITY;
  int best_m = 0, st = ORC_ENOCONV, m, used = 0;
  for (m = 0; m < max_iter; ++m) {
    zdouble cn = x[2 * (size_t)r0] + I * x[2 * (size_t)r0 + 1];
    if (c_out) { c_out[2 * m] = creal(cn); c_out[2 * m + 1] = cimag(cn); }
    sum += cn;
    S[2 * m] = creal(sum);
    S[2 * m + 1] = cimag(sum);
    double est[2];
    int ws = orc_wynn(m + 1, S, est);
    zdouble e = est[0] + I * est[1];
    used = m + 1;
    if (ws == ORC_EBREAKDOWN) { /* keep the best estimate seen so far */
      st = ORC_EBREAKDOWN;
      if (best_m == 0) best = e;
      used = best_m > 0 ? best_m : used;
      break;
    }
    if (m > 0) {
      double d = cabs(e - last) / cabs(e);
      if (m + 1 >= min_iter && d <= tol) { st = ORC_OK; best = e; break; }
      if (d < best_d) { best_d = d; best = e; best_m = m + 1; }
    }
    last = e;
    if (m + 1 < max_iter) {
      orc_kapply(n_ch, N, M, O, Vt, row_ptr, col, val, g, x, y);
      double *t = x; x = y; y = t;
    }
  }
  if (st == ORC_ENOCONV && best_m == 0) best = last;
  U00[0] = creal(best);
  U00[1] = cimag(best);
  *n_terms = (st == ORC_ENOCONV && best_m > 0) ? best_m : used;

  free(x); free(y); free(S);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Vector form of the summation: the minimal-residual (reduced-rank)         */
/* extrapolation of the iterates of u = b + K u, computed through an         */
/* orthonormal Krylov basis (modified Gram-Schmidt Arnoldi, i.e. GMRES on    */
/* (I - K) u = b).  Used for residual-targeted solves.  u holds the initial  */
/* guess on entry (warm start) and the solution on exit.  Returns the number */
/* of K applications in *n_kapply and the final true relative residual.     */
/* ------------------------------------------------------------------------ */
static double znorm(size_t n, const zdouble *v) {
  double s = 0.0;
  for (size_t i = 0; i < n; ++i) s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
  return sqrt(s);
}

static void kapply_z(int n_ch, int N, int M, const double *O, const double *Vt,
                     const int64_t *row_ptr, const int32_t *col, const double *val, const double *g,
                     const zdouble *in, zdouble *out) {
  /* zdouble is layout-compatible with interleaved (re, im) doubles */
  orc_kapply(n_ch, N, M, O, Vt, row_ptr, col, val, g, (const double *)in, (double *)out);
}

int orc_solve_gmres(int n_ch, int N, int M, const double *O, const double *Vt,
                    const int64_t *row_ptr, const int32_t *col, const double *val, const double *g,
                    const double *b_in, double *u_io, int max_iter, double tol, int *n_kapply,
                    double *relres) {
  size_t n = (size_t)n_ch * N * M;
  int m = max_iter;
  zdouble *V = malloc(sizeof(zdouble) * n * (size_t)(m + 1));
  zdouble *H = calloc((size_t)(m + 1) * m, sizeof(zdouble));
  zdouble *w = malloc(sizeof(zdouble) * n), *r = malloc(sizeof(zdouble) * n);
  zdouble *cs = malloc(sizeof(zdouble) * m), *sn = malloc(sizeof(zdouble) * m);
  zdouble *bet = calloc((size_t)m + 1, sizeof(zdouble)), *yv = malloc(sizeof(zdouble) * m);
  if (!V || !H || !w || !r || !cs || !sn || !bet || !yv) {
    free(V); free(H); free(w); free(r); free(cs); free(sn); free(bet); free(yv);
    return ORC_ENOMEM;
  }
  const zdouble *b = (const zdouble *)b_in;
  zdouble *u = (zdouble *)u_io;
  int nk = 0;
  /* r = b - (I - K) u = b - u + K u */
  kapply_z(n_ch, N, M, O, Vt, row_ptr, col, val, g, u, w);
  ++nk;
  for (size_t i = 0; i < n; ++i) r[i] = b[i] - u[i] + w[i];
  double bn = znorm(n, b), rn = znorm(n, r);
  if (bn == 0.0) bn = 1.0;
  int k = 0, st = ORC_ENOCONV;
  if (rn <= tol * bn) { st = ORC_OK; goto done; }
  for (size_t i = 0; i < n; ++i) V[i] = r[i] / rn;
  bet[0] = rn;
  for (k = 0; k < m; ++k) {
    zdouble *vk = V + n * (size_t)k, *vn = V + n * (size_t)(k + 1);
    kapply_z(n_ch, N, M, O, Vt, row_ptr, col, val, g, vk, w);
    ++nk;
    for (size_t i = 0; i < n; ++i) w[i] = vk[i] - w[i];
    for (int jj = 0; jj <= k; ++jj) {
      zdouble *vj = V + n * (size_t)jj, h = 0.0;
      for (size_t i = 0; i < n; ++i) h += conj(vj[i]) * w[i];
      for (size_t i = 0; i < n; ++i) w[i] -= h * vj[i];
      H[(size_t)jj * m + k] = h;
    }
    double hn = znorm(n, w);
    H[(size_t)(k + 1) * m + k] = hn;
    if (hn > 0.0)
      for (size_t i = 0; i < n; ++i) vn[i] = w[i] / hn;
    /* Givens rotations on column k */
    for (int jj = 0; jj < k; ++jj) {
      zdouble h0 = H[(size_t)jj * m + k], h1 = H[(size_t)(jj + 1) * m + k];
      H[(size_t)jj * m + k] = conj(cs[jj]) * h0 + conj(sn[jj]) * h1;
      H[(size_t)(jj + 1) * m + k] = -sn[jj] * h0 + cs[jj] * h1;
    }
    zdouble h0 = H[(size_t)k * m + k], h1 = H[(size_t)(k + 1) * m + k];
    double den = sqrt(creal(h0 * conj(h0)) + creal(h1 * conj(h1)));
    if (den == 0.0) { st = ORC_EBREAKDOWN; ++k; break; }
    cs[k] = h0 / den;
    sn[k] = h1 / den;
    H[(size_t)k * m + k] = den;
    H[(size_t)(k + 1) * m + k] = 0.0;
    bet[k + 1] = -sn[k] * bet[k];
    bet[k] = conj(cs[k]) * bet[k];
    if (cabs(bet[k + 1]) <= tol * bn || hn == 0.0) { st = ORC_OK; ++k; break; }
  }
  if (k > m) k = m;
  /* back substitution, u += V y */
  for (int i = k - 1; i >= 0; --i) {
    zdouble s = bet[i];
    for (int jj = i + 1; jj < k; ++jj) s -= H[(size_t)i * m + jj] * yv[jj];
    yv[i] = s / H[(size_t)i * m + i];
  }
  for (int jj = 0; jj < k; ++jj) {
    zdouble *vj = V + n * (size_t)jj;
    for (size_t i = 0; i < n; ++i) u[i] += yv[jj] * vj[i];
  }
done:
  /* true residual */
  kapply_z(n_ch, N, M, O, Vt, row_ptr, col, val, g, u, w);
  ++nk;
  for (size_t i = 0; i < n; ++i) r[i] = b[i] - u[i] + w[i];
  *relres = znorm(n, r) / bn;
  *n_kapply = nk;
  free(V); free(H); free(w); free(r); free(cs); free(sn); free(bet); free(yv);
  return st;
}
