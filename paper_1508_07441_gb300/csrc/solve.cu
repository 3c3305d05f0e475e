// Steps 3 and 4 of the numerical scheme (Sec. 3.3): the channel resolvent
// G1 and the iterative solution of the matrix Faddeev equation (Eq. m_pvg)
// with the factorised kernel K = O P0 Vt G1 (Eq. kernel).
//
// One K application (FP64):
//   gemm_kernel<VT>  Y[ch] = Vt[ch] (G1 o X)[ch]   (G1 fused into the B load)
//   spmv_kernel      Z[l][c] = sum_{c', l'} P0[(l,c),(l',c')] Y[l'][c']
//   gemm_kernel<O>   X'[ch] = O[ch] Z[ch]          (optional epilogue V - .)
// Complex vectors are interleaved, so an [N][M] complex block is an
// [N][2M] real matrix and the (real) block matrices multiply it directly.
//
// Summation of the iterates:
//   KRYLOV  the vector form: Arnoldi with two-pass classical Gram-Schmidt on
//           the iterates of (I - K), the least-squares problem updated by
//           Givens rotations on the device; equivalent to the
//           minimal-residual (reduced-rank) extrapolation of the iterates.
//   WYNN    the paper's scalar route: c_n = e0^T K^n u0 collected on the
//           device and summed by Wynn's epsilon algorithm (device kernel).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "wpcd_internal.h"

namespace wpcd {
namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// ---------------------------------------------------------------------------
// resolvent
// ---------------------------------------------------------------------------
__device__ double f_lin(double q, double s, double sg) {
  // antiderivative of q^2 ln|q + sg s|; (q^3 + sg s^3) ln|.| -> 0 at q = -sg s
  double d = q + sg * s;
  double cube = d * (q * q - sg * q * s + s * s);  // q^3 + sg s^3
  double lg = d == 0.0 ? 0.0 : cube * log(fabs(d)) / 3.0;
  return lg - q * q * q / 9.0 + sg * s * q * q / 6.0 - s * s * q / 3.0;
}

// int_{qa}^{qb} q^2 ln|a - 3q^2/4| dq without the ln(3/4) B term (it cancels
// in the difference taken by the caller)
__device__ double phi_noconst(double qa, double qb, double a) {
  if (a > 0.0) {
    double s = sqrt(a / 0.75);
    return f_lin(qb, s, 1.0) + f_lin(qb, s, -1.0) - f_lin(qa, s, 1.0) - f_lin(qa, s, -1.0);
  }
  if (a < 0.0) {
    double t = sqrt(-a / 0.75);
    auto F = [&](double q) {
      return q * q * q / 3.0 * log(q * q + t * t) -
             (2.0 / 3.0) * (q * q * q / 3.0 - t * t * q + t * t * t * atan(q / t));
    };
    return F(qb) - F(qa);
  }
  auto F0 = [&](double q) { return q > 0.0 ? (2.0 / 3.0) * q * q * q * (log(q) - 1.0 / 3.0) : 0.0; };
  return F0(qb) - F0(qa);
}

struct ResParams {
  int n_ch, N, M, n_E;
  const double *qe, *eps;
  const double *Elo, *Ehi;  // per energy
  const double *gl_t, *gl_w; // 32-point GL rule
};

__global__ void resolvent_kernel(ResParams R, double *g) {
  const int dim = R.n_ch * R.N * R.M;
  const int64_t total = (int64_t)R.n_E * dim;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int e = (int)(idx / dim);
    int r = (int)(idx % dim);
    int j = r % R.M;
    int chk = r / R.M;  // ch*N + k
    double ek = R.eps[chk];
    double Elo = R.Elo[e], Ehi = R.Ehi[e], D = Ehi - Elo;
    double qa = R.qe[j], qb = R.qe[j + 1];
    double Bq = (qb - qa) * (qb * qb + qb * qa + qa * qa) / 3.0;
    double lo_a = Elo - ek - 0.75 * qa * qa, lo_b = Elo - ek - 0.75 * qb * qb;
    double hi_a = Ehi - ek - 0.75 * qa * qa, hi_b = Ehi - ek - 0.75 * qb * qb;
    bool no_sign_change = (lo_a > 0.0 && lo_b > 0.0 && hi_a > 0.0 && hi_b > 0.0) ||
                          (lo_a < 0.0 && lo_b < 0.0 && hi_a < 0.0 && hi_b < 0.0);
    double dist = fmin(fabs(lo_a), fabs(lo_b));
    double re;
    if (no_sign_change && fabs(D) < 0.05 * dist) {
      // smooth integrand: q^2 log(1 + D / (E_lo - eps - 3q^2/4)) by 32-point GL
      double half = 0.5 * (qb - qa), mid = 0.5 * (qb + qa), s = 0.0;
      for (int m = 0; m < 32; ++m) {
        double q = mid + half * R.gl_t[m];
        s += R.gl_w[m] * q * q * log1p(D / (Elo - ek - 0.75 * q * q));
      }
      re = half * s;
    } else {
      re = phi_noconst(qa, qb, Ehi - ek) - phi_noconst(qa, qb, Elo - ek);
    }
    re /= D * Bq;
    double im = 0.0;
    if (Ehi - ek > 0.0) {
      double lo = sqrt(fmax((Elo - ek) / 0.75, 0.0)), hi = sqrt((Ehi - ek) / 0.75);
      double a = fmax(qa, lo), b = fmin(qb, hi);
      if (b > a) im = -kPi * ((b - a) * (b * b + b * a + a * a) / 3.0) / (D * Bq);
    }
    g[2 * idx] = re;
    g[2 * idx + 1] = im;
  }
}

// ---------------------------------------------------------------------------
// dense block GEMM (FP64):  C[b] (n x ncol) = A[b] (n x n) * B'[b] (n x ncol)
// B' = B, or the G1-scaled complex block (ncol = 2M, complex pairs)
// epilogue: C = out, or C = S - out
// ---------------------------------------------------------------------------
// 32 x 64 output tiles: 7 x 7 x 3 = 147 CTAs for the 200-bin, 3-channel
// blocks, close to one wave over the 152 SMs (FP64 work is issue-bound, so
// SM coverage matters more than data reuse here)
constexpr int GB_M = 32, GB_N = 64, GB_K = 16, G_THREADS = 256;

template <bool SCALE_G, bool SUB>
__global__ void __launch_bounds__(G_THREADS) gemm_kernel(int n, int ncol, const double *__restrict__ A,
                                                         const double *__restrict__ B,
                                                         const double *__restrict__ G,
                                                         const double *__restrict__ S,
                                                         double *__restrict__ C) {
  __shared__ double As[GB_K][GB_M + 1];
  __shared__ double Bs[GB_K][GB_N];
  const int b = blockIdx.z;
  const size_t offA = (size_t)b * n * n, offB = (size_t)b * n * ncol;
  const int row0 = blockIdx.y * GB_M, col0 = blockIdx.x * GB_N;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 2 x 4 outputs each
  double acc[2][4] = {};
  for (int k0 = 0; k0 < n; k0 += GB_K) {
    for (int t = threadIdx.x; t < GB_M * GB_K; t += G_THREADS) {
      int r = t / GB_K, kk = t % GB_K;
      int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < n && gk < n) ? A[offA + (size_t)gr * n + gk] : 0.0;
    }
    for (int t = threadIdx.x; t < GB_K * GB_N; t += G_THREADS) {
      int kk = t / GB_N, cc = t % GB_N;
      int gk = k0 + kk, gc = col0 + cc;
      double v = 0.0;
      if (gk < n && gc < ncol) {
        size_t o = offB + (size_t)gk * ncol + gc;
        if (SCALE_G) {
          size_t oc = o & ~(size_t)1;  // complex pair (re at even column)
          double xr = B[oc], xi = B[oc + 1], gr_ = G[oc], gi = G[oc + 1];
          v = (gc & 1) ? (gr_ * xi + gi * xr) : (gr_ * xr - gi * xi);
        } else {
          v = B[o];
        }
      }
      Bs[kk][cc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      double a[2], bb[4];
#pragma unroll
      for (int u = 0; u < 2; ++u) a[u] = As[kk][ty + 16 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u) bb[u] = Bs[kk][tx + 16 * u];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], bb[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int gr = row0 + ty + 16 * u, gc = col0 + tx + 16 * v;
      if (gr < n && gc < ncol) {
        size_t o = offB + (size_t)gr * ncol + gc;
        C[o] = SUB ? S[o] - acc[u][v] : acc[u][v];
      }
    }
}

// ---------------------------------------------------------------------------
// block-CSR SpMV on complex vectors: Z[l][c] = sum P0 Y
// LPR lanes per row; values pair-major (val[m][nnz]), real = double / float
// ---------------------------------------------------------------------------
struct SpmvParams {
  int n_cells, n_ch, n_pairs;
  int pl[kMaxPairs], plp[kMaxPairs];
  const int64_t *row_ptr;
  const int32_t *col;
  int64_t nnz;
};

template <typename real, int NCH, int LPR>
__global__ void __launch_bounds__(256) spmv_kernel(SpmvParams S, const real *__restrict__ val,
                                                   const double2 *__restrict__ y, double2 *__restrict__ z) {
  constexpr int NPAIR = pair_count(NCH);
  constexpr int GPW = 32 / LPR;  // row groups per warp
  const int lane = threadIdx.x % LPR;
  const int gw = threadIdx.x / LPR % GPW;
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int n_warps = gridDim.x * blockDim.x / 32;
  // the loop bound depends on the warp only, so every lane reaches the
  // full-mask shuffles below
  for (int base = warp_global * GPW; base < S.n_cells; base += n_warps * GPW) {
    const int c = base + gw;
    const bool active = c < S.n_cells;
    double2 acc[NCH];
#pragma unroll
    for (int l = 0; l < NCH; ++l) acc[l] = make_double2(0.0, 0.0);
    const int64_t b = active ? S.row_ptr[c] : 0, e = active ? S.row_ptr[c + 1] : 0;
    for (int64_t o = b + lane; o < e; o += LPR) {
      const int t = __ldg(S.col + o);
      double2 yv[NCH];
#pragma unroll
      for (int l = 0; l < NCH; ++l) yv[l] = __ldg(y + (size_t)l * S.n_cells + t);
#pragma unroll
      for (int m = 0; m < NPAIR; ++m) {
        const int l = pair_first(NCH, m), lp = pair_second(NCH, m);
        double v = (double)__ldg(val + (size_t)m * S.nnz + o);
        acc[l].x = fma(v, yv[lp].x, acc[l].x);
        acc[l].y = fma(v, yv[lp].y, acc[l].y);
      }
    }
#pragma unroll
    for (int off = LPR / 2; off > 0; off >>= 1)
#pragma unroll
      for (int l = 0; l < NCH; ++l) {
        acc[l].x += __shfl_xor_sync(0xffffffffu, acc[l].x, off, LPR);
        acc[l].y += __shfl_xor_sync(0xffffffffu, acc[l].y, off, LPR);
      }
    if (active && lane == 0)
#pragma unroll
      for (int l = 0; l < NCH; ++l) z[(size_t)l * S.n_cells + c] = acc[l];
  }
}

// ---------------------------------------------------------------------------
// vector kernels for the Krylov basis (complex, interleaved)
// ---------------------------------------------------------------------------
constexpr int V_THREADS = 256;

// partial[j][blk] = sum_{i in blk} conj(V_j[i]) w[i], j < nv
__global__ void __launch_bounds__(V_THREADS) multi_dot_kernel(int n, int nv, const double2 *__restrict__ V,
                                                              size_t ld, const double2 *__restrict__ w,
                                                              double2 *__restrict__ partial) {
  __shared__ double2 red[V_THREADS / 32];
  const int nblk = gridDim.x;
  for (int j = 0; j < nv; ++j) {
    double2 s = make_double2(0.0, 0.0);
    for (int i = blockIdx.x * V_THREADS + threadIdx.x; i < n; i += nblk * V_THREADS) {
      double2 a = V[(size_t)j * ld + i], b = w[i];
      s.x += a.x * b.x + a.y * b.y;
      s.y += a.x * b.y - a.y * b.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      s.x += __shfl_down_sync(0xffffffffu, s.x, o);
      s.y += __shfl_down_sync(0xffffffffu, s.y, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double2 t = make_double2(0.0, 0.0);
      for (int k = 0; k < V_THREADS / 32; ++k) { t.x += red[k].x; t.y += red[k].y; }
      partial[(size_t)j * nblk + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// out[j] (+)= sum_blk partial[j][blk]   (accumulate: add to out)
__global__ void reduce_partials_kernel(int nv, int nblk, const double2 *partial, double2 *out, int accumulate) {
  int j = blockIdx.x;
  __shared__ double2 red[256];
  double2 s = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    s.x += partial[(size_t)j * nblk + b].x;
    s.y += partial[(size_t)j * nblk + b].y;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) { red[threadIdx.x].x += red[threadIdx.x + o].x; red[threadIdx.x].y += red[threadIdx.x + o].y; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (accumulate) { out[j].x += red[0].x; out[j].y += red[0].y; }
    else out[j] = red[0];
  }
}

// w[i] -= sum_j h[j] V_j[i]  (sign = -1) or w[i] += ... (sign = +1)
__global__ void multi_axpy_kernel(int n, int nv, const double2 *__restrict__ V, size_t ld,
                                  const double2 *__restrict__ h, double2 *__restrict__ w, double sign) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double2 acc = w[i];
    for (int j = 0; j < nv; ++j) {
      double2 a = V[(size_t)j * ld + i], c = h[j];
      acc.x += sign * (c.x * a.x - c.y * a.y);
      acc.y += sign * (c.x * a.y + c.y * a.x);
    }
    w[i] = acc;
  }
}

// dst = src * (1 / |nrm|)  where nrm is a device scalar (real part used)
__global__ void scale_kernel(int n, const double2 *src, const double2 *nrm2, double2 *dst) {
  double s = nrm2->x > 0.0 ? 1.0 / sqrt(nrm2->x) : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double2 a = src[i];
    dst[i] = make_double2(a.x * s, a.y * s);
  }
}

// Krylov state on the device
struct KrylovState {
  int m;          // capacity (columns)
  int k;          // columns done
  int status;
  double bnorm;
  double relres;
  double2 H[1];   // [(m+1) * m] column-major Hessenberg, then cs, sn, bet, y
};

// one Givens/least-squares update for column k; h[0..k] holds the Gram-Schmidt
// coefficients (accumulated over both passes), hn2 the squared norm of the
// new vector (real part)
__global__ void givens_kernel(int m, int k, const double2 *h, const double2 *hn2, double2 *H,
                              double2 *cs, double2 *sn, double2 *bet, double *resid, double bnorm) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double2 *col = H + (size_t)k * (m + 1);
  for (int i = 0; i <= k; ++i) col[i] = h[i];
  // H stores -h for the (I - K) operator convention handled by the caller
  double hn = sqrt(fmax(hn2->x, 0.0));
  col[k + 1] = make_double2(hn, 0.0);
  for (int i = 0; i < k; ++i) {
    double2 a = col[i], b = col[i + 1], c = cs[i], s = sn[i];
    // [a'; b'] = [conj(c) conj(s); -s c] [a; b]
    double2 na = make_double2(c.x * a.x + c.y * a.y + s.x * b.x + s.y * b.y,
                              c.x * a.y - c.y * a.x + s.x * b.y - s.y * b.x);
    double2 nb = make_double2(-(s.x * a.x - s.y * a.y) + (c.x * b.x - c.y * b.y),
                              -(s.x * a.y + s.y * a.x) + (c.x * b.y + c.y * b.x));
    col[i] = na;
    col[i + 1] = nb;
  }
  double2 a = col[k], b = col[k + 1];
  double den = sqrt(a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y);
  double2 c = den > 0 ? make_double2(a.x / den, a.y / den) : make_double2(1.0, 0.0);
  double2 s = den > 0 ? make_double2(b.x / den, b.y / den) : make_double2(0.0, 0.0);
  cs[k] = c;
  sn[k] = s;
  col[k] = make_double2(den, 0.0);
  col[k + 1] = make_double2(0.0, 0.0);
  double2 bk = bet[k];
  bet[k + 1] = make_double2(-(s.x * bk.x - s.y * bk.y), -(s.x * bk.y + s.y * bk.x));
  bet[k] = make_double2(c.x * bk.x + c.y * bk.y, c.x * bk.y - c.y * bk.x);
  *resid = sqrt(bet[k + 1].x * bet[k + 1].x + bet[k + 1].y * bet[k + 1].y) / bnorm;
}

// back substitution H y = bet (k x k upper triangular)
__global__ void backsub_kernel(int m, int k, const double2 *H, const double2 *bet, double2 *y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double2 s = bet[i];
    for (int j = i + 1; j < k; ++j) {
      double2 h = H[(size_t)j * (m + 1) + i], yj = y[j];
      s.x -= h.x * yj.x - h.y * yj.y;
      s.y -= h.x * yj.y + h.y * yj.x;
    }
    double2 d = H[(size_t)i * (m + 1) + i];
    double dd = d.x * d.x + d.y * d.y;
    y[i] = make_double2((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd);
  }
}

// amplitude from the on-shell element: S = 1 - 2 pi i U00 / D, paper's A
__global__ void amplitude_kernel(const double2 *u, int r0, double D, double pref, double *out) {
  double2 U = u[r0];
  out[0] = U.x;
  out[1] = U.y;
  out[2] = 1.0 + 2.0 * kPi * U.y / D;   // Re S
  out[3] = -2.0 * kPi * U.x / D;        // Im S
  out[4] = pref * U.x;
  out[5] = pref * U.y;
}

// Wynn epsilon over the partial sums of c[0..n-1] (complex); writes the
// deepest even-column estimate into est[n-1] and the breakdown flag
__global__ void wynn_kernel(int n, const double2 *c, double2 *work, double2 *est, int *breakdown) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double2 *prev = work, *cur = work + n + 1, *nxt = work + 2 * (n + 1);
  double2 s = make_double2(0.0, 0.0);
  for (int i = 0; i < n; ++i) {
    s.x += c[i].x;
    s.y += c[i].y;
    cur[i] = s;
    prev[i] = make_double2(0.0, 0.0);
  }
  prev[n] = make_double2(0.0, 0.0);
  double2 best = cur[n - 1];
  int len = n, col = 0, bd = 0;
  while (len > 1) {
    for (int i = 0; i + 1 < len; ++i) {
      double dx = cur[i + 1].x - cur[i].x, dy = cur[i + 1].y - cur[i].y;
      double d2 = dx * dx + dy * dy;
      if (d2 == 0.0) { bd = 1; break; }
      nxt[i] = make_double2(prev[i + 1].x + dx / d2, prev[i + 1].y - dy / d2);
    }
    if (bd) break;
    double2 *t = prev;
    prev = cur;
    cur = nxt;
    nxt = t;
    --len;
    ++col;
    if ((col & 1) == 0) best = cur[len - 1];
  }
  est[n - 1] = best;
  *breakdown = bd;
}

__global__ void extract_kernel(const double2 *x, int r0, double2 *c_out) { *c_out = x[r0]; }

__global__ void set_unit_kernel(int n, int r0, double2 *x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] = make_double2(i == r0 ? 1.0 : 0.0, 0.0);
}

int grid_for(int64_t n, int threads, int cap = 152 * 8) {
  int64_t g = (n + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// ---------------------------------------------------------------------------
// K application machinery
// ---------------------------------------------------------------------------
struct Workspace {
  double *y = nullptr, *z = nullptr;  // [dim] complex
  ~Workspace() {
    cudaFree(y);
    cudaFree(z);
  }
};

wpcd_status launch_spmv(const wpcd_problem *pr, const wpcd_P *P, const double *y, double *z, cudaStream_t s) {
  SpmvParams S{};
  S.n_cells = pr->N * pr->M;
  S.n_ch = pr->n_ch;
  S.n_pairs = pr->n_pairs;
  for (int m = 0; m < pr->n_pairs; ++m) {
    S.pl[m] = pr->pair_l[m];
    S.plp[m] = pr->pair_lp[m];
  }
  S.row_ptr = P->row_ptr;
  S.col = P->col;
  S.nnz = P->nnz;
  const double2 *yy = reinterpret_cast<const double2 *>(y);
  double2 *zz = reinterpret_cast<double2 *>(z);
  constexpr int LPR = 16;
  int grid = grid_for((int64_t)S.n_cells, 256 / LPR, 152 * 16);  // blocks of 256 threads
  bool f64 = P->prec == WPCD_FP64;
#define WPCD_SPMV_CASE(NCH, NPAIR)                                                                 \
  if (pr->n_ch == NCH) {                                                                           \
    if (f64)                                                                                       \
      spmv_kernel<double, NCH, LPR><<<grid, 256, 0, s>>>(S, P->val64, yy, zz);                     \
    else                                                                                           \
      spmv_kernel<float, NCH, LPR><<<grid, 256, 0, s>>>(S, P->val32, yy, zz);                      \
    count_launches(1);                                                                             \
    return cudaGetLastError() == cudaSuccess ? WPCD_OK : set_error(WPCD_ECUDA, "spmv launch");    \
  }
  WPCD_SPMV_CASE(1, 1)
  WPCD_SPMV_CASE(2, 2)
  WPCD_SPMV_CASE(3, 5)
  WPCD_SPMV_CASE(4, 8)
  WPCD_SPMV_CASE(5, 13)
#undef WPCD_SPMV_CASE
  return set_error(WPCD_EINVAL, "unsupported channel count for the SpMV");
}

// y = O P0 Vt (g o x)   or, with sub, y = sub - O P0 Vt (g o x)
wpcd_status kapply_ws(const wpcd_problem *pr, const wpcd_P *P, const double *g, const double *x,
                      double *out, const double *sub, Workspace &ws, cudaStream_t s) {
  const int N = pr->N, M = pr->M, n_ch = pr->n_ch;
  const int ncol = 2 * M;
  dim3 grid((ncol + GB_N - 1) / GB_N, (N + GB_M - 1) / GB_M, n_ch);
  if (g)
    gemm_kernel<true, false><<<grid, G_THREADS, 0, s>>>(N, ncol, pr->d.Vt, x, g, nullptr, ws.y);
  else
    gemm_kernel<false, false><<<grid, G_THREADS, 0, s>>>(N, ncol, pr->d.Vt, x, nullptr, nullptr, ws.y);
  count_launches(1);
  wpcd_status st = launch_spmv(pr, P, ws.y, ws.z, s);
  if (st != WPCD_OK) return st;
  if (sub)
    gemm_kernel<false, true><<<grid, G_THREADS, 0, s>>>(N, ncol, pr->d.O, ws.z, nullptr, sub, out);
  else
    gemm_kernel<false, false><<<grid, G_THREADS, 0, s>>>(N, ncol, pr->d.O, ws.z, nullptr, nullptr, out);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "kapply launch");
}

}  // namespace

// ---------------------------------------------------------------------------
// host entry points
// ---------------------------------------------------------------------------
wpcd_status onshell(const wpcd_problem *pr, double E, int *j0, double *Elo, double *Ehi, double *q0) {
  if (!std::isfinite(E)) return set_error(WPCD_EINVAL, "energy is not finite");
  if (!(E > pr->eps_b)) return set_error(WPCD_ENOBOUND, "energy at or below the dimer threshold");
  double q = std::sqrt((E - pr->eps_b) / 0.75);
  const std::vector<double> &qe = pr->qe;
  if (!(q < qe[pr->M])) return set_error(WPCD_EINVAL, "on-shell momentum beyond the q grid");
  // bin containing q: largest j with qe[j] <= q
  int lo = 0, hi = pr->M - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (qe[mid] <= q) lo = mid; else hi = mid - 1;
  }
  *j0 = lo;
  *Elo = pr->eps_b + 0.75 * qe[lo] * qe[lo];
  *Ehi = pr->eps_b + 0.75 * qe[lo + 1] * qe[lo + 1];
  if (q0) *q0 = q;
  return WPCD_OK;
}

wpcd_status resolvent(const wpcd_problem *pr, const double *E, int n_E, double *g, int *j0,
                      double *D, cudaStream_t s) {
  if (n_E < 0 || (n_E > 0 && (!E || !g))) return set_error(WPCD_EINVAL, "bad resolvent arguments");
  if (n_E == 0) return WPCD_OK;
  std::vector<double> lohi(2 * (size_t)n_E + 64);
  for (int e = 0; e < n_E; ++e) {
    int jj;
    double lo, hi;
    wpcd_status st = onshell(pr, E[e], &jj, &lo, &hi, nullptr);
    if (st != WPCD_OK) return st;
    lohi[e] = lo;
    lohi[n_E + e] = hi;
    if (j0) j0[e] = jj;
    if (D) D[e] = hi - lo;
  }
  gauss_legendre(32, lohi.data() + 2 * n_E, lohi.data() + 2 * n_E + 32);
  WPCD_CUDA_TRY(cudaSetDevice(pr->device));
  double *d_lohi = nullptr;
  WPCD_CUDA_TRY(cudaMallocAsync(&d_lohi, sizeof(double) * lohi.size(), s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(d_lohi, lohi.data(), sizeof(double) * lohi.size(), cudaMemcpyHostToDevice, s));
  ResParams R{};
  R.n_ch = pr->n_ch;
  R.N = pr->N;
  R.M = pr->M;
  R.n_E = n_E;
  R.qe = pr->d.qe;
  R.eps = pr->d.eps;
  R.Elo = d_lohi;
  R.Ehi = d_lohi + n_E;
  R.gl_t = d_lohi + 2 * n_E;
  R.gl_w = d_lohi + 2 * n_E + 32;
  int64_t total = (int64_t)n_E * pr->n_ch * pr->N * pr->M;
  resolvent_kernel<<<grid_for(total, 256, 152 * 16), 256, 0, s>>>(R, g); count_launches(1);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(d_lohi, s);
  // the host staging buffer must outlive the copy
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "resolvent launch");
  if (e2 != cudaSuccess) return cuda_error(e2, "resolvent");
  return WPCD_OK;
}

wpcd_status kapply(const wpcd_problem *pr, const wpcd_P *P, const double *g, const double *x,
                   double *y, cudaStream_t s) {
  WPCD_CUDA_TRY(cudaSetDevice(pr->device));
  const size_t dim = (size_t)pr->n_ch * pr->N * pr->M;
  Workspace ws;
  WPCD_CUDA_TRY(cudaMalloc(&ws.y, 16 * dim));
  WPCD_CUDA_TRY(cudaMalloc(&ws.z, 16 * dim));
  wpcd_status st = kapply_ws(pr, P, g, x, y, nullptr, ws, s);
  if (st != WPCD_OK) return st;
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  return WPCD_OK;
}

namespace {

struct SolveBuffers {
  double *g = nullptr;       // [dim] complex
  double *V = nullptr;       // [(m+1)][dim] complex basis (or iterates)
  double *w = nullptr;       // [dim] complex
  double *u = nullptr;       // [dim] complex solution
  double2 *small = nullptr;  // Krylov scalars
  double2 *partial = nullptr;
  double *resid = nullptr;
  int *flag = nullptr;
  double *amp = nullptr;
  ~SolveBuffers() {
    cudaFree(g); cudaFree(V); cudaFree(w); cudaFree(u); cudaFree(small); cudaFree(partial);
    cudaFree(resid); cudaFree(flag); cudaFree(amp);
  }
};

// Krylov solve of (I - K) u = b with u0 = 0; b = Born term.  Returns U00 etc.
wpcd_status solve_krylov(const wpcd_problem *pr, const wpcd_P *P, double E, const wpcd_solve_opts &o,
                         SolveBuffers &B, Workspace &ws, wpcd_solve_stats &out, cudaStream_t s) {
  const int dim = pr->n_ch * pr->N * pr->M;
  const int m = o.max_iter;
  int j0;
  double Elo, Ehi, q0;
  wpcd_status st = onshell(pr, E, &j0, &Elo, &Ehi, &q0);
  if (st != WPCD_OK) return st;
  double D = Ehi - Elo;
  st = resolvent(pr, &E, 1, B.g, nullptr, nullptr, s);
  if (st != WPCD_OK) return st;
  const int r0 = j0;
  double2 *V = reinterpret_cast<double2 *>(B.V);
  double2 *w = reinterpret_cast<double2 *>(B.w);
  const size_t ld = (size_t)dim;
  double2 *H = B.small;                       // (m+1) * m
  double2 *cs = H + (size_t)(m + 1) * m;
  double2 *sn = cs + m;
  double2 *bet = sn + m;                      // m + 1
  double2 *h = bet + (m + 1);                 // m + 1
  double2 *h2 = h + (m + 1);                  // m + 1
  double2 *nrm = h2 + (m + 1);                // 1
  double2 *yv = nrm + 1;                      // m
  const int nblk = 152 * 2;
  const int vgrid = grid_for(dim, 256, 152 * 8);
  cudaEvent_t e0, e1;
  WPCD_CUDA_TRY(cudaEventCreate(&e0));
  WPCD_CUDA_TRY(cudaEventCreate(&e1));
  cudaEventRecord(e0, s);
  // b = O P0 Vt e0  (into w), then v0 = b / |b|
  set_unit_kernel<<<vgrid, 256, 0, s>>>(dim, r0, reinterpret_cast<double2 *>(B.u)); count_launches(1);
  st = kapply_ws(pr, P, nullptr, B.u, B.w, nullptr, ws, s);
  if (st != WPCD_OK) return st;
  multi_dot_kernel<<<nblk, V_THREADS, 0, s>>>(dim, 1, w, ld, w, B.partial); count_launches(1);
  reduce_partials_kernel<<<1, 256, 0, s>>>(1, nblk, B.partial, nrm, 0); count_launches(1);
  scale_kernel<<<vgrid, 256, 0, s>>>(dim, w, nrm, V); count_launches(1);
  double2 nrm_h;
  WPCD_CUDA_TRY(cudaMemcpyAsync(&nrm_h, nrm, sizeof(double2), cudaMemcpyDeviceToHost, s));
  WPCD_CUDA_TRY(cudaMemsetAsync(B.small, 0, sizeof(double2) * ((size_t)(m + 1) * m + 5 * (m + 1) + 2), s));
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  double bnorm = std::sqrt(nrm_h.x);
  if (!(bnorm > 0.0)) return set_error(WPCD_EBREAKDOWN, "Born term is zero");
  double2 bet0 = make_double2(bnorm, 0.0);
  WPCD_CUDA_TRY(cudaMemcpyAsync(bet, &bet0, sizeof(double2), cudaMemcpyHostToDevice, s));
  int k = 0, status = WPCD_ENOCONV;
  double resid = 1.0;
  for (k = 0; k < m; ++k) {
    // w = (I - K) v_k = v_k - O P0 Vt G1 v_k
    st = kapply_ws(pr, P, B.g, reinterpret_cast<double *>(V + (size_t)k * ld), B.w,
                   reinterpret_cast<double *>(V + (size_t)k * ld), ws, s);
    if (st != WPCD_OK) return st;
    // two-pass classical Gram-Schmidt
    multi_dot_kernel<<<nblk, V_THREADS, 0, s>>>(dim, k + 1, V, ld, w, B.partial); count_launches(1);
    reduce_partials_kernel<<<k + 1, 256, 0, s>>>(k + 1, nblk, B.partial, h, 0); count_launches(1);
    multi_axpy_kernel<<<vgrid, 256, 0, s>>>(dim, k + 1, V, ld, h, w, -1.0); count_launches(1);
    multi_dot_kernel<<<nblk, V_THREADS, 0, s>>>(dim, k + 1, V, ld, w, B.partial); count_launches(1);
    reduce_partials_kernel<<<k + 1, 256, 0, s>>>(k + 1, nblk, B.partial, h2, 0); count_launches(1);
    multi_axpy_kernel<<<vgrid, 256, 0, s>>>(dim, k + 1, V, ld, h2, w, -1.0); count_launches(1);
    reduce_partials_kernel<<<k + 1, 256, 0, s>>>(k + 1, nblk, B.partial, h, 1);  // h += h2
    multi_dot_kernel<<<nblk, V_THREADS, 0, s>>>(dim, 1, w, ld, w, B.partial); count_launches(1);
    reduce_partials_kernel<<<1, 256, 0, s>>>(1, nblk, B.partial, nrm, 0); count_launches(1);
    scale_kernel<<<vgrid, 256, 0, s>>>(dim, w, nrm, V + (size_t)(k + 1) * ld); count_launches(1);
    givens_kernel<<<1, 1, 0, s>>>(m, k, h, nrm, H, cs, sn, bet, B.resid, bnorm); count_launches(1);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_error(ce, "krylov step launch");
    bool check = ((k + 1) % (o.check_every > 0 ? o.check_every : 1) == 0) || k + 1 == m;
    if (check) {
      WPCD_CUDA_TRY(cudaMemcpyAsync(&resid, B.resid, sizeof(double), cudaMemcpyDeviceToHost, s));
      WPCD_CUDA_TRY(cudaStreamSynchronize(s));
      if (!std::isfinite(resid)) { status = WPCD_EBREAKDOWN; ++k; break; }
      if (resid <= o.tol) { status = WPCD_OK; ++k; break; }
    }
  }
  if (k > m) k = m;
  // u = V y
  backsub_kernel<<<1, 1, 0, s>>>(m, k, H, bet, yv); count_launches(1);
  WPCD_CUDA_TRY(cudaMemsetAsync(B.u, 0, 16 * (size_t)dim, s));
  multi_axpy_kernel<<<vgrid, 256, 0, s>>>(dim, k, V, ld, yv, reinterpret_cast<double2 *>(B.u), 1.0); count_launches(1);
  double pref = 2.0 / (3.0 * q0) / (pr->qe[j0 + 1] - pr->qe[j0]);
  amplitude_kernel<<<1, 1, 0, s>>>(reinterpret_cast<double2 *>(B.u), r0, D, pref, B.amp); count_launches(1);
  cudaEventRecord(e1, s);
  double amp[6];
  WPCD_CUDA_TRY(cudaMemcpyAsync(amp, B.amp, sizeof(amp), cudaMemcpyDeviceToHost, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(&resid, B.resid, sizeof(double), cudaMemcpyDeviceToHost, s));
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  cudaEventElapsedTime(&out.ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  out.status = status;
  out.n_kapply = k + 1;  // including the Born term
  out.j0 = j0;
  out.D = D;
  out.relres = resid;
  for (int i = 0; i < 2; ++i) {
    out.U00[i] = amp[i];
    out.S[i] = amp[2 + i];
    out.A[i] = amp[4 + i];
  }
  return WPCD_OK;
}

// Paper's route: iterate x_{n+1} = K x_n from the Born term, collect
// c_n = x_n[r0], Wynn epsilon on the device.  Stops on two successive
// estimates within tol (relative), else returns the best (least changing)
// estimate with ENOCONV.
wpcd_status solve_wynn(const wpcd_problem *pr, const wpcd_P *P, double E, const wpcd_solve_opts &o,
                       SolveBuffers &B, Workspace &ws, wpcd_solve_stats &out, cudaStream_t s) {
  const int dim = pr->n_ch * pr->N * pr->M;
  const int m = o.max_iter;
  int j0;
  double Elo, Ehi, q0;
  wpcd_status st = onshell(pr, E, &j0, &Elo, &Ehi, &q0);
  if (st != WPCD_OK) return st;
  double D = Ehi - Elo;
  st = resolvent(pr, &E, 1, B.g, nullptr, nullptr, s);
  if (st != WPCD_OK) return st;
  const int r0 = j0;
  double2 *c = B.small;              // m
  double2 *est = c + m;              // m
  double2 *work = est + m;           // 3 (m + 1)
  double2 *x0 = reinterpret_cast<double2 *>(B.u), *x1 = reinterpret_cast<double2 *>(B.w);
  const int vgrid = grid_for(dim, 256, 152 * 8);
  cudaEvent_t e0, e1;
  WPCD_CUDA_TRY(cudaEventCreate(&e0));
  WPCD_CUDA_TRY(cudaEventCreate(&e1));
  cudaEventRecord(e0, s);
  set_unit_kernel<<<vgrid, 256, 0, s>>>(dim, r0, x1); count_launches(1);
  st = kapply_ws(pr, P, nullptr, B.w, B.u, nullptr, ws, s);  // x0 = Born
  if (st != WPCD_OK) return st;
  std::vector<double2> est_h(m);
  int n = 0, status = WPCD_ENOCONV, bd = 0, checked = 0, used = 0;
  double best_d = INFINITY;
  double2 best = make_double2(0.0, 0.0), last = make_double2(0.0, 0.0);
  int best_n = 0;
  const int every = o.check_every > 0 ? o.check_every : 1;
  for (n = 0; n < m; ++n) {
    extract_kernel<<<1, 1, 0, s>>>(x0, r0, c + n); count_launches(1);
    wynn_kernel<<<1, 1, 0, s>>>(n + 1, c, work, est, B.flag); count_launches(1);
    if (n + 1 < m) {
      st = kapply_ws(pr, P, B.g, reinterpret_cast<double *>(x0), reinterpret_cast<double *>(x1), nullptr, ws, s);
      if (st != WPCD_OK) return st;
      std::swap(x0, x1);
    }
    if ((n + 1) % every != 0 && n + 1 != m) continue;
    WPCD_CUDA_TRY(cudaMemcpyAsync(est_h.data(), est, sizeof(double2) * (n + 1), cudaMemcpyDeviceToHost, s));
    WPCD_CUDA_TRY(cudaMemcpyAsync(&bd, B.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    WPCD_CUDA_TRY(cudaStreamSynchronize(s));
    bool done = false;
    for (int t = checked; t <= n; ++t) {
      double2 e = est_h[t];
      used = t + 1;
      if (t > 0) {
        double2 p = est_h[t - 1];
        double d = std::hypot(e.x - p.x, e.y - p.y) / std::hypot(e.x, e.y);
        if (t + 1 >= o.min_iter && d <= o.tol) {
          best = e;
          status = WPCD_OK;
          done = true;
          break;
        }
        if (d < best_d) {
          best_d = d;
          best = e;
          best_n = t + 1;
        }
      }
      last = e;
    }
    checked = n + 1;
    if (done) break;
    if (bd) {
      status = WPCD_EBREAKDOWN;
      break;
    }
  }
  cudaEventRecord(e1, s);
  WPCD_CUDA_TRY(cudaEventSynchronize(e1));
  cudaEventElapsedTime(&out.ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != WPCD_OK && best_n == 0) best = last;
  out.status = status;
  out.n_kapply = (status == WPCD_OK) ? used : (best_n > 0 ? best_n : used);
  out.j0 = j0;
  out.D = D;
  out.relres = status == WPCD_OK ? 0.0 : best_d;
  out.U00[0] = best.x;
  out.U00[1] = best.y;
  out.S[0] = 1.0 + 2.0 * kPi * best.y / D;
  out.S[1] = -2.0 * kPi * best.x / D;
  double pref = 2.0 / (3.0 * q0) / (pr->qe[j0 + 1] - pr->qe[j0]);
  out.A[0] = pref * best.x;
  out.A[1] = pref * best.y;
  return WPCD_OK;
}

}  // namespace

wpcd_status solve(wpcd_problem *pr, const wpcd_P *P, const double *E, int n_E,
                  const wpcd_solve_opts *o, double *U00, wpcd_solve_stats *st_out, cudaStream_t s) {
  wpcd_solve_opts opt{WPCD_SUM_KRYLOV, 100, 4, 1e-10, 4};
  if (o) opt = *o;
  if (opt.max_iter < 2 || opt.max_iter > 512) return set_error(WPCD_EINVAL, "max_iter must be in [2, 512]");
  if (!(opt.tol > 0.0)) return set_error(WPCD_EINVAL, "tol must be positive");
  if (opt.method != WPCD_SUM_KRYLOV && opt.method != WPCD_SUM_WYNN) return set_error(WPCD_EINVAL, "unknown method");
  if (n_E < 0 || (n_E > 0 && (!E || !U00))) return set_error(WPCD_EINVAL, "bad energies / output");
  for (int e = 0; e < n_E; ++e) {
    int j0;
    double lo, hi;
    wpcd_status st = onshell(pr, E[e], &j0, &lo, &hi, nullptr);
    if (st != WPCD_OK) return st;
  }
  WPCD_CUDA_TRY(cudaSetDevice(pr->device));
  const size_t dim = (size_t)pr->n_ch * pr->N * pr->M;
  const int m = opt.max_iter;
  SolveBuffers B;
  Workspace ws;
  const size_t nvec = opt.method == WPCD_SUM_KRYLOV ? (size_t)m + 1 : 1;
  WPCD_CUDA_TRY(cudaMalloc(&ws.y, 16 * dim));
  WPCD_CUDA_TRY(cudaMalloc(&ws.z, 16 * dim));
  WPCD_CUDA_TRY(cudaMalloc(&B.g, 16 * dim));
  WPCD_CUDA_TRY(cudaMalloc(&B.V, 16 * dim * nvec));
  WPCD_CUDA_TRY(cudaMalloc(&B.w, 16 * dim));
  WPCD_CUDA_TRY(cudaMalloc(&B.u, 16 * dim));
  WPCD_CUDA_TRY(cudaMalloc(&B.small, sizeof(double2) * ((size_t)(m + 1) * (m + 8) + 16)));
  WPCD_CUDA_TRY(cudaMalloc(&B.partial, sizeof(double2) * (size_t)(m + 1) * 152 * 2));
  WPCD_CUDA_TRY(cudaMalloc(&B.resid, sizeof(double)));
  WPCD_CUDA_TRY(cudaMalloc(&B.flag, sizeof(int)));
  WPCD_CUDA_TRY(cudaMalloc(&B.amp, sizeof(double) * 8));
  wpcd_status worst = WPCD_OK;
  for (int e = 0; e < n_E; ++e) {
    wpcd_solve_stats one{};
    wpcd_status st = opt.method == WPCD_SUM_KRYLOV ? solve_krylov(pr, P, E[e], opt, B, ws, one, s)
                                                   : solve_wynn(pr, P, E[e], opt, B, ws, one, s);
    if (st != WPCD_OK) return st;
    U00[2 * e] = one.U00[0];
    U00[2 * e + 1] = one.U00[1];
    if (st_out) st_out[e] = one;
    if (one.status < worst) worst = one.status;
  }
  if (worst != WPCD_OK)
    set_error(worst, worst == WPCD_ENOCONV ? "summation did not reach the tolerance for some energy"
                                           : "Pade/Krylov breakdown for some energy");
  return worst;
}

}  // namespace wpcd
