// Steps 3 and 4 of the numerical scheme (Sec. 3.3): the channel resolvent
// G1 and the iterative solution of the matrix Faddeev equation (Eq. m_pvg)
// with the factorised kernel K = O P0 Vt G1 (Eq. kernel), batched over
// energies.
//
// Device layout of a batch of B energies: the energy index is innermost,
// element (r, e) of a channel-basis vector at r * B + e (complex
// interleaved), r = ch*N*M + k*M + j.  So an [N][M][B] complex block per
// channel is an [N][2MB] real matrix and one K application is
//   gemm_kernel<T>   Y[ch] = Vt[ch] (G1 o X)[ch]   (G1 fused into the B load)
//   spmm_kernel      Z[l][c][e] = sum_{c', l'} P0[(l,c),(l',c')] Y[l'][c'][e]
//   gemm_kernel<T>   X'[ch] = O[ch] Z[ch]           (optional epilogue S - .)
// P0 is read once for the whole batch; each energy has its own G1.
//
// Summation of the iterates:
//   KRYLOV (vector form)  Arnoldi with two-pass classical Gram-Schmidt on the
//          iterates of (I - K), one basis per energy, Givens updates on the
//          device: the minimal-residual (reduced-rank) extrapolation of the
//          iterates.  FP64, or MIXED: FP32 inner cycles (FP32 values,
//          compensated SpMM sums, CUDA-graph replay) inside an FP64
//          iterative-refinement loop r = b - (I - K) u.
//   WYNN (the paper's scalar route)  c_n = e0^T K^n u0 summed by Wynn's
//          epsilon algorithm on the device (FP64, one energy at a time).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "wpcd_internal.h"

namespace wpcd {
namespace {



// ---------------------------------------------------------------------------
// resolvent
// ---------------------------------------------------------------------------
// 1 / i for the Mercator series of log(1 + x)
__constant__ double kInvInt[17] = {0.0,       1.0,        1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,
                                   1.0 / 6,   1.0 / 7,    1.0 / 8,  1.0 / 9,  1.0 / 10, 1.0 / 11,
                                   1.0 / 12,  1.0 / 13,   1.0 / 14, 1.0 / 15, 1.0 / 16};

// reciprocal constants: an FP64 division costs a multi-instruction
// sequence on the narrow FP64 pipe, a multiplication one instruction
constexpr double kThird = 1.0 / 3.0, kSixth = 1.0 / 6.0, kNinth = 1.0 / 9.0;
constexpr double kTwoThirds = 2.0 / 3.0, kFourThirds = 4.0 / 3.0;

__device__ double f_lin(double q, double s, double sg) {
  // antiderivative of q^2 ln|q + sg s|; (q^3 + sg s^3) ln|.| -> 0 at q = -sg s
  double d = q + sg * s;
  double cube = d * (q * q - sg * q * s + s * s);  // q^3 + sg s^3
  double lg = d == 0.0 ? 0.0 : cube * log(fabs(d)) * kThird;
  return lg - q * q * q * kNinth + sg * s * q * q * kSixth - s * s * q * kThird;
}

// int_{qa}^{qb} q^2 ln|a - 3q^2/4| dq without the ln(3/4) B term (it cancels
// in the difference taken by the caller)
__device__ double phi_noconst(double qa, double qb, double a) {
  if (a > 0.0) {
    double s = sqrt(a * kFourThirds);
    return f_lin(qb, s, 1.0) + f_lin(qb, s, -1.0) - f_lin(qa, s, 1.0) - f_lin(qa, s, -1.0);
  }
  if (a < 0.0) {
    double t = sqrt(-a * kFourThirds), it = 1.0 / t;
    auto F = [&](double q) {
      return q * q * q * kThird * log(q * q + t * t) -
             kTwoThirds * (q * q * q * kThird - t * t * q + t * t * t * atan(q * it));
    };
    return F(qb) - F(qa);
  }
  auto F0 = [&](double q) { return q > 0.0 ? kTwoThirds * q * q * q * (log(q) - kThird) : 0.0; };
  return F0(qb) - F0(qa);
}

struct ResParams {
  int n_ch, N, M, n_E, minor;  // n_E: distinct on-shell bins; minor: energy index innermost
  int n_out;                   // energies of the output (the bins' energies, uoff / elist)
  const int *uoff, *elist;     // bin u serves energies elist[uoff[u] .. uoff[u+1]-1]
  const double *qe, *eps;
  const double *Elo, *Ehi;     // per energy
  const double *gl8_t, *gl8_w; // 8-point GL rule
  const double *gl4_t, *gl4_w; // 4-point GL rule
  const double *gl3_t, *gl3_w; // 3-point GL rule
  double4 *shell;              // [n_E][n_ch N] (a_lo, a_hi, sqrt|a_lo|, sqrt|a_hi|)
};

// a = (E - eps) 4/3 at the bin edges E_lo, E_hi of each energy and for each
// pseudostate (the q^2 where 3q^2/4 = E - eps), and sqrt|a|: shared by all
// q-bins, so the main kernel takes no square root
__global__ void res_shell_kernel(ResParams R) {
  const int nchk = R.n_ch * R.N;
  const int64_t total = (int64_t)R.n_E * nchk;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int chk = (int)(idx % nchk), e = (int)(idx / nchk);
    const double ek = R.eps[chk];
    const double alo = (R.Elo[e] - ek) * kFourThirds, ahi = (R.Ehi[e] - ek) * kFourThirds;
    R.shell[idx] = make_double4(alo, ahi, sqrt(fabs(alo)), sqrt(fabs(ahi)));
  }
}

__global__ void resolvent_kernel(ResParams R, double *g) {
  const int dim = R.n_ch * R.N * R.M;
  const int64_t total = (int64_t)R.n_E * dim;
  const int nchk = R.n_ch * R.N;
  // threads run over (on-shell bin, q-bin j, pseudostate ch*N + k) with the
  // pseudostate fastest: a warp shares the energy bin and the q-bin, so its
  // lanes mostly take the same branch below.  G1 depends on an energy only
  // through its on-shell bin (E_lo, E_hi: the average over that energy bin,
  // Sec. 2.3), so each distinct bin is computed once and written for every
  // energy in it (the writes are scattered; their traffic is small next to
  // the arithmetic)
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int chk = (int)(idx % nchk);
    const int64_t rest = idx / nchk;
    const int j = (int)(rest % R.M);
    const int e = (int)(rest / R.M);
    const int r = chk * R.M + j;
    double ek = R.eps[chk];
    double Elo = R.Elo[e], Ehi = R.Ehi[e], D = Ehi - Elo;
    double qa = R.qe[j], qb = R.qe[j + 1];
    double Bq = (qb - qa) * (qb * qb + qb * qa + qa * qa) * kThird;
    double lo_a = Elo - ek - 0.75 * qa * qa, lo_b = Elo - ek - 0.75 * qb * qb;
    double hi_a = Ehi - ek - 0.75 * qa * qa, hi_b = Ehi - ek - 0.75 * qb * qb;
    bool no_sign_change = (lo_a > 0.0 && lo_b > 0.0 && hi_a > 0.0 && hi_b > 0.0) ||
                          (lo_a < 0.0 && lo_b < 0.0 && hi_a < 0.0 && hi_b < 0.0);
    // Where the energy shell does not cross the bin, the real part is the
    // integral of the smooth q^2 log(1 + D / (E_lo - eps - 3q^2/4)); its
    // singularities sit at q^2 = (E_lo - eps)/(3/4) and (E_hi - eps)/(3/4),
    // outside the bin.  At a distance rho, in half bin widths, from the bin
    // centre the n-point GL error falls like r^-2n with r = rho +
    // sqrt(rho^2 - 1) (Bernstein ellipse).  Measured against an 100-point
    // rule on random bins: 3 points for rho > 512 (worst 1.2e-13 relative),
    // 4 for rho > 32 (2.2e-13), 8 for rho > 4 (1.7e-14).  Closer
    // singularities, and bins the shell crosses, take the closed form.
    // rho^2 is compared, from the shared a and sqrt|a| of the pseudostate.
    const double4 sh = R.shell[(int64_t)e * nchk + chk];
    double half = 0.5 * (qb - qa), mid = 0.5 * (qb + qa);
    double rho2 = 0.0;  // (rho half)^2 until the division below
    if (no_sign_change) {
      // a real singular point at sqrt(a) (a > 0), or a complex pair +-i sqrt|a|
      const double dl = sh.x > 0.0 ? (sh.z - mid) * (sh.z - mid) : mid * mid + fabs(sh.x);
      const double dh = sh.y > 0.0 ? (sh.w - mid) * (sh.w - mid) : mid * mid + fabs(sh.y);
      rho2 = fmin(dl, dh) / (half * half);
    }
    double re;
    if (rho2 > 16.0) {
      const int npts = rho2 > 512.0 * 512.0 ? 3 : rho2 > 32.0 * 32.0 ? 4 : 8;
      const double *t = npts == 3 ? R.gl3_t : npts == 4 ? R.gl4_t : R.gl8_t;
      const double *wg = npts == 3 ? R.gl3_w : npts == 4 ? R.gl4_w : R.gl8_w;
      const double dist = fmin(fabs(lo_a), fabs(lo_b));
      const double xmax = fabs(D) / dist;  // |x| at every node of the bin
      double s = 0.0;
      if (xmax < 0.05) {
        // log(1 + x) by its Mercator series, x (1 - x (1/2 - x (1/3 - ...))),
        // with nt terms, nt the least with xmax^nt / (nt + 1) < 1e-17
        int nt = 1;
        for (double pw = xmax; nt < 16 && pw > 1e-17 * (nt + 1); pw *= xmax) ++nt;
        for (int m = 0; m < npts; ++m) {
          double q = mid + half * t[m];
          const double x = D / (Elo - ek - 0.75 * q * q);
          double h = 1.0 / nt;
          for (int i = nt - 1; i >= 1; --i) h = fma(-x, h, kInvInt[i]);
          s += wg[m] * q * q * (x * h);
        }
      } else {
        for (int m = 0; m < npts; ++m) {
          double q = mid + half * t[m];
          s += wg[m] * q * q * log1p(D / (Elo - ek - 0.75 * q * q));
        }
      }
      re = half * s;
    } else {
      re = phi_noconst(qa, qb, Ehi - ek) - phi_noconst(qa, qb, Elo - ek);
    }
    const double inv = 1.0 / (D * Bq);
    re *= inv;
    double im = 0.0;
    if (Ehi - ek > 0.0) {
      double lo = sh.x > 0.0 ? sh.z : 0.0, hi = sh.w;
      double a = fmax(qa, lo), b = fmin(qb, hi);
      if (b > a) im = -kPi * ((b - a) * (b * b + b * a + a * a) * kThird) * inv;
    }
    for (int k = R.uoff[e]; k < R.uoff[e + 1]; ++k) {
      const int eo = R.elist[k];
      const int64_t out = R.minor ? (int64_t)r * R.n_out + eo : (int64_t)eo * dim + r;
      g[2 * out] = re;
      g[2 * out + 1] = im;
    }
  }
}

// ---------------------------------------------------------------------------
// dense block GEMM:  C[b] (n x ncol) = A[b] (n x n) * B'[b] (n x ncol)
// B' = B, or the G1-scaled complex block (complex pairs along the columns)
// epilogue: C = out, or C = S - out
// ---------------------------------------------------------------------------
// 32 x 64 output tiles: 7 x 7 x 3 = 147 CTAs for the 200-bin, 3-channel,
// one-energy blocks, close to one wave over the 152 SMs (FP64 work is
// issue-bound, so SM coverage matters more than data reuse there)
// one 32 x 64 output tile per CTA; grid.z walks the channel blocks
template <typename T, bool SCALE_G, bool SUB>
__global__ void __launch_bounds__(G_THREADS) gemm_kernel(int n, int64_t ncol, const T *__restrict__ A,
                                                         const T *__restrict__ B,
                                                         const T *__restrict__ G,
                                                         const T *__restrict__ S, T *__restrict__ C) {
  __shared__ GemmSmem<T> sm;
  const int b = blockIdx.z;
  const size_t offA = (size_t)b * n * n, offB = (size_t)b * n * ncol;
  gemm_tile<T, SCALE_G, SUB>(n, ncol, A + offA, B + offB, SCALE_G ? G + offB : nullptr, SUB ? S + offB : nullptr,
                             C + offB, blockIdx.y * GB_M, (int64_t)blockIdx.x * GB_N, sm);
}

// ---------------------------------------------------------------------------
// block-CSR SpMM on complex batches: Z[l][c][e] = sum P0 Y[l'][c'][e]
// A warp holds `rpw` rows; each row's 32/rpw lanes split into `el` energy
// lanes times 32/(rpw el) nonzero lanes; every lane keeps EPT energies
// (RHS tile = el * EPT, grid.y walks the tiles).  Values pair-major.
// FP64 sums in double; FP32 sums blocked and compensated (spmm_row).
// ---------------------------------------------------------------------------

// SACC (FP32): the compensated accumulators live in dynamic shared memory
// (acc_sm: 2 NCH EPT hi/lo pairs per thread) while the row is summed, and
// come back to registers for the lane reduction.  Measured on the 3-channel
// 200 x 200 lattice at 128 energies: 0.82 ms per SpMM at three CTAs per SM
// (80 registers) against 0.92 ms with the sums in registers (123 registers,
// two CTAs per SM); four CTAs per SM spill and lose (1.03 ms).
template <typename VT, typename T, int NCH, int EPT, bool VEC, bool SACC>
__device__ __forceinline__ void spmm_body(const SpmmParams &S, const VT *__restrict__ val,
                                          const typename Cx<T>::t *__restrict__ y, typename Cx<T>::t *__restrict__ z,
                                          float *acc_sm) {
  using C2 = typename Cx<T>::t;
  using Acc = typename AccOf<T>::t;
  static_assert(!SACC || sizeof(T) == 4, "shared-memory accumulators are FP32 compensated sums");
  const int lane = threadIdx.x & 31;
  const int lpr = 32 / S.rpw;          // lanes per row
  const int nl_count = lpr / S.el;     // nonzero lanes per row
  const int r_in = lane / lpr, sub = lane % lpr;
  const int el = sub % S.el, nl = sub / S.el;
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int n_warps = gridDim.x * blockDim.x / 32;
  const int e_base = blockIdx.y * S.el * EPT;
  const int B = S.B;
  // the loop bound depends on the warp only, so every lane reaches the
  // full-mask shuffles below
  for (int base = warp_global * S.rpw; base < S.n_cells; base += n_warps * S.rpw) {
    const int c = base + r_in;
    const bool active = c < S.n_cells;
    Acc acc[NCH][EPT][2];
    const int64_t b = active ? S.row_ptr[c] : 0, e = active ? S.row_ptr[c + 1] : 0;
    // lane energies: strided (el + S.el t); with VEC in adjacent pairs
    // (2 el + S.el (t - t % 2) + t % 2), so that the energy lanes of one
    // 16-byte gather cover 16 S.el contiguous bytes of a vector row
    const int en0 = VEC ? e_base + 2 * el : e_base + el, estride = S.el;
    spmm_row_sums<VT, T, NCH, EPT, VEC, SACC>(b, e, nl, nl_count, S.col, val, S.nnz, y, S.n_cells, B, en0, estride,
                                              acc, acc_sm);
    // reduce over the nonzero lanes of the row (xor offsets el .. lpr/2)
    for (int off = S.el; off < lpr; off <<= 1)
#pragma unroll
      for (int l = 0; l < NCH; ++l)
#pragma unroll
        for (int t = 0; t < EPT; ++t) {
          acc[l][t][0].add_shfl(off);
          acc[l][t][1].add_shfl(off);
        }
    if (active && nl == 0) {
#pragma unroll
      for (int t = 0; t < EPT; ++t) {
        const int en = VEC ? e_base + 2 * el + S.el * (t & ~1) + (t & 1) : e_base + el + S.el * t;
        if (en < B)
#pragma unroll
          for (int l = 0; l < NCH; ++l) {
            C2 out;
            out.x = (T)acc[l][t][0].value();
            out.y = (T)acc[l][t][1].value();
            z[((size_t)l * S.n_cells + c) * B + en] = out;
          }
      }
    }
  }
}

template <typename VT, typename T, int NCH, int EPT, bool VEC>
__global__ void __launch_bounds__(256) spmm_kernel(SpmmParams S, const VT *__restrict__ val,
                                                   const typename Cx<T>::t *__restrict__ y,
                                                   typename Cx<T>::t *__restrict__ z) {
  spmm_body<VT, T, NCH, EPT, VEC, false>(S, val, y, z, nullptr);
}

template <int NCH, int EPT, bool VEC>
__global__ void __launch_bounds__(256, NCH <= 3 ? 3 : 2) spmm_sacc_kernel(SpmmParams S, const float *__restrict__ val,
                                                           const float2 *__restrict__ y, float2 *__restrict__ z) {
  extern __shared__ float acc_sm[];
  spmm_body<float, float, NCH, EPT, VEC, true>(S, val, y, z, acc_sm);
}

template <int NCH, int EPT, bool VEC>
cudaError_t spmm_sacc_smem(size_t *bytes) {
  static bool opted_in = false;
  return sacc_smem<NCH, EPT>(spmm_sacc_kernel<NCH, EPT, VEC>, bytes, opted_in);
}

// ---------------------------------------------------------------------------
// batched Krylov vector kernels (energy index innermost); scalars in FP64
// ---------------------------------------------------------------------------
constexpr int V_THREADS = 256;

// partial[(j * nblk + blk) * B + e] = sum_{rows of blk} conj(V_j[row, e]) w[row, e]
// One pass over w per chunk of JC basis vectors; per-thread sums in the
// vector type T, block sums in FP64.
constexpr int JC = 8;

template <typename T>
__global__ void __launch_bounds__(V_THREADS) bdot_kernel(int rows, int B, int nv,
                                                         const typename Cx<T>::t *__restrict__ V,
                                                         size_t ld, const typename Cx<T>::t *__restrict__ w,
                                                         double2 *__restrict__ partial) {
  using C2 = typename Cx<T>::t;
  __shared__ double2 red[JC][V_THREADS];
  const int EL = blockDim.x;  // energy lanes (<= 32)
  const int RB = blockDim.y;  // row lanes
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * EL + tx;
  const int e = blockIdx.y * EL + tx;
  const int nblk = gridDim.x;
  const int stride = nblk * RB;
  for (int j0 = 0; j0 < nv; j0 += JC) {
    T sx[JC], sy[JC];
#pragma unroll
    for (int c = 0; c < JC; ++c) sx[c] = sy[c] = T(0);
    if (e < B) {
      for (int r = blockIdx.x * RB + ty; r < rows; r += stride) {
        const size_t f = (size_t)r * B + e;
        const C2 b = w[f];
#pragma unroll
        for (int c = 0; c < JC; ++c) {
          if (j0 + c < nv) {
            const C2 a = V[(size_t)(j0 + c) * ld + f];
            sx[c] = fma(a.x, b.x, fma(a.y, b.y, sx[c]));
            sy[c] = fma(a.x, b.y, fma(-a.y, b.x, sy[c]));
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < JC; ++c) red[c][tid] = make_double2((double)sx[c], (double)sy[c]);
    __syncthreads();
    for (int h = RB / 2; h > 0; h >>= 1) {
      if (ty < h)
#pragma unroll
        for (int c = 0; c < JC; ++c) {
          double2 o = red[c][(ty + h) * EL + tx];
          red[c][tid].x += o.x;
          red[c][tid].y += o.y;
        }
      __syncthreads();
    }
    if (ty == 0 && e < B)
#pragma unroll
      for (int c = 0; c < JC; ++c)
        if (j0 + c < nv) partial[((size_t)(j0 + c) * nblk + blockIdx.x) * B + e] = red[c][tx];
    __syncthreads();
  }
}

// The FP32 dots with B even: as bdot_kernel, two adjacent energies per
// thread in 16-byte loads (a warp reads 512 contiguous bytes of each
// vector per row); the block sums in FP32, the cross-block sums (breduce)
// in FP64.  JCT basis vectors per pass over w and U rows per thread per
// iteration, their loads issued together: few vectors leave few loads in
// flight per row, so those launches take more rows at once (the dispatch
// picks U from nv; 1 vector at U = 1 ran at a third of HBM bandwidth, at
// U = 8 at 6.4 TB/s).
template <int JCT, int U>
__global__ void __launch_bounds__(V_THREADS) bdot2_kernel(int rows, int B, int nv, const float4 *__restrict__ V,
                                                          size_t ld2, const float4 *__restrict__ w,
                                                          double2 *__restrict__ partial) {
  __shared__ float4 red[JCT][V_THREADS];
  const int EL = blockDim.x;  // energy-pair lanes (<= 32)
  const int RB = blockDim.y;  // row lanes
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * EL + tx;
  const int B2 = B / 2;
  const int e2 = blockIdx.y * EL + tx;
  const int nblk = gridDim.x;
  const int rstep = nblk * RB;
  for (int j0 = 0; j0 < nv; j0 += JCT) {
    float4 acc[JCT];
#pragma unroll
    for (int c = 0; c < JCT; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e2 < B2) {
      for (int r = blockIdx.x * RB + ty; r < rows; r += U * rstep) {
        float4 b[U], a[U][JCT];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int rr = r + u * rstep;
          const bool ok = rr < rows;
          const size_t f = (size_t)rr * B2 + e2;
          b[u] = ok ? w[f] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int c = 0; c < JCT; ++c)
            a[u][c] = ok && j0 + c < nv ? V[(size_t)(j0 + c) * ld2 + f] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int c = 0; c < JCT; ++c) {
            const float4 av = a[u][c], bv = b[u];
            acc[c].x = fmaf(av.x, bv.x, fmaf(av.y, bv.y, acc[c].x));
            acc[c].y = fmaf(av.x, bv.y, fmaf(-av.y, bv.x, acc[c].y));
            acc[c].z = fmaf(av.z, bv.z, fmaf(av.w, bv.w, acc[c].z));
            acc[c].w = fmaf(av.z, bv.w, fmaf(-av.w, bv.z, acc[c].w));
          }
      }
    }
#pragma unroll
    for (int c = 0; c < JCT; ++c) red[c][tid] = acc[c];
    __syncthreads();
    for (int h = RB / 2; h > 0; h >>= 1) {
      if (ty < h)
#pragma unroll
        for (int c = 0; c < JCT; ++c) {
          const float4 o = red[c][(ty + h) * EL + tx];
          red[c][tid].x += o.x;
          red[c][tid].y += o.y;
          red[c][tid].z += o.z;
          red[c][tid].w += o.w;
        }
      __syncthreads();
    }
    if (ty == 0 && e2 < B2)
#pragma unroll
      for (int c = 0; c < JCT; ++c)
        if (j0 + c < nv) {
          const float4 v = red[c][tx];
          double2 *o = partial + ((size_t)(j0 + c) * nblk + blockIdx.x) * B + 2 * e2;
          o[0] = make_double2(v.x, v.y);
          o[1] = make_double2(v.z, v.w);
        }
    __syncthreads();
  }
}

// partial[blk * B + e] = (sum over blk's rows of |x[row, e]|^2, 0): the norm
// pass, one vector read once, four rows in flight per thread, squares summed
// in the vector type per thread and in FP64 across the block
template <typename T>
__global__ void __launch_bounds__(V_THREADS) bnorm_kernel(int rows, int B, const typename Cx<T>::t *__restrict__ x,
                                                          double2 *__restrict__ partial) {
  __shared__ double red[V_THREADS];
  const int EL = blockDim.x, RB = blockDim.y;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * EL + tx;
  const int e = blockIdx.y * EL + tx;
  const int stride = gridDim.x * RB;
  T acc = T(0);
  if (e < B) {
    int r = blockIdx.x * RB + ty;
    for (; r + 3 * stride < rows; r += 4 * stride) {
      typename Cx<T>::t a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = x[(size_t)(r + u * stride) * B + e];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc = fma(a[u].x, a[u].x, fma(a[u].y, a[u].y, acc));
    }
    for (; r < rows; r += stride) {
      const auto a = x[(size_t)r * B + e];
      acc = fma(a.x, a.x, fma(a.y, a.y, acc));
    }
  }
  red[tid] = (double)acc;
  __syncthreads();
  for (int h = RB / 2; h > 0; h >>= 1) {
    if (ty < h) red[tid] += red[(ty + h) * EL + tx];
    __syncthreads();
  }
  if (ty == 0 && e < B) partial[(size_t)blockIdx.x * B + e] = make_double2(red[tx], 0.0);
}

// out[j * B + e] (+)= sum_blk partial[(j * nblk + blk) * B + e]; also, in
// the vector precision T, coef = sign * (this pass's sum) for an axpy, and
// for a norm pass (nv = 1) inv = 1 / sqrt(sum.x) (0 for a zero norm), so
// that the elementwise kernels do no FP64 arithmetic
template <typename T>
__global__ void breduce_kernel(int nv, int nblk, int B, const double2 *partial, double2 *out, int accumulate,
                               typename Cx<T>::t *coef, double sign, T *inv) {
  // one warp per output (j, e): the lanes stride over the block partials
  const int idx = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (idx >= nv * B) return;  // warp-uniform
  const int j = idx / B, e = idx % B;
  double sx = 0.0, sy = 0.0;
  for (int b = lane; b < nblk; b += 32) {
    const double2 p = partial[((size_t)j * nblk + b) * B + e];
    sx += p.x;
    sy += p.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  if (lane != 0) return;
  if (coef) {
    coef[idx].x = (T)(sign * sx);
    coef[idx].y = (T)(sign * sy);
  }
  if (inv) inv[idx] = (T)(sx > 0.0 ? 1.0 / sqrt(sx) : 0.0);
  if (accumulate) {
    out[idx].x += sx;
    out[idx].y += sy;
  } else {
    out[idx] = make_double2(sx, sy);
  }
}

// launch shape of breduce_kernel: one warp per output
inline int breduce_blocks(int outputs) { return (outputs * 32 + 255) / 256; }

// w[f] += sum_j c[j * B + e] V_j[f]   (coefficients in the vector precision)
template <typename T>
__global__ void baxpy_kernel(int64_t n, int B, int nv, const typename Cx<T>::t *__restrict__ V,
                             size_t ld, const typename Cx<T>::t *__restrict__ c,
                             typename Cx<T>::t *__restrict__ w) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(f % B);
    T ax = w[f].x, ay = w[f].y;
    for (int j = 0; j < nv; ++j) {
      const auto a = V[(size_t)j * ld + f];
      const auto cj = c[j * B + e];
      ax = fma(cj.x, a.x, fma(-cj.y, a.y, ax));
      ay = fma(cj.x, a.y, fma(cj.y, a.x, ay));
    }
    w[f].x = ax;
    w[f].y = ay;
  }
}

// the FP32 axpy with B even: two adjacent energies of one row per thread,
// in 16-byte loads of the vectors and of the coefficients (n2 = n / 2)
__global__ void baxpy2_kernel(int64_t n2, int B2, int nv, const float4 *__restrict__ V, size_t ld2,
                              const float4 *__restrict__ c, float4 *__restrict__ w) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n2;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int e2 = (int)(f % B2);
    float4 a = w[f];
    for (int j = 0; j < nv; ++j) {
      const float4 v = V[(size_t)j * ld2 + f];
      const float4 cj = c[j * B2 + e2];
      a.x = fmaf(cj.x, v.x, fmaf(-cj.y, v.y, a.x));
      a.y = fmaf(cj.x, v.y, fmaf(cj.y, v.x, a.y));
      a.z = fmaf(cj.z, v.z, fmaf(-cj.w, v.w, a.z));
      a.w = fmaf(cj.z, v.w, fmaf(cj.w, v.z, a.w));
    }
    w[f] = a;
  }
}

// the same with the vector count bounded by NVT: every vector's load for the
// element is issued before the multiply-adds (the runtime loop waits on one
// load per vector: 4.8-5.0 TB/s at 8-10 vectors), the sums in the same order;
// 32-bit index arithmetic (n2 < 2^31)
// NORM: the norm pass of the Arnoldi step folded in: each thread sums the
// squares of its two energies' new values (the grid stride is a multiple of
// B2, so a thread keeps its energies), and the block writes
// partial[blk * B + e] = (sum, 0) as the norm kernel does
template <int NVT, bool NORM>
__global__ void __launch_bounds__(256) baxpy2t_kernel(int n2, int B2, int nv, const float4 *__restrict__ V,
                                                      size_t ld2, const float4 *__restrict__ c,
                                                      float4 *__restrict__ w, double2 *__restrict__ partial) {
  float s0 = 0.f, s1 = 0.f;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < n2; f += gridDim.x * blockDim.x) {
    const int e2 = f % B2;
    float4 v[NVT];
#pragma unroll
    for (int j = 0; j < NVT; ++j) v[j] = j < nv ? V[(size_t)j * ld2 + f] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 a = w[f];
#pragma unroll
    for (int j = 0; j < NVT; ++j)
      if (j < nv) {
        const float4 cj = c[j * B2 + e2];
        a.x = fmaf(cj.x, v[j].x, fmaf(-cj.y, v[j].y, a.x));
        a.y = fmaf(cj.x, v[j].y, fmaf(cj.y, v[j].x, a.y));
        a.z = fmaf(cj.z, v[j].z, fmaf(-cj.w, v[j].w, a.z));
        a.w = fmaf(cj.z, v[j].w, fmaf(cj.w, v[j].z, a.w));
      }
    w[f] = a;
    if (NORM) {
      s0 = fmaf(a.x, a.x, fmaf(a.y, a.y, s0));
      s1 = fmaf(a.z, a.z, fmaf(a.w, a.w, s1));
    }
  }
  if (NORM) {
    __shared__ double red[2][256];
    const int tid = threadIdx.x;
    red[0][tid] = s0;
    red[1][tid] = s1;
    __syncthreads();
    if (tid < B2) {  // threads tid, tid + B2, ... hold energies 2 tid, 2 tid + 1
      double t0 = 0.0, t1 = 0.0;
      for (int q = tid; q < 256; q += B2) {
        t0 += red[0][q];
        t1 += red[1][q];
      }
      partial[(size_t)blockIdx.x * 2 * B2 + 2 * tid] = make_double2(t0, 0.0);
      partial[(size_t)blockIdx.x * 2 * B2 + 2 * tid + 1] = make_double2(t1, 0.0);
    }
  }
}

// dst[f] = src[f] * inv[e]
// the FP32 scaling with B even: two adjacent energies per thread in 16-byte
// loads, 32-bit index arithmetic (n2 = n / 2 < 2^31)
__global__ void bscale2_kernel(int n2, int B2, const float4 *__restrict__ src, const float2 *__restrict__ inv,
                               float4 *__restrict__ dst) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < n2; f += gridDim.x * blockDim.x) {
    const float2 sc = inv[f % B2];
    const float4 a = src[f];
    dst[f] = make_float4(a.x * sc.x, a.y * sc.x, a.z * sc.y, a.w * sc.y);
  }
}

template <typename T>
__global__ void bscale_kernel(int64_t n, int B, const typename Cx<T>::t *src, const T *__restrict__ inv,
                              typename Cx<T>::t *dst) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n;
       f += (int64_t)gridDim.x * blockDim.x) {
    const T sc = inv[(int)(f % B)];
    dst[f].x = src[f].x * sc;
    dst[f].y = src[f].y * sc;
  }
}

// u[f] += sum_j c[j * B + e] V_j[f]: the correction formed in the basis
// precision T (coefficients from bupdate_coef_kernel), added to u in FP64
template <typename T>
__global__ void bupdate_kernel(int64_t n, int B, int k, const typename Cx<T>::t *__restrict__ V,
                               size_t ld, const typename Cx<T>::t *__restrict__ c, double2 *__restrict__ u) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(f % B);
    T ax = T(0), ay = T(0);
    for (int j = 0; j < k; ++j) {
      const auto a = V[(size_t)j * ld + f];
      const auto cj = c[(size_t)j * B + e];
      ax = fma(cj.x, a.x, fma(-cj.y, a.y, ax));
      ay = fma(cj.x, a.y, fma(cj.y, a.x, ay));
    }
    u[f].x += (double)ax;
    u[f].y += (double)ay;
  }
}


// the FP32 update with B even: two adjacent energies per thread, 16-byte
// loads of the basis and the coefficients; u += sum_j c_j V_j in FP64
__global__ void bupdate2_kernel(int64_t n2, int B2, int k, const float4 *__restrict__ V, size_t ld2,
                                const float4 *__restrict__ c, double2 *__restrict__ u) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n2;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int e2 = (int)(f % B2);
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j = 0; j < k; ++j) {
      const float4 v = V[(size_t)j * ld2 + f];
      const float4 cj = c[(size_t)j * B2 + e2];
      a.x = fmaf(cj.x, v.x, fmaf(-cj.y, v.y, a.x));
      a.y = fmaf(cj.x, v.y, fmaf(cj.y, v.x, a.y));
      a.z = fmaf(cj.z, v.z, fmaf(-cj.w, v.w, a.z));
      a.w = fmaf(cj.z, v.w, fmaf(cj.w, v.z, a.w));
    }
    double2 u0 = u[2 * f], u1 = u[2 * f + 1];
    u0.x += (double)a.x;
    u0.y += (double)a.y;
    u1.x += (double)a.z;
    u1.y += (double)a.w;
    u[2 * f] = u0;
    u[2 * f + 1] = u1;
  }
}

// dst32[f] = (float)(src[f] * inv[e]) (the inner cycle's start vector,
// scaled in FP64 and rounded once)
__global__ void bnormalize_f32_kernel(int64_t n, int B, const double2 *src, const double *__restrict__ inv,
                                      float2 *dst) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n;
       f += (int64_t)gridDim.x * blockDim.x) {
    const double sc = inv[(int)(f % B)];
    const double2 v = src[f];
    dst[f] = make_float2(f64_to_f32_rn(v.x * sc), f64_to_f32_rn(v.y * sc));
  }
}

__global__ void d2f_kernel(int64_t n, const double *src, float *dst) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n;
       f += (int64_t)gridDim.x * blockDim.x)
    dst[f] = f64_to_f32_rn(src[f]);
}

// unit vectors: X[r0[e] * B + e] = 1
__global__ void bunits_kernel(int64_t n, int B, const int *r0, double2 *x) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(f % B);
    const int64_t r = f / B;
    x[f] = make_double2(r == r0[e] ? 1.0 : 0.0, 0.0);
  }
}

// energy-major [B][dim] <-> energy-minor [dim][B] (complex)
__global__ void transpose_kernel(int64_t dim, int B, const double2 *src, double2 *dst, int to_minor) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < dim * B;
       f += (int64_t)gridDim.x * blockDim.x) {
    if (to_minor) {
      const int64_t r = f / B;
      const int e = (int)(f % B);
      dst[f] = src[(size_t)e * dim + r];
    } else {
      const int e = (int)(f / dim);
      const int64_t r = f % dim;
      dst[f] = src[(size_t)r * B + e];
    }
  }
}

// S = 1 - 2 pi i U00 / D, paper's A; out[e * 6 + ...]
__global__ void bamplitude_kernel(int B, const double2 *u, const int *r0, const double *D,
                                  const double *pref, double *out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  double2 U = u[(size_t)r0[e] * B + e];
  double *o = out + 6 * (size_t)e;
  o[0] = U.x;
  o[1] = U.y;
  o[2] = 1.0 + 2.0 * kPi * U.y / D[e];
  o[3] = -2.0 * kPi * U.x / D[e];
  o[4] = pref[e] * U.x;
  o[5] = pref[e] * U.y;
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
      if (d2 == 0.0) {
        bd = 1;
        break;
      }
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


// ---------------------------------------------------------------------------
// K application machinery
// ---------------------------------------------------------------------------
template <typename T>
struct Workspace {
  T *y = nullptr, *z = nullptr;  // [dim * B] complex
  cudaStream_t st = nullptr;     // stream of the pool frees
  ~Workspace() {
    pool_free(y, st);
    pool_free(z, st);
  }
  cudaError_t alloc(size_t dim, int B, cudaStream_t s) {
    st = s;
    cudaError_t e = pool_malloc(&y, 2 * sizeof(T) * dim * B, s);
    if (e != cudaSuccess) return e;
    return pool_malloc(&z, 2 * sizeof(T) * dim * B, s);
  }
};

template <typename VT, typename T>
wpcd_status launch_spmm_cfg(const wpcd_problem *pr, const wpcd_P *P, const VT *val, const T *y, T *z,
                            int B, const SpmmConfig &cfg, cudaStream_t s) {
  // one right-hand side with values in the vectors' precision: the SpMV of
  // spmv.cu (cfg.rpw rows per warp, cfg.ept chunks per step)
  if (B == 1 && sizeof(VT) == sizeof(T)) return launch_spmv1(pr, P, sizeof(T) == 8, val, y, z, cfg, s);
  // the row-tiled FP32 SpMM (spmm_tile.cu)
  if (cfg.tile) {
    if constexpr (sizeof(T) == 4 && sizeof(VT) == 4)
      return launch_spmm_tile(pr, const_cast<wpcd_P *>(P), reinterpret_cast<const float *>(val),
                              reinterpret_cast<const float *>(y), reinterpret_cast<float *>(z), B, cfg, s);
    return set_error(WPCD_EINVAL, "tile SpMM: FP32 values and vectors only");
  }
  SpmmParams S{};
  S.n_cells = pr->N * pr->M;
  S.B = B;
  S.rpw = cfg.rpw;
  S.el = cfg.el;
  S.row_ptr = P->row_ptr;
  S.col = P->col;
  S.nnz = P->nnz;
  using C2 = typename Cx<T>::t;
  const C2 *yy = reinterpret_cast<const C2 *>(y);
  C2 *zz = reinterpret_cast<C2 *>(z);
  const int rows_per_block = 8 * cfg.rpw;
  dim3 grid(grid_for((int64_t)S.n_cells, rows_per_block, 152 * 16),
            (B + cfg.el * cfg.ept - 1) / (cfg.el * cfg.ept));
  // FP32 vectors with an even batch load two adjacent energies at a time
  const bool vec = sizeof(T) == 4 && B % 2 == 0;
  // FP32 (values and vectors): compensated sums in shared memory
  constexpr bool sacc = sizeof(T) == 4 && sizeof(VT) == 4;
#define WPCD_SPMM_EPT(NCH, EPT, VEC)                                                                      \
  do {                                                                                                    \
    if constexpr (sacc) {                                                                                 \
      size_t smem = 0;                                                                                    \
      cudaError_t ae = spmm_sacc_smem<NCH, EPT, VEC>(&smem);                                              \
      if (ae != cudaSuccess) return cuda_error(ae, "spmm shared-memory attribute");                       \
      spmm_sacc_kernel<NCH, EPT, VEC><<<grid, 256, smem, s>>>(S, reinterpret_cast<const float *>(val),    \
                                  reinterpret_cast<const float2 *>(yy), reinterpret_cast<float2 *>(zz));  \
    } else {                                                                                              \
      spmm_kernel<VT, T, NCH, EPT, VEC><<<grid, 256, 0, s>>>(S, val, yy, zz);                             \
    }                                                                                                     \
  } while (0)
#define WPCD_SPMM_CASE(NCH)                                                          \
  case NCH:                                                                          \
    if (cfg.ept == 1)                                                                \
      WPCD_SPMM_EPT(NCH, 1, false);                                                  \
    else if (cfg.ept == 2) {                                                         \
      if (vec)                                                                       \
        WPCD_SPMM_EPT(NCH, 2, sizeof(T) == 4);                                       \
      else                                                                           \
        WPCD_SPMM_EPT(NCH, 2, false);                                                \
    } else {                                                                         \
      if (vec)                                                                       \
        WPCD_SPMM_EPT(NCH, 4, sizeof(T) == 4);                                       \
      else                                                                           \
        WPCD_SPMM_EPT(NCH, 4, false);                                                \
    }                                                                                \
    break;
  switch (pr->n_ch) {
    WPCD_SPMM_CASE(1)
    WPCD_SPMM_CASE(2)
    WPCD_SPMM_CASE(3)
    WPCD_SPMM_CASE(4)
    WPCD_SPMM_CASE(5)
    default:
      return set_error(WPCD_EINVAL, "unsupported channel count for the SpMM");
  }
#undef WPCD_SPMM_CASE
#undef WPCD_SPMM_EPT
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "spmm launch");
}


std::mutex g_tune_mutex;

// choices made in this process, shared by every P0 of the same shape: the
// tuning key plus the value precision, the nonzero count and the device
// (a re-assembled P0 of an unchanged problem reuses the choice)
std::map<std::tuple<int64_t, int, int64_t, int>, SpmmConfig> g_tuned_shapes;

bool load_cached(int64_t key, SpmmConfig *out) {
  const char *path = std::getenv("WPCD_TUNE_CACHE");
  if (!path || !*path) return false;
  std::ifstream f(path);
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    long long k;
    SpmmConfig c;
    // a shape the kernels can run: rows per warp and energy lanes powers of
    // two sharing the 32 lanes, 1, 2 or 4 energies per lane; others ignored
    const auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    // an optional fifth field: cells per tile of the row-tiled SpMM (2 or 4)
    if (is >> k >> c.rpw >> c.el >> c.ept && k == key && pow2(c.rpw) && pow2(c.el) && c.rpw * c.el <= 64 &&
        (c.ept == 1 || c.ept == 2 || c.ept == 4)) {
      if (!(is >> c.tile)) c.tile = 0;
      if (c.tile == 0 ? c.rpw * c.el > 32
                      : !((c.tile == 2 && (c.ept == 2 || c.ept == 4)) || (c.tile == 4 && c.ept == 2)) || c.rpw > 2)
        continue;
      *out = c;
      found = true;
    }
  }
  return found;
}

void store_cached(int64_t key, const SpmmConfig &c) {
  const char *path = std::getenv("WPCD_TUNE_CACHE");
  if (!path || !*path) return;
  std::ofstream f(path, std::ios::app);
  f << (long long)key << " " << c.rpw << " " << c.el << " " << c.ept << " " << c.tile << "\n";
}

}  // namespace

// Time every candidate launch shape on the real P0 (3 launches each, CUDA
// events, the minimum kept) and remember the fastest.  mode: 0 FP64
// vectors, 1 FP32, 2 float-float (the refinement residual's SpMM).
wpcd_status tune_spmm(const wpcd_problem *pr, wpcd_P *P, int B, int mode, cudaStream_t s, SpmmConfig *out) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  if (mode < 0 || mode > 2) return set_error(WPCD_EINVAL, "unknown SpMM tuning mode");
  const bool fp32 = mode == 1, ff = mode == 2;
  const int64_t key = spmm_tune_key(pr->n_ch, pr->N, pr->M, B, mode);
  auto it = P->tuned.find(key);
  if (it != P->tuned.end()) {
    *out = it->second;
    return WPCD_OK;
  }
  const auto shape = std::make_tuple(key, P->prec, P->nnz, pr->device);
  auto its = g_tuned_shapes.find(shape);
  if (its != g_tuned_shapes.end()) {
    P->tuned[key] = its->second;
    *out = its->second;
    return WPCD_OK;
  }
  SpmmConfig cached;
  if (load_cached(key, &cached)) {
    P->tuned[key] = cached;
    *out = cached;
    return WPCD_OK;
  }
  if (fp32 && !P->val32 && !P->val32_copy) return set_error(WPCD_EINVAL, "no FP32 values to tune on");
  if (ff && P->prec == WPCD_FP64 && !P->val_h) return set_error(WPCD_EINVAL, "no float-float values to tune on");
  std::vector<SpmmConfig> cands = candidates(B);
  if (fp32 && B >= 16 && tile_supported(pr, B))  // the row-tiled SpMM: 2-cell tiles (4 or 2 energies per lane), 2 x 2
    for (int fab : {1, 2})  // rpw: plain blocks of 32 (1) or 64 (2) columns
      for (const SpmmConfig &c : {SpmmConfig{fab, 32, 4, 2}, SpmmConfig{fab, 32, 2, 2}, SpmmConfig{fab, 32, 2, 4}})
        cands.push_back(c);
  const size_t dim = (size_t)pr->n_ch * pr->N * pr->M;
  void *y = nullptr, *z = nullptr;
  // float-float vectors: hi and lo float arrays, the size of one FP64 vector
  const size_t esz = fp32 ? sizeof(float) : sizeof(double);
  WPCD_CUDA_TRY(dev_malloc(&y, 2 * esz * dim * B));
  cudaError_t ce = dev_malloc(&z, 2 * esz * dim * B);
  if (ce != cudaSuccess) {
    dev_free(y);
    return cuda_error(ce, "cudaMalloc (tuning)");
  }
  cudaMemsetAsync(y, 0, 2 * esz * dim * B, s);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  SpmmConfig pick;
  wpcd_status st = WPCD_OK;
  for (const SpmmConfig &c : cands) {
    float tmin = 1e30f;
    for (int rep = 0; rep < 3 && st == WPCD_OK; ++rep) {
      cudaEventRecord(a, s);
      if (ff) {
        const size_t half = 2 * dim * (size_t)B;  // floats per part
        st = launch_spmm_df_cfg(pr, P, (const float *)y, (const float *)y + half, (float *)z, (float *)z + half, B,
                                c, s);
      } else if (fp32) {
        const float *v32 = P->val32 ? P->val32 : P->val32_copy;
        st = launch_spmm_cfg<float, float>(pr, P, v32, (const float *)y, (float *)z, B, c, s);
      } else if (P->prec == WPCD_FP64) {
        st = launch_spmm_cfg<double, double>(pr, P, P->val64, (const double *)y, (double *)z, B, c, s);
      } else {
        st = launch_spmm_cfg<float, double>(pr, P, P->val32, (const double *)y, (double *)z, B, c, s);
      }
      cudaEventRecord(b, s);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      tmin = std::min(tmin, ms);
    }
    if (st != WPCD_OK) break;
    if (std::getenv("WPCD_TUNE_LOG"))
      std::fprintf(stderr, "wpcd tune B=%d mode=%d rpw=%d el=%d ept=%d tile=%d: %.4f ms\n", B, mode, c.rpw, c.el,
                   c.ept, c.tile, tmin);
    if (tmin < best) {
      best = tmin;
      pick = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  dev_free(y);
  dev_free(z);
  if (st != WPCD_OK) return st;
  P->tuned[key] = pick;
  g_tuned_shapes[shape] = pick;
  store_cached(key, pick);
  *out = pick;
  return WPCD_OK;
}

namespace {

// SpMM with the tuned shape (values: the P's own precision for FP64 T, FP32
// values for FP32 T)
template <typename T>
wpcd_status spmm(const wpcd_problem *pr, const wpcd_P *P, const T *y, T *z, int B, cudaStream_t s) {
  SpmmConfig cfg;
  wpcd_status st = tune_spmm(pr, const_cast<wpcd_P *>(P), B, sizeof(T) == 4 ? 1 : 0, s, &cfg);
  if (st != WPCD_OK) return st;
  if (sizeof(T) == 4) {
    const float *v32 = P->val32 ? P->val32 : P->val32_copy;
    return launch_spmm_cfg<float, float>(pr, P, v32, (const float *)y, (float *)z, B, cfg, s);
  }
  if (P->prec == WPCD_FP64)
    return launch_spmm_cfg<double, double>(pr, P, P->val64, (const double *)y, (double *)z, B, cfg, s);
  return launch_spmm_cfg<float, double>(pr, P, P->val32, (const double *)y, (double *)z, B, cfg, s);
}

// out = O P0 Vt (g o x)  or  out = sub - O P0 Vt (g o x), batch of B energies
template <typename T>
wpcd_status kapply_ws(const wpcd_problem *pr, const wpcd_P *P, const T *g, const T *x, T *out,
                      const T *sub, int B, Workspace<T> &ws, cudaStream_t s) {
  const int N = pr->N, M = pr->M, n_ch = pr->n_ch;
  const int64_t ncol = 2LL * M * B;
  const T *Vt = sizeof(T) == 8 ? (const T *)(const void *)pr->d.Vt : (const T *)(const void *)pr->d.Vt32;
  const T *O = sizeof(T) == 8 ? (const T *)(const void *)pr->d.O : (const T *)(const void *)pr->d.O32;
  if constexpr (sizeof(T) == 4) {
    // FP32 vectors: tensor-core channel blocks when the operands are packed
    if (pr->d.O_tc && tc_enabled()) {
      wpcd_status st = tc_gemm(pr, false, (const float *)g, (const float *)x, nullptr, (float *)ws.y, ncol, s);
      if (st == WPCD_OK) st = spmm<T>(pr, P, ws.y, ws.z, B, s);
      if (st == WPCD_OK) st = tc_gemm(pr, true, nullptr, (const float *)ws.z, (const float *)sub, (float *)out, ncol, s);
      return st;
    }
  }
  dim3 grid((unsigned)((ncol + GB_N - 1) / GB_N), (N + GB_M - 1) / GB_M, n_ch);
  if (g)
    gemm_kernel<T, true, false><<<grid, G_THREADS, 0, s>>>(N, ncol, Vt, x, g, nullptr, ws.y);
  else
    gemm_kernel<T, false, false><<<grid, G_THREADS, 0, s>>>(N, ncol, Vt, x, nullptr, nullptr, ws.y);
  count_launches(1);
  wpcd_status st = spmm<T>(pr, P, ws.y, ws.z, B, s);
  if (st != WPCD_OK) return st;
  if (sub)
    gemm_kernel<T, false, true><<<grid, G_THREADS, 0, s>>>(N, ncol, O, ws.z, nullptr, sub, out);
  else
    gemm_kernel<T, false, false><<<grid, G_THREADS, 0, s>>>(N, ncol, O, ws.z, nullptr, nullptr, out);
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
    if (qe[mid] <= q)
      lo = mid;
    else
      hi = mid - 1;
  }
  *j0 = lo;
  *Elo = pr->eps_b + 0.75 * qe[lo] * qe[lo];
  *Ehi = pr->eps_b + 0.75 * qe[lo + 1] * qe[lo + 1];
  if (q0) *q0 = q;
  return WPCD_OK;
}

namespace {

// max_blocks caps the grid (measured: the full grid is faster than one CTA
// per SM even next to the Born term, which then finds fewer free slots)
wpcd_status resolvent_impl(const wpcd_problem *pr, const double *E, int n_E, double *g, int minor,
                           int *j0, double *D, cudaStream_t s, int max_blocks = 152 * 16) {
  if (n_E < 0 || (n_E > 0 && (!E || !g))) return set_error(WPCD_EINVAL, "bad resolvent arguments");
  if (n_E == 0) return WPCD_OK;
  // distinct on-shell bins (in order of first appearance) and their energies
  std::vector<int> jj(n_E), bin_of(pr->M, -1), uoff, elist(n_E);
  std::vector<double> ulo, uhi;
  for (int e = 0; e < n_E; ++e) {
    double lo, hi;
    wpcd_status st = onshell(pr, E[e], &jj[e], &lo, &hi, nullptr);
    if (st != WPCD_OK) return st;
    if (bin_of[jj[e]] < 0) {
      bin_of[jj[e]] = (int)ulo.size();
      ulo.push_back(lo);
      uhi.push_back(hi);
    }
    if (j0) j0[e] = jj[e];
    if (D) D[e] = hi - lo;
  }
  const int n_U = (int)ulo.size();
  uoff.assign(n_U + 1, 0);
  for (int e = 0; e < n_E; ++e) ++uoff[bin_of[jj[e]] + 1];
  for (int u = 0; u < n_U; ++u) uoff[u + 1] += uoff[u];
  {
    std::vector<int> fill(uoff.begin(), uoff.end() - 1);
    for (int e = 0; e < n_E; ++e) elist[fill[bin_of[jj[e]]]++] = e;
  }
  // staging: E_lo, E_hi per bin, 8-, 4- and 3-point GL rules; the shell
  // table; the bin -> energies lists
  const int64_t n_shell = (int64_t)n_U * pr->n_ch * pr->N;
  std::vector<double> lohi(2 * (size_t)n_U + 30);
  std::copy(ulo.begin(), ulo.end(), lohi.begin());
  std::copy(uhi.begin(), uhi.end(), lohi.begin() + n_U);
  gauss_legendre(8, lohi.data() + 2 * n_U, lohi.data() + 2 * n_U + 8);
  gauss_legendre(4, lohi.data() + 2 * n_U + 16, lohi.data() + 2 * n_U + 20);
  gauss_legendre(3, lohi.data() + 2 * n_U + 24, lohi.data() + 2 * n_U + 27);
  const size_t shell_at = (lohi.size() + 3) & ~(size_t)3;  // in doubles, 32-byte aligned
  const size_t ints_at = shell_at + 4 * (size_t)n_shell;    // in doubles
  std::vector<int> ints(uoff);
  ints.insert(ints.end(), elist.begin(), elist.end());
  WPCD_CUDA_TRY(cudaSetDevice(pr->device));
  double *d_lohi = nullptr;
  WPCD_CUDA_TRY(pool_malloc(&d_lohi, sizeof(double) * ints_at + sizeof(int) * ints.size(), s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(d_lohi, lohi.data(), sizeof(double) * lohi.size(), cudaMemcpyHostToDevice, s));
  int *d_ints = reinterpret_cast<int *>(d_lohi + ints_at);
  WPCD_CUDA_TRY(cudaMemcpyAsync(d_ints, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice, s));
  ResParams R{};
  R.n_ch = pr->n_ch;
  R.N = pr->N;
  R.M = pr->M;
  R.n_E = n_U;
  R.n_out = n_E;
  R.minor = minor;
  R.qe = pr->d.qe;
  R.eps = pr->d.eps;
  R.Elo = d_lohi;
  R.Ehi = d_lohi + n_U;
  R.gl8_t = d_lohi + 2 * n_U;
  R.gl8_w = d_lohi + 2 * n_U + 8;
  R.gl4_t = d_lohi + 2 * n_U + 16;
  R.gl4_w = d_lohi + 2 * n_U + 20;
  R.gl3_t = d_lohi + 2 * n_U + 24;
  R.gl3_w = d_lohi + 2 * n_U + 27;
  R.shell = reinterpret_cast<double4 *>(d_lohi + shell_at);
  R.uoff = d_ints;
  R.elist = d_ints + n_U + 1;
  res_shell_kernel<<<grid_for(n_shell, 256), 256, 0, s>>>(R);
  int64_t total = (int64_t)n_U * pr->n_ch * pr->N * pr->M;
  resolvent_kernel<<<grid_for(total, 256, max_blocks), 256, 0, s>>>(R, g);
  count_launches(2);
  cudaError_t e = cudaGetLastError();
  pool_free(d_lohi, s);
  // a copy from pageable memory returns once the data is staged, so the
  // host vectors may go; no synchronisation (the work stays asynchronous)
  if (e != cudaSuccess) return cuda_error(e, "resolvent launch");
  return WPCD_OK;
}

}  // namespace

// the ABI call synchronises its stream; the solves' internal calls do not
wpcd_status resolvent(const wpcd_problem *pr, const double *E, int n_E, double *g, int *j0,
                      double *D, cudaStream_t s) {
  wpcd_status st = resolvent_impl(pr, E, n_E, g, 0, j0, D, s);
  if (st != WPCD_OK) return st;
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  return WPCD_OK;
}

wpcd_status resolvent_minor(const wpcd_problem *pr, const double *E, int n_E, double *g, cudaStream_t s) {
  return resolvent_impl(pr, E, n_E, g, 1, nullptr, nullptr, s);
}

// One FP64 K application into caller-provided intermediates (two [dim]
// complex buffers) with the SpMM shape already tuned for one right-hand side
// if there is one, else a fixed shape: no allocation, no tuning, no sync.
wpcd_status kapply_scratch(const wpcd_problem *pr, const wpcd_P *P, const double *g, const double *x,
                           double *y, double *scratch_y, double *scratch_z, cudaStream_t s) {
  const int N = pr->N, M = pr->M, n_ch = pr->n_ch;
  const int64_t ncol = 2LL * M;
  dim3 grid((unsigned)((ncol + GB_N - 1) / GB_N), (N + GB_M - 1) / GB_M, n_ch);
  if (g)
    gemm_kernel<double, true, false><<<grid, G_THREADS, 0, s>>>(N, ncol, pr->d.Vt, x, g, nullptr, scratch_y);
  else
    gemm_kernel<double, false, false><<<grid, G_THREADS, 0, s>>>(N, ncol, pr->d.Vt, x, nullptr, nullptr, scratch_y);
  count_launches(1);
  // the choice tune_spmm made for one FP64 right-hand side (mode 0), if any;
  // the map is read under the tuner's lock, which inserts into it
  SpmmConfig cfg{2, 1, 1};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = P->tuned.find(spmm_tune_key(pr->n_ch, pr->N, pr->M, 1, 0));
    if (it != P->tuned.end()) cfg = it->second;
  }

  wpcd_status st = P->prec == WPCD_FP64
                       ? launch_spmm_cfg<double, double>(pr, P, P->val64, scratch_y, scratch_z, 1, cfg, s)
                       : launch_spmm_cfg<float, double>(pr, P, P->val32, scratch_y, scratch_z, 1, cfg, s);
  if (st != WPCD_OK) return st;
  gemm_kernel<double, false, false><<<grid, G_THREADS, 0, s>>>(N, ncol, pr->d.O, scratch_z, nullptr, nullptr, y);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "kapply launch");
}

wpcd_status kapply(const wpcd_problem *pr, const wpcd_P *P, const double *g, const double *x,
                   double *y, cudaStream_t s) {
  WPCD_CUDA_TRY(cudaSetDevice(pr->device));
  const size_t dim = (size_t)pr->n_ch * pr->N * pr->M;
  Workspace<double> ws;
  WPCD_CUDA_TRY(ws.alloc(dim, 1, s));
  wpcd_status st = kapply_ws<double>(pr, P, g, x, y, nullptr, 1, ws, s);
  if (st != WPCD_OK) return st;
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  return WPCD_OK;
}

namespace {

// Krylov basis and least-squares state for a batch of B energies
template <typename T>
struct Krylov {
  int m = 0, B = 0;
  size_t dim = 0;
  T *V = nullptr;  // [(m+1)][dim][B] complex
  T *w = nullptr;  // [dim][B] complex
  double2 *H = nullptr, *cs = nullptr, *sn = nullptr, *bet = nullptr;
  double2 *h = nullptr, *h2 = nullptr, *nrm = nullptr, *y = nullptr, *partial = nullptr;
  double *resid = nullptr, *bnorm = nullptr;
  typename Cx<T>::t *hc = nullptr;  // axpy coefficients in T [(m+1)][B]
  T *inv = nullptr;                  // 1 / |w| per energy in T [B]
  int nblk = 0;
  cudaStream_t st = nullptr;  // stream of the pool frees
  ~Krylov() {
    for (void *q : {(void *)V, (void *)w, (void *)H, (void *)cs, (void *)sn, (void *)bet, (void *)h, (void *)h2,
                    (void *)nrm, (void *)y, (void *)partial, (void *)resid, (void *)bnorm, (void *)hc, (void *)inv})
      pool_free(q, st);
  }
  cudaError_t alloc(int m_, int B_, size_t dim_, cudaStream_t s, bool vectors = true) {
    m = m_;
    B = B_;
    dim = dim_;
    nblk = 152 * 2;
    st = s;
    cudaError_t e;
    if (vectors) {
      if ((e = pool_malloc(&V, 2 * sizeof(T) * dim * B * (m + 1), s)) != cudaSuccess) return e;
      if ((e = pool_malloc(&w, 2 * sizeof(T) * dim * B, s)) != cudaSuccess) return e;
    }
    if ((e = pool_malloc(&H, sizeof(double2) * (size_t)B * (m + 1) * m, s)) != cudaSuccess) return e;
    if ((e = pool_malloc(&cs, sizeof(double2) * (size_t)B * m, s)) != cudaSuccess) return e;
    if ((e = pool_malloc(&sn, sizeof(double2) * (size_t)B * m, s)) != cudaSuccess) return e;
    if ((e = pool_malloc(&bet, sizeof(double2) * (size_t)B * (m + 1), s)) != cudaSuccess) return e;
    if ((e = pool_malloc(&h, sizeof(double2) * (size_t)B * (m + 1), s)) != cudaSuccess) return e;
    if ((e = pool_malloc(&h2, sizeof(double2) * (size_t)B * (m + 1), s)) != cudaSuccess) return e;
    if ((e = pool_malloc(&nrm, sizeof(double2) * (size_t)B, s)) != cudaSuccess) return e;
    if ((e = pool_malloc(&y, sizeof(double2) * (size_t)B * m, s)) != cudaSuccess) return e;
    if ((e = pool_malloc(&partial, sizeof(double2) * (size_t)B * (m + 1) * nblk, s)) != cudaSuccess) return e;
    if ((e = pool_malloc(&resid, sizeof(double) * B, s)) != cudaSuccess) return e;
    if ((e = pool_malloc(&hc, 2 * sizeof(T) * (size_t)B * (m + 1), s)) != cudaSuccess) return e;
    if ((e = pool_malloc(&inv, sizeof(T) * (size_t)B, s)) != cudaSuccess) return e;
    return pool_malloc(&bnorm, sizeof(double) * B, s);
  }
  using C2 = typename Cx<T>::t;
  C2 *vec(int j) { return reinterpret_cast<C2 *>(V) + (size_t)j * dim * B; }
  C2 *wv() { return reinterpret_cast<C2 *>(w); }
  dim3 dot_block() const {
    int el = 1;
    while (el < B && el < 32) el *= 2;
    return dim3(el, V_THREADS / el);
  }
  dim3 dot_grid() const {
    dim3 b = dot_block();
    return dim3(nblk, (B + b.x - 1) / b.x);
  }
  // out[j * B + e] = <V_j, x>, j < nv; with hcoef, also hc = -out in T
  template <typename U>
  void dots(int nv, const typename Cx<U>::t *base, size_t ld, const typename Cx<U>::t *x, double2 *out,
            int accumulate, cudaStream_t s, bool hcoef = false, bool scale = false) {
    if (sizeof(U) == 4 && B % 2 == 0) {  // FP32, B even: two energies per thread
      int el = 1;
      while (el < B / 2 && el < 32) el *= 2;
      const dim3 blk(el, V_THREADS / el), grd(nblk, (B / 2 + el - 1) / el);
      const float4 *Vb = reinterpret_cast<const float4 *>(base), *xb = reinterpret_cast<const float4 *>(x);
      if (nv == 1)
        bdot2_kernel<1, 8><<<grd, blk, 0, s>>>((int)dim, B, nv, Vb, ld / 2, xb, partial);
      else if (nv == 2)
        bdot2_kernel<2, 4><<<grd, blk, 0, s>>>((int)dim, B, nv, Vb, ld / 2, xb, partial);
      else if (nv <= 4)
        bdot2_kernel<4, 2><<<grd, blk, 0, s>>>((int)dim, B, nv, Vb, ld / 2, xb, partial);
      else if (nv <= 6)
        bdot2_kernel<6, 2><<<grd, blk, 0, s>>>((int)dim, B, nv, Vb, ld / 2, xb, partial);
      // more vectors: passes of at most six, w re-read per pass (one pass over
      // eleven or eight vectors, 12 or 9 streams per thread, ran at 3.5-4.2
      // TB/s against 6.5 for six); 7-8 vectors as two passes of four (185,
      // 200 us against 213, 219 as six + rest), 9-10 as six + rest (226, 235
      // us against 240, 251 as two passes of five)
      else if (nv <= 8)
        bdot2_kernel<4, 2><<<grd, blk, 0, s>>>((int)dim, B, nv, Vb, ld / 2, xb, partial);
      else
        bdot2_kernel<6, 2><<<grd, blk, 0, s>>>((int)dim, B, nv, Vb, ld / 2, xb, partial);
    } else {
      bdot_kernel<U><<<dot_grid(), dot_block(), 0, s>>>((int)dim, B, nv, base, ld, x, partial);
    }
    breduce_kernel<T><<<breduce_blocks(nv * B), 256, 0, s>>>(nv, nblk, B, partial, out, accumulate,
                                                           hcoef ? hc : nullptr, -1.0, scale ? inv : nullptr);
    count_launches(2);
  }
  // nrm[e] = |x_e|^2 (and inv = 1 / |x_e| in T with scale)
  template <typename U>
  void norms(const typename Cx<U>::t *x, cudaStream_t s, bool scale = false) {
    bnorm_kernel<U><<<dot_grid(), dot_block(), 0, s>>>((int)dim, B, x, partial);
    breduce_kernel<T><<<breduce_blocks(B), 256, 0, s>>>(1, nblk, B, partial, nrm, 0, nullptr, -1.0,
                                                      scale ? inv : nullptr);
    count_launches(2);
  }
  template <bool NORM>
  void axpy2t(int nv, int g, cudaStream_t s) {
    const int n2 = (int)((int64_t)dim * B / 2);
    const float4 *Vv = reinterpret_cast<const float4 *>(V), *cc = reinterpret_cast<const float4 *>(hc);
    float4 *ww = reinterpret_cast<float4 *>(w);
    const size_t ld2 = dim * B / 2;
    if (nv <= 2)
      baxpy2t_kernel<2, NORM><<<g, 256, 0, s>>>(n2, B / 2, nv, Vv, ld2, cc, ww, partial);
    else if (nv <= 4)
      baxpy2t_kernel<4, NORM><<<g, 256, 0, s>>>(n2, B / 2, nv, Vv, ld2, cc, ww, partial);
    else if (nv <= 8)
      baxpy2t_kernel<8, NORM><<<g, 256, 0, s>>>(n2, B / 2, nv, Vv, ld2, cc, ww, partial);
    else
      baxpy2t_kernel<12, NORM><<<g, 256, 0, s>>>(n2, B / 2, nv, Vv, ld2, cc, ww, partial);
  }
  // w += sum_{j < nv} hc_j V_j (FP32 with B even: two energies per thread).
  // With with_norm, where the shape allows (FP32, B / 2 dividing 256, the
  // partial buffer holding a block partial per block of the axpy's grid),
  // the norm pass's block partials of the new w come out of the same kernel;
  // returns their block count (0: not done)
  int axpy(int nv, cudaStream_t s, bool with_norm = false) {
    const int64_t n = (int64_t)dim * B;
    const bool t_ok = sizeof(T) == 4 && B % 2 == 0 && nv <= 12 && n / 2 < INT32_MAX;
    const int g = grid_for(n / 2, 256);
    if (with_norm && t_ok && 256 % (B / 2) == 0 && g <= (m + 1) * nblk) {
      axpy2t<true>(nv, g, s);
      return g;
    }
    // the unrolled form except at three vectors (112 against 103 us there;
    // 47-256 against 58-292 us elsewhere up to ten)
    if (t_ok && nv != 3) {
      axpy2t<false>(nv, g, s);
    } else if (sizeof(T) == 4 && B % 2 == 0)
      baxpy2_kernel<<<grid_for(n / 2, 256), 256, 0, s>>>(n / 2, B / 2, nv, reinterpret_cast<const float4 *>(V),
                                                         dim * B / 2, reinterpret_cast<const float4 *>(hc),
                                                         reinterpret_cast<float4 *>(w));
    else
      baxpy_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(n, B, nv, vec(0), dim * B, hc, wv());
    return 0;
  }
  // one Arnoldi step from column k (w holds (I - K) v_k on entry); classical
  // Gram-Schmidt with a second pass (reorth = true) or a single pass
  void step(int k, cudaStream_t s, bool reorth = true) {
    const int64_t n = (int64_t)dim * B;
    const size_t ld = dim * B;
    const int vg = grid_for(n, 256);
    dots<T>(k + 1, vec(0), ld, wv(), h, 0, s, true);
    const int normed = axpy(k + 1, s, !reorth);
    if (reorth) {
      dots<T>(k + 1, vec(0), ld, wv(), h2, 0, s, true);
      axpy(k + 1, s);
      // h += h2 (the second pass's partials are still in place)
      breduce_kernel<T><<<breduce_blocks((k + 1) * B), 256, 0, s>>>(k + 1, nblk, B, partial, h, 1, nullptr, 0.0,
                                                                   nullptr);
      count_launches(2);
    }
    if (normed) {  // the axpy left the norm partials of its `normed` blocks
      breduce_kernel<T><<<breduce_blocks(B), 256, 0, s>>>(1, normed, B, partial, nrm, 0, nullptr, -1.0, inv);
      count_launches(1);
    } else {
      norms<T>(wv(), s, true);
    }
    if (sizeof(T) == 4 && B % 2 == 0 && n / 2 < INT32_MAX)
      bscale2_kernel<<<grid_for(n / 2, 256), 256, 0, s>>>((int)(n / 2), B / 2, reinterpret_cast<const float4 *>(wv()),
                                                         reinterpret_cast<const float2 *>(inv),
                                                         reinterpret_cast<float4 *>(vec(k + 1)));
    else
      bscale_kernel<T><<<vg, 256, 0, s>>>(n, B, wv(), inv, vec(k + 1));
    bgivens_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, m, k, h, nrm, H, cs, sn, bet, resid, bnorm);
    count_launches(3);
  }
};

struct SolveCtx {
  int B = 0;
  size_t dim = 0;
  double *g = nullptr;  // [dim][B] complex FP64 resolvent
  float *g32 = nullptr; // FP32 copy (mixed)
  double *b = nullptr, *u = nullptr, *r = nullptr, *t = nullptr;  // FP64 [dim][B] complex
  int *r0 = nullptr;    // [B]
  double *Dd = nullptr, *pref = nullptr, *amp = nullptr;
  cudaStream_t st = nullptr;  // stream of the pool allocations and frees
  ~SolveCtx() {
    for (void *q : {(void *)g, (void *)g32, (void *)b, (void *)u, (void *)r, (void *)t, (void *)r0, (void *)Dd,
                    (void *)pref, (void *)amp})
      pool_free(q, st);
  }
};

struct BatchInfo {
  std::vector<int> j0;
  std::vector<double> D, pref;
};

// on-shell data of the batch (host) and its upload; the resolvent follows
// separately (batch_resolvent) so that it can overlap the Born term
wpcd_status batch_setup(const wpcd_problem *pr, const double *E, int B, SolveCtx &cx, BatchInfo &bi,
                        cudaStream_t s) {
  bi.j0.assign(B, 0);
  bi.D.assign(B, 0.0);
  bi.pref.assign(B, 0.0);
  for (int e = 0; e < B; ++e) {
    double lo, hi, q0;
    wpcd_status st = onshell(pr, E[e], &bi.j0[e], &lo, &hi, &q0);
    if (st != WPCD_OK) return st;
    bi.D[e] = hi - lo;
    bi.pref[e] = 2.0 / (3.0 * q0) / (pr->qe[bi.j0[e] + 1] - pr->qe[bi.j0[e]]);
  }
  // e0 = channel 0, k = 0 (the dimer), q-bin j0: vector index j0
  WPCD_CUDA_TRY(cudaMemcpyAsync(cx.r0, bi.j0.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(cx.Dd, bi.D.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(cx.pref, bi.pref.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s));
  // copies from pageable host memory are staged before the calls return
  return WPCD_OK;
}

// G1 of the batch (and its FP32 copy) on stream s2, ordered after the
// work already queued on s and before the work queued on s afterwards;
// meanwhile s may run the Born term, which does not involve G1 (the
// resolvent keeps the FP64 pipe busy, the float-float Born term the FP32
// pipe)
wpcd_status batch_resolvent(const wpcd_problem *pr, const double *E, int B, SolveCtx &cx, bool need32,
                            cudaStream_t s, cudaStream_t s2, cudaEvent_t before, cudaEvent_t after) {
  const size_t dim = (size_t)pr->n_ch * pr->N * pr->M;
  WPCD_CUDA_TRY(cudaStreamWaitEvent(s2, before, 0));
  wpcd_status st = resolvent_impl(pr, E, B, cx.g, 1, nullptr, nullptr, s2);
  if (st != WPCD_OK) return st;
  if (need32) {
    d2f_kernel<<<grid_for(2 * (int64_t)dim * B, 256), 256, 0, s2>>>(2 * (int64_t)dim * B, cx.g, cx.g32);
    count_launches(1);
  }
  WPCD_CUDA_TRY(cudaEventRecord(after, s2));
  WPCD_CUDA_TRY(cudaStreamWaitEvent(s, after, 0));
  return WPCD_OK;
}

// Vt e0 for every energy: column 0 of Vt_0 placed at (channel 0, q-bin j0)
__global__ void born_vt_kernel(int64_t n, int B, int N, int M, const double *Vt0, const int *r0, double2 *y) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(f % B);
    const int64_t r = f / B;  // ch*N*M + i*M + j
    double v = 0.0;
    if (r < (int64_t)N * M && (int)(r % M) == r0[e]) v = Vt0[(r / M) * N];  // Vt_0[i][0]
    y[f] = make_double2(v, 0.0);
  }
}

// Born term b = O P0 Vt e0 for every energy of the batch (FP64); the unit
// vector makes Vt e0 a column of Vt_0, so only the SpMM and the O GEMM run
wpcd_status born(const wpcd_problem *pr, const wpcd_P *P, SolveCtx &cx, Workspace<double> &ws, cudaStream_t s) {
  const int64_t n = (int64_t)cx.dim * cx.B;
  const int N = pr->N, M = pr->M, n_ch = pr->n_ch, B = cx.B;
  born_vt_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, B, N, M, pr->d.Vt, cx.r0, (double2 *)ws.y);
  count_launches(1);
  wpcd_status st = spmm<double>(pr, P, ws.y, ws.z, B, s);
  if (st != WPCD_OK) return st;
  const int64_t ncol = 2LL * M * B;
  dim3 grid((unsigned)((ncol + GB_N - 1) / GB_N), (N + GB_M - 1) / GB_M, n_ch);
  gemm_kernel<double, false, false><<<grid, G_THREADS, 0, s>>>(N, ncol, pr->d.O, ws.z, nullptr, nullptr, cx.b);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "born launch");
}

// b[r][e] = bu[r][map[e]] (complex FP64, energy index innermost)
__global__ void expand_kernel(int64_t n, int B, int BU, const int *__restrict__ map, const double2 *__restrict__ bu,
                              double2 *__restrict__ b) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(f % B);
    b[f] = bu[(f / B) * BU + map[e]];
  }
}

// Born terms of a batch.  The Born term O P0 Vt e0 depends on an energy only
// through its on-shell bin (e0 is the unit vector of bin j0), so it is formed
// once per distinct bin and copied to each energy of the bin
wpcd_status batch_born(const wpcd_problem *pr, const wpcd_P *P, SolveCtx &cx, const std::vector<int> &j0,
                       bool dfres, Workspace<double> &ws64, DfWork &dfw, cudaStream_t s) {
  const int B = cx.B;
  std::vector<int> bin_of(pr->M, -1), ints;
  for (int e = 0; e < B; ++e)
    if (bin_of[j0[e]] < 0) {
      bin_of[j0[e]] = (int)ints.size();
      ints.push_back(j0[e]);
    }
  const int BU = (int)ints.size();
  if (BU == B) return dfres ? df_born(pr, P, cx.r0, B, cx.b, dfw, s) : born(pr, P, cx, ws64, s);
  for (int e = 0; e < B; ++e) ints.push_back(bin_of[j0[e]]);  // [BU] bins, then [B] energy -> bin
  SolveCtx cu;
  cu.B = BU;
  cu.dim = cx.dim;
  cu.st = s;
  WPCD_CUDA_TRY(pool_malloc(&cu.b, 16 * cx.dim * BU, s));
  WPCD_CUDA_TRY(pool_malloc(&cu.r0, sizeof(int) * ints.size(), s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(cu.r0, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice, s));
  wpcd_status st = dfres ? df_born(pr, P, cu.r0, BU, cu.b, dfw, s) : born(pr, P, cu, ws64, s);
  if (st != WPCD_OK) return st;
  const int64_t n = (int64_t)cx.dim * B;
  expand_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, B, BU, cu.r0 + BU, reinterpret_cast<const double2 *>(cu.b),
                                                 reinterpret_cast<double2 *>(cx.b));
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "born expand launch");
}

// Plain FP64 Krylov on (I - K) u = b, started from u (0 or a warm start).
// A warm start whose residual is not below |b| is replaced by u = 0 for that
// energy (the plain iteration is the fallback).  conv[e] receives the number
// of Krylov steps after which energy e met the tolerance (checked every
// check_every steps; m + 1 if it never did).
wpcd_status solve_fp64(const wpcd_problem *pr, const wpcd_P *P, const wpcd_solve_opts &o, SolveCtx &cx,
                       Krylov<double> &kr, Workspace<double> &ws, std::vector<int> &status,
                       std::vector<double> &relres, std::vector<int> &conv, std::vector<int> &fallback,
                       int &n_apply, bool warm, cudaStream_t s) {
  const int B = cx.B, m = kr.m;
  const int64_t n = (int64_t)cx.dim * B;
  const int vg = grid_for(n, 256);
  n_apply = 0;
  fallback.assign(B, 0);
  if (warm) {  // r = b - (I - K) u
    wpcd_status st = kapply_ws<double>(pr, P, cx.g, cx.u, cx.t, nullptr, B, ws, s);
    if (st != WPCD_OK) return st;
    ++n_apply;
    bresid_kernel<<<vg, 256, 0, s>>>(n, (double2 *)cx.b, (double2 *)cx.u, (double2 *)cx.t, (double2 *)cx.r);
    count_launches(1);
  } else {
    WPCD_CUDA_TRY(cudaMemcpyAsync(cx.r, cx.b, 16 * n, cudaMemcpyDeviceToDevice, s));
    WPCD_CUDA_TRY(cudaMemsetAsync(cx.u, 0, 16 * n, s));
  }
  // |b| is the reference of the relative residual
  kr.norms<double>((const double2 *)cx.b, s);
  std::vector<double2> nb(B), nr(B);
  WPCD_CUDA_TRY(cudaMemcpyAsync(nb.data(), kr.nrm, sizeof(double2) * B, cudaMemcpyDeviceToHost, s));
  kr.norms<double>((const double2 *)cx.r, s);
  WPCD_CUDA_TRY(cudaMemcpyAsync(nr.data(), kr.nrm, sizeof(double2) * B, cudaMemcpyDeviceToHost, s));
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  if (warm) {
    bool any = false;
    for (int e = 0; e < B; ++e)
      if (!(nr[e].x < nb[e].x)) {  // not better than the zero start (also NaN)
        fallback[e] = 1;
        any = true;
      }
    if (any) {
      int *d_flag = nullptr;
      WPCD_CUDA_TRY(pool_malloc(&d_flag, sizeof(int) * B, s));
      WPCD_CUDA_TRY(cudaMemcpyAsync(d_flag, fallback.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
      bfallback_kernel<<<vg, 256, 0, s>>>(n, B, d_flag, (const double2 *)cx.b, (double2 *)cx.u, (double2 *)cx.r);
      count_launches(1);
      kr.norms<double>((const double2 *)cx.r, s);
      WPCD_CUDA_TRY(cudaMemcpyAsync(nr.data(), kr.nrm, sizeof(double2) * B, cudaMemcpyDeviceToHost, s));
      WPCD_CUDA_TRY(cudaStreamSynchronize(s));
      pool_free(d_flag, s);
    }
  }
  std::vector<double> bn(B);
  std::vector<double2> bet0((size_t)B * (m + 1), make_double2(0.0, 0.0));
  for (int e = 0; e < B; ++e) {
    bn[e] = std::sqrt(nb[e].x);
    if (!(bn[e] > 0.0)) return set_error(WPCD_EBREAKDOWN, "Born term is zero");
    bet0[(size_t)e * (m + 1)] = make_double2(std::sqrt(nr[e].x), 0.0);
  }
  // v0 = r / |r| ; bet = |r| e1
  kr.norms<double>((const double2 *)cx.r, s, true);  // inv = 1 / |r| for v0
  bscale_kernel<double><<<vg, 256, 0, s>>>(n, B, (const double2 *)cx.r, kr.inv, kr.vec(0));
  count_launches(1);
  WPCD_CUDA_TRY(cudaMemsetAsync(kr.H, 0, sizeof(double2) * (size_t)B * (m + 1) * m, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(kr.bet, bet0.data(), sizeof(double2) * bet0.size(), cudaMemcpyHostToDevice, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(kr.bnorm, bn.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s));
  status.assign(B, WPCD_ENOCONV);
  relres.assign(B, 1.0);
  conv.assign(B, m + 1);
  std::vector<double> res(B);
  bool done = true;
  for (int e = 0; e < B; ++e) {
    relres[e] = std::sqrt(nr[e].x) / bn[e];
    if (relres[e] <= o.tol) {
      status[e] = WPCD_OK;
      conv[e] = 0;
    } else {
      done = false;
    }
  }
  int k = 0;
  for (k = 0; k < m && !done; ++k) {
    // w = (I - K) v_k
    wpcd_status st = kapply_ws<double>(pr, P, cx.g, (double *)kr.vec(k), kr.w, (double *)kr.vec(k), B, ws, s);
    if (st != WPCD_OK) return st;
    ++n_apply;
    kr.step(k, s);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_error(ce, "krylov step launch");
    bool check = ((k + 1) % std::max(o.check_every, 1) == 0) || k + 1 == m;
    if (check) {
      WPCD_CUDA_TRY(cudaMemcpyAsync(res.data(), kr.resid, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
      WPCD_CUDA_TRY(cudaStreamSynchronize(s));
      done = true;
      for (int e = 0; e < B; ++e) {
        if (status[e] == WPCD_OK) continue;  // keeps its count and residual
        relres[e] = res[e];
        if (!std::isfinite(res[e])) {
          status[e] = WPCD_EBREAKDOWN;
        } else if (res[e] <= o.tol) {
          status[e] = WPCD_OK;
          conv[e] = k + 1;
        } else {
          done = false;
        }
      }
    }
  }
  bbacksub_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, m, k, kr.H, kr.bet, kr.y);
  bupdate_coef_kernel<double><<<std::max(1, (k * B + 255) / 256), 256, 0, s>>>(k, B, kr.y, nullptr, kr.hc);
  bupdate_kernel<double><<<vg, 256, 0, s>>>(n, B, k, kr.vec(0), cx.dim * B, kr.hc, (double2 *)cx.u);
  count_launches(3);
  return WPCD_OK;
}

// Mixed precision: FP64 refinement around FP32 inner Krylov cycles
// (dfw non-NULL: the FP64 K applications of the residual in float-float)
wpcd_status solve_mixed(const wpcd_problem *pr, const wpcd_P *P, const wpcd_solve_opts &o, SolveCtx &cx,
                        Krylov<float> &kr, Krylov<double> &k64, Workspace<double> &ws64,
                        Workspace<float> &ws32, DfWork *dfw, std::vector<int> &status, std::vector<double> &relres,
                        int &n64, int &n32, int &n_outer, bool warm, cudaStream_t s) {
  const int B = cx.B, m = kr.m;
  const int64_t n = (int64_t)cx.dim * B;
  const int vg = grid_for(n, 256);
  n64 = n32 = n_outer = 0;
  if (!warm) WPCD_CUDA_TRY(cudaMemsetAsync(cx.u, 0, 16 * n, s));
  // |b|
  k64.norms<double>((const double2 *)cx.b, s);
  std::vector<double2> nb(B);
  WPCD_CUDA_TRY(cudaMemcpyAsync(nb.data(), k64.nrm, sizeof(double2) * B, cudaMemcpyDeviceToHost, s));
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<double> bn(B);
  for (int e = 0; e < B; ++e) {
    bn[e] = std::sqrt(nb[e].x);
    if (!(bn[e] > 0.0)) return set_error(WPCD_EBREAKDOWN, "Born term is zero");
  }
  // inner right-hand sides are normalised: bet = e1, reference norm 1
  std::vector<double> ones(B, 1.0);
  std::vector<double2> bet0((size_t)B * (m + 1), make_double2(0.0, 0.0));
  for (int e = 0; e < B; ++e) bet0[(size_t)e * (m + 1)] = make_double2(1.0, 0.0);
  double2 *d_bet0 = nullptr;
  WPCD_CUDA_TRY(pool_malloc(&d_bet0, sizeof(double2) * bet0.size(), s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(kr.bnorm, ones.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(d_bet0, bet0.data(), sizeof(double2) * bet0.size(), cudaMemcpyHostToDevice, s));
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));  // host staging vectors

  // the inner cycle of mm <= m steps: fixed sizes and pointers, so the full
  // m-step cycle can be captured once and replayed as a CUDA graph
  auto inner_cycle = [&](int mm) -> wpcd_status {
    cudaMemsetAsync(kr.H, 0, sizeof(double2) * (size_t)B * (m + 1) * m, s);
    cudaMemcpyAsync(kr.bet, d_bet0, sizeof(double2) * bet0.size(), cudaMemcpyDeviceToDevice, s);
    for (int k = 0; k < mm; ++k) {
      wpcd_status st = kapply_ws<float>(pr, P, cx.g32, (float *)kr.vec(k), kr.w, (float *)kr.vec(k), B, ws32, s);
      if (st != WPCD_OK) return st;
      // single-pass Gram-Schmidt: the short FP32 cycle only has to cut the
      // residual, whose FP64 value the refinement loop recomputes and judges
      kr.step(k, s, false);
    }
    bbacksub_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, m, mm, kr.H, kr.bet, kr.y);
    // u += |r| (V y)   (FP64 accumulation of the FP32 correction)
    bupdate_coef_kernel<float><<<(mm * B + 255) / 256, 256, 0, s>>>(mm, B, kr.y, k64.nrm, kr.hc);
    if (B % 2 == 0)
      bupdate2_kernel<<<grid_for(n / 2, 256), 256, 0, s>>>(n / 2, B / 2, mm, reinterpret_cast<const float4 *>(kr.vec(0)),
                                                           cx.dim * B / 2, reinterpret_cast<const float4 *>(kr.hc),
                                                           (double2 *)cx.u);
    else
      bupdate_kernel<float><<<vg, 256, 0, s>>>(n, B, mm, kr.vec(0), cx.dim * B, kr.hc, (double2 *)cx.u);
    count_launches(3);
    return WPCD_OK;
  };
  // the SpMM shapes are tuned before any capture (tuning synchronises)
  {
    SpmmConfig c;
    wpcd_status st = tune_spmm(pr, const_cast<wpcd_P *>(P), B, 1, s, &c);
    // a row-tiled choice (possibly from the tuning cache) builds its tile
    // structure here, outside the capture
    if (st == WPCD_OK && c.tile)
      st = tile_prepare(pr, const_cast<wpcd_P *>(P), P->val32 ? P->val32 : P->val32_copy, c.tile, s);
    if (st == WPCD_OK) st = tune_spmm(pr, const_cast<wpcd_P *>(P), B, 0, s, &c);
    if (st != WPCD_OK) {
      pool_free(d_bet0, s);
      return st;
    }
  }
  cudaGraphExec_t exec = nullptr;
  int64_t launches0 = 0;
  int graph_kernels = 0;
  status.assign(B, WPCD_ENOCONV);
  relres.assign(B, 1.0);
  std::vector<double2> nr(B);
  const int max_outer = o.max_outer > 0 ? o.max_outer : 12;
  wpcd_status result = WPCD_OK;
  // cycle lengths after the first from the previous cycle's reduction of the
  // worst residual (next_cycle_steps): a cycle that falls just short then
  // costs a few steps, not another m
  double worst_prev = 0.0;
  int mm_prev = 0;
  for (int outer = 0; outer <= max_outer; ++outer) {
    // r = b - (I - K) u in FP64
    if (outer > 0 || warm) {
      wpcd_status st = dfw ? df_kapply(pr, P, cx.g, cx.u, cx.t, B, *dfw, s)
                           : kapply_ws<double>(pr, P, cx.g, cx.u, cx.t, nullptr, B, ws64, s);
      if (st != WPCD_OK) {
        result = st;
        break;
      }
      ++n64;
      bresid_kernel<<<vg, 256, 0, s>>>(n, (double2 *)cx.b, (double2 *)cx.u, (double2 *)cx.t, (double2 *)cx.r);
      count_launches(1);
    } else {
      cudaMemcpyAsync(cx.r, cx.b, 16 * n, cudaMemcpyDeviceToDevice, s);
    }
    k64.norms<double>((const double2 *)cx.r, s, true);  // |r|^2 and 1 / |r|
    cudaMemcpyAsync(nr.data(), k64.nrm, sizeof(double2) * B, cudaMemcpyDeviceToHost, s);
    cudaError_t ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
      result = cuda_error(ce, "refinement residual");
      break;
    }
    bool done = true;
    double worst = 0.0;
    for (int e = 0; e < B; ++e) {
      relres[e] = std::sqrt(nr[e].x) / bn[e];
      if (!std::isfinite(relres[e])) {
        status[e] = WPCD_EBREAKDOWN;
      } else if (relres[e] <= o.tol) {
        status[e] = WPCD_OK;
      } else {
        status[e] = WPCD_ENOCONV;
        done = false;
        worst = std::max(worst, relres[e]);
      }
    }
    if (done || outer == max_outer) break;
    ++n_outer;
    const int mm = next_cycle_steps(worst, worst_prev, mm_prev, m, o.tol);
    worst_prev = worst;
    mm_prev = mm;
    // v0 = (float)(r / |r|)
    bnormalize_f32_kernel<<<vg, 256, 0, s>>>(n, B, (const double2 *)cx.r, k64.inv, kr.vec(0));
    count_launches(1);
    if (o.use_graph && s != nullptr && mm == m) {  // the legacy default stream cannot be captured
      if (!exec) {
        cudaGraph_t graph;
        launches0 = wpcd_launch_count();
        ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) {
          result = cuda_error(ce, "begin capture");
          break;
        }
        wpcd_status st = inner_cycle(m);
        ce = cudaStreamEndCapture(s, &graph);
        if (st != WPCD_OK) {
          result = st;
          break;
        }
        if (ce != cudaSuccess) {
          result = cuda_error(ce, "end capture");
          break;
        }
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
          result = cuda_error(ce, "graph instantiate");
          break;
        }
        // captured kernels run at each replay, not at capture
        graph_kernels = (int)(wpcd_launch_count() - launches0);
        count_launches(-graph_kernels);
      }
      ce = cudaGraphLaunch(exec, s);
      if (ce != cudaSuccess) {
        result = cuda_error(ce, "graph launch");
        break;
      }
      count_launches(graph_kernels);
    } else {
      wpcd_status st = inner_cycle(mm);
      if (st != WPCD_OK) {
        result = st;
        break;
      }
    }
    n32 += mm;
  }
  if (exec) cudaGraphExecDestroy(exec);
  pool_free(d_bet0, s);
  return result;
}

// Paper's route, one energy: x_{n+1} = K x_n from the Born term, c_n =
// x_n[r0], Wynn epsilon on the device.
wpcd_status solve_wynn(const wpcd_problem *pr, const wpcd_P *P, double E, const wpcd_solve_opts &o,
                       wpcd_solve_stats &out, cudaStream_t s) {
  const size_t dim = (size_t)pr->n_ch * pr->N * pr->M;
  const int m = o.max_iter;
  int j0;
  double Elo, Ehi, q0;
  wpcd_status st = onshell(pr, E, &j0, &Elo, &Ehi, &q0);
  if (st != WPCD_OK) return st;
  double D = Ehi - Elo;
  Workspace<double> ws;
  WPCD_CUDA_TRY(ws.alloc(dim, 1, s));
  struct Free {
    std::vector<void *> p;
    ~Free() {
      for (void *q : p) dev_free(q);
    }
  } fr;
  double *g = nullptr, *x0d = nullptr, *x1d = nullptr;
  double2 *small = nullptr;
  int *flag = nullptr;
  WPCD_CUDA_TRY(dev_malloc(&g, 16 * dim));
  fr.p.push_back(g);
  WPCD_CUDA_TRY(dev_malloc(&x0d, 16 * dim));
  fr.p.push_back(x0d);
  WPCD_CUDA_TRY(dev_malloc(&x1d, 16 * dim));
  fr.p.push_back(x1d);
  WPCD_CUDA_TRY(dev_malloc(&small, sizeof(double2) * (5 * (size_t)m + 8)));
  fr.p.push_back(small);
  WPCD_CUDA_TRY(dev_malloc(&flag, 2 * sizeof(int)));
  fr.p.push_back(flag);
  st = resolvent_impl(pr, &E, 1, g, 1, nullptr, nullptr, s);
  if (st != WPCD_OK) return st;
  double2 *c = small, *est = c + m, *work = est + m;  // work: 3 (m + 1)
  double2 *x0 = reinterpret_cast<double2 *>(x0d), *x1 = reinterpret_cast<double2 *>(x1d);
  int *r0d = flag + 1;
  cudaEvent_t e0, e1;
  WPCD_CUDA_TRY(cudaEventCreate(&e0));
  WPCD_CUDA_TRY(cudaEventCreate(&e1));
  cudaEventRecord(e0, s);
  WPCD_CUDA_TRY(cudaMemcpyAsync(r0d, &j0, sizeof(int), cudaMemcpyHostToDevice, s));
  bunits_kernel<<<grid_for((int64_t)dim, 256), 256, 0, s>>>((int64_t)dim, 1, r0d, x1);
  count_launches(1);
  st = kapply_ws<double>(pr, P, nullptr, x1d, x0d, nullptr, 1, ws, s);  // x0 = Born
  if (st != WPCD_OK) return st;
  std::vector<double2> est_h(m);
  int n = 0, status = WPCD_ENOCONV, bd = 0, checked = 0, used = 0;
  double best_d = INFINITY;
  double2 best = make_double2(0.0, 0.0), last = make_double2(0.0, 0.0);
  int best_n = 0;
  const int every = o.check_every > 0 ? o.check_every : 1;
  for (n = 0; n < m; ++n) {
    extract_kernel<<<1, 1, 0, s>>>(x0, j0, c + n);
    wynn_kernel<<<1, 1, 0, s>>>(n + 1, c, work, est, flag);
    count_launches(2);
    if (n + 1 < m) {
      st = kapply_ws<double>(pr, P, g, reinterpret_cast<double *>(x0), reinterpret_cast<double *>(x1), nullptr, 1,
                             ws, s);
      if (st != WPCD_OK) return st;
      std::swap(x0, x1);
    }
    if ((n + 1) % every != 0 && n + 1 != m) continue;
    WPCD_CUDA_TRY(cudaMemcpyAsync(est_h.data(), est, sizeof(double2) * (n + 1), cudaMemcpyDeviceToHost, s));
    WPCD_CUDA_TRY(cudaMemcpyAsync(&bd, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    WPCD_CUDA_TRY(cudaStreamSynchronize(s));
    bool done = false;
    for (int t = checked; t <= n; ++t) {
      double2 ev = est_h[t];
      used = t + 1;
      if (t > 0) {
        double2 p = est_h[t - 1];
        double d = std::hypot(ev.x - p.x, ev.y - p.y) / std::hypot(ev.x, ev.y);
        if (t + 1 >= o.min_iter && d <= o.tol) {
          best = ev;
          status = WPCD_OK;
          done = true;
          break;
        }
        if (d < best_d) {
          best_d = d;
          best = ev;
          best_n = t + 1;
        }
      }
      last = ev;
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
  out.n_kapply32 = 0;
  out.n_outer = 0;
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

wpcd_status born_vectors(wpcd_problem *pr, const wpcd_P *P, const double *E, int n_E, double *b_major,
                         cudaStream_t s) {
  if (n_E < 1 || !E || !b_major) return set_error(WPCD_EINVAL, "bad Born arguments");
  const size_t dim = (size_t)pr->n_ch * pr->N * pr->M;
  std::vector<int> j0(n_E);
  for (int e = 0; e < n_E; ++e) {
    double lo, hi;
    wpcd_status st = onshell(pr, E[e], &j0[e], &lo, &hi, nullptr);
    if (st != WPCD_OK) return st;
  }
  WPCD_CUDA_TRY(cudaSetDevice(pr->device));
  SolveCtx cx;
  cx.B = n_E;
  cx.dim = dim;
  cx.st = s;
  WPCD_CUDA_TRY(pool_malloc(&cx.b, 16 * dim * n_E, s));
  WPCD_CUDA_TRY(pool_malloc(&cx.t, 16 * dim * n_E, s));
  WPCD_CUDA_TRY(pool_malloc(&cx.r0, sizeof(int) * n_E, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(cx.r0, j0.data(), sizeof(int) * n_E, cudaMemcpyHostToDevice, s));
  Workspace<double> ws;
  WPCD_CUDA_TRY(ws.alloc(dim, n_E, s));
  wpcd_status st = born(pr, P, cx, ws, s);
  if (st != WPCD_OK) return st;
  const int64_t n = (int64_t)dim * n_E;
  transpose_kernel<<<grid_for(n, 256), 256, 0, s>>>((int64_t)dim, n_E, (const double2 *)cx.b, (double2 *)b_major, 0);
  count_launches(1);
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  return WPCD_OK;
}

wpcd_status solve(wpcd_problem *pr, const wpcd_P *Pc, const double *E, int n_E,
                  const wpcd_solve_opts *o, double *U00, wpcd_solve_stats *st_out, cudaStream_t s) {
  wpcd_solve_opts opt{};
  opt.method = WPCD_SUM_KRYLOV;
  opt.max_iter = 100;
  opt.min_iter = 4;
  opt.tol = 1e-10;
  opt.check_every = 4;
  opt.precision = WPCD_SOLVE_FP64;
  opt.use_graph = 1;
  if (o) opt = *o;
  wpcd_P *P = const_cast<wpcd_P *>(Pc);
  if (opt.max_iter < 2 || opt.max_iter > 512) return set_error(WPCD_EINVAL, "max_iter must be in [2, 512]");
  if (!(opt.tol > 0.0)) return set_error(WPCD_EINVAL, "tol must be positive");
  if (opt.method != WPCD_SUM_KRYLOV && opt.method != WPCD_SUM_WYNN) return set_error(WPCD_EINVAL, "unknown method");
  if (opt.precision != WPCD_SOLVE_FP64 && opt.precision != WPCD_SOLVE_MIXED &&
      opt.precision != WPCD_SOLVE_MIXED_FP64)
    return set_error(WPCD_EINVAL, "unknown precision");
  if (opt.method == WPCD_SUM_WYNN && opt.precision != WPCD_SOLVE_FP64)
    return set_error(WPCD_EINVAL, "the Wynn summation runs in FP64 only");
  if (opt.method == WPCD_SUM_WYNN && (opt.u_init || opt.u_out))
    return set_error(WPCD_EINVAL, "the Wynn summation takes no vectors");
  if (opt.batch < 0 || opt.batch > 1024) return set_error(WPCD_EINVAL, "batch must be in [0, 1024]");
  if (opt.inner_iter < 0 || opt.inner_iter > 128) return set_error(WPCD_EINVAL, "inner_iter must be in [0, 128]");
  if (n_E < 0 || (n_E > 0 && (!E || !U00))) return set_error(WPCD_EINVAL, "bad energies / output");
  for (int e = 0; e < n_E; ++e) {
    int j0;
    double lo, hi;
    wpcd_status st = onshell(pr, E[e], &j0, &lo, &hi, nullptr);
    if (st != WPCD_OK) return st;
  }
  WPCD_CUDA_TRY(cudaSetDevice(pr->device));
  if (n_E == 0) return WPCD_OK;
  if (wpcd_status st = tc_clear(pr, s); st != WPCD_OK) return st;
  wpcd_status worst = WPCD_OK;
  if (opt.method == WPCD_SUM_WYNN) {
    for (int e = 0; e < n_E; ++e) {
      wpcd_solve_stats one{};
      wpcd_status st = solve_wynn(pr, P, E[e], opt, one, s);
      if (st != WPCD_OK) return st;
      U00[2 * e] = one.U00[0];
      U00[2 * e + 1] = one.U00[1];
      if (st_out) st_out[e] = one;
      if (one.status < worst) worst = one.status;
    }
  } else {
    const bool mixed = opt.precision != WPCD_SOLVE_FP64;
    const bool dfres = opt.precision == WPCD_SOLVE_MIXED;  // float-float residual
    if (dfres) {
      wpcd_status st = df_prepare(pr, P, s);
      if (st != WPCD_OK) return st;
    }
    const int Bmax = opt.batch > 0 ? std::min(opt.batch, n_E) : n_E;
    const size_t dim = (size_t)pr->n_ch * pr->N * pr->M;
    if (mixed && tc_enabled() && tc_supported(pr)) {
      wpcd_status st = tc_prepare(pr, s);
      if (st != WPCD_OK) return st;
    }
    if (mixed && !P->val32 && !P->val32_copy) {
      WPCD_CUDA_TRY(dev_malloc(&P->val32_copy, sizeof(float) * (size_t)P->nnz * P->n_pairs + 4));
      int64_t nv = (int64_t)P->nnz * P->n_pairs;
      d2f_kernel<<<grid_for(nv, 256), 256, 0, s>>>(nv, P->val64, P->val32_copy);
      count_launches(1);
    }
    for (int e0 = 0; e0 < n_E; e0 += Bmax) {
      const int B = std::min(Bmax, n_E - e0);
      SolveCtx cx;
      cx.B = B;
      cx.dim = dim;
      cx.st = s;
      const size_t nb = 16 * dim * B;
      WPCD_CUDA_TRY(pool_malloc(&cx.g, nb, s));
      if (mixed) WPCD_CUDA_TRY(pool_malloc(&cx.g32, nb / 2, s));
      WPCD_CUDA_TRY(pool_malloc(&cx.b, nb, s));
      WPCD_CUDA_TRY(pool_malloc(&cx.u, nb, s));
      WPCD_CUDA_TRY(pool_malloc(&cx.r, nb, s));
      WPCD_CUDA_TRY(pool_malloc(&cx.t, nb, s));
      WPCD_CUDA_TRY(pool_malloc(&cx.r0, sizeof(int) * B, s));
      WPCD_CUDA_TRY(pool_malloc(&cx.Dd, sizeof(double) * B, s));
      WPCD_CUDA_TRY(pool_malloc(&cx.pref, sizeof(double) * B, s));
      WPCD_CUDA_TRY(pool_malloc(&cx.amp, sizeof(double) * 6 * B, s));
      BatchInfo bi;
      cudaEvent_t ev0, ev1;
      WPCD_CUDA_TRY(cudaEventCreate(&ev0));
      WPCD_CUDA_TRY(cudaEventCreate(&ev1));
      cudaEventRecord(ev0, s);
      wpcd_status st = batch_setup(pr, E + e0, B, cx, bi, s);
      if (st != WPCD_OK) return st;
      Workspace<double> ws64;
      WPCD_CUDA_TRY(ws64.alloc(dim, B, s));
      DfWork dfw;
      if (dfres) WPCD_CUDA_TRY(dfw.alloc(dim, B, s));
      // Born term on s, resolvent concurrently on a side stream
      struct Side {
        cudaStream_t s2 = nullptr;
        cudaEvent_t before = nullptr, after = nullptr;
        ~Side() {
          if (before) cudaEventDestroy(before);
          if (after) cudaEventDestroy(after);
          if (s2) cudaStreamDestroy(s2);
        }
      } side;
      WPCD_CUDA_TRY(cudaStreamCreateWithFlags(&side.s2, cudaStreamNonBlocking));
      WPCD_CUDA_TRY(cudaEventCreateWithFlags(&side.before, cudaEventDisableTiming));
      WPCD_CUDA_TRY(cudaEventCreateWithFlags(&side.after, cudaEventDisableTiming));
      WPCD_CUDA_TRY(cudaEventRecord(side.before, s));
      st = batch_born(pr, P, cx, bi.j0, dfres, ws64, dfw, s);
      if (st != WPCD_OK) return st;
      st = batch_resolvent(pr, E + e0, B, cx, mixed, s, side.s2, side.before, side.after);
      if (st != WPCD_OK) return st;
      const bool warm = opt.u_init != nullptr;
      const int64_t n = (int64_t)dim * B;
      if (warm) {
        transpose_kernel<<<grid_for(n, 256), 256, 0, s>>>((int64_t)dim, B,
                                                          (const double2 *)opt.u_init + (size_t)e0 * dim,
                                                          (double2 *)cx.u, 1);
        count_launches(1);
      }
      std::vector<int> status, conv, fallback;
      std::vector<double> relres;
      int n64 = 0, n32 = 0, n_outer = 0;
      if (mixed) {
        const int m_in = opt.inner_iter > 0 ? opt.inner_iter : kDefaultInner;
        Krylov<float> kr;
        Krylov<double> k64;
        WPCD_CUDA_TRY(kr.alloc(m_in, B, dim, s));
        WPCD_CUDA_TRY(k64.alloc(1, B, dim, s, false));  // norms only
        Workspace<float> ws32;
        WPCD_CUDA_TRY(ws32.alloc(dim, B, s));
        st = solve_mixed(pr, P, opt, cx, kr, k64, ws64, ws32, dfres ? &dfw : nullptr, status, relres, n64, n32,
                         n_outer, warm, s);
      } else {
        Krylov<double> kr;
        WPCD_CUDA_TRY(kr.alloc(opt.max_iter, B, dim, s));
        st = solve_fp64(pr, P, opt, cx, kr, ws64, status, relres, conv, fallback, n64, warm, s);
      }
      if (st != WPCD_OK) return st;
      n64 += 1;  // the Born term
      bamplitude_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, (const double2 *)cx.u, cx.r0, cx.Dd, cx.pref, cx.amp);
      count_launches(1);
      if (opt.u_out) {
        transpose_kernel<<<grid_for(n, 256), 256, 0, s>>>((int64_t)dim, B, (const double2 *)cx.u,
                                                          (double2 *)opt.u_out + (size_t)e0 * dim, 0);
        count_launches(1);
      }
      cudaEventRecord(ev1, s);
      std::vector<double> amp(6 * (size_t)B);
      WPCD_CUDA_TRY(cudaMemcpyAsync(amp.data(), cx.amp, sizeof(double) * 6 * B, cudaMemcpyDeviceToHost, s));
      WPCD_CUDA_TRY(cudaStreamSynchronize(s));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev0, ev1);
      cudaEventDestroy(ev0);
      cudaEventDestroy(ev1);
      for (int e = 0; e < B; ++e) {
        U00[2 * (e0 + e)] = amp[6 * e];
        U00[2 * (e0 + e) + 1] = amp[6 * e + 1];
        if (st_out) {
          wpcd_solve_stats &so = st_out[e0 + e];
          so.status = status[e];
          // FP64 K applications: the batch's total, or for the plain solve
          // this energy's own count to convergence (+ Born, + warm residual)
          so.n_kapply = conv.empty() ? n64 : std::min(conv[e], n64) + 1 + (warm ? 1 : 0);
          so.warm_fallback = fallback.empty() ? 0 : fallback[e];
          so.n_kapply32 = n32;
          so.n_outer = n_outer;
          so.j0 = bi.j0[e];
          so.D = bi.D[e];
          so.relres = relres[e];
          for (int i = 0; i < 2; ++i) {
            so.U00[i] = amp[6 * e + i];
            so.S[i] = amp[6 * e + 2 + i];
            so.A[i] = amp[6 * e + 4 + i];
          }
          so.ms = ms / B;
        }
        if (status[e] < worst) worst = status[e];
      }
    }
  }
  {
    wpcd_status st = tc_check(pr, s);
    if (st != WPCD_OK) return st;
  }
  if (worst != WPCD_OK)
    set_error(worst, worst == WPCD_ENOCONV ? "summation did not reach the tolerance for some energy"
                                           : "Pade/Krylov breakdown for some energy");
  return worst;
}

// z = P0 y for n_rhs vectors (the sparse step of the K application)
wpcd_status spmm_apply(wpcd_problem *pr, wpcd_P *P, int mode, const void *y, void *z, int n_rhs, float *ms,
                       cudaStream_t s) {
  if (!y || !z || y == z || n_rhs < 1) return set_error(WPCD_EINVAL, "bad vectors or n_rhs");
  if (mode < WPCD_SPMM_FP64 || mode > WPCD_SPMM_FP32_BLOCKED) return set_error(WPCD_EINVAL, "unknown SpMM mode");
  WPCD_CUDA_TRY(cudaSetDevice(pr->device));
  if (mode == WPCD_SPMM_FF) return df_spmm_op(pr, P, (const double *)y, (double *)z, n_rhs, ms, s);
  const bool fp32 = mode == WPCD_SPMM_FP32 || mode == WPCD_SPMM_FP32_BLOCKED;
  if (fp32 && !P->val32 && !P->val32_copy) {
    WPCD_CUDA_TRY(dev_malloc(&P->val32_copy, sizeof(float) * (size_t)P->nnz * P->n_pairs + 4));
    const int64_t nv = (int64_t)P->nnz * P->n_pairs;
    d2f_kernel<<<grid_for(nv, 256), 256, 0, s>>>(nv, P->val64, P->val32_copy);
    count_launches(1);
  }
  if (mode == WPCD_SPMM_FP32_BLOCKED) {  // the row-tiled kernel, 2 x 2 tiles (built before the timed launch)
    if (!tile_supported(pr, n_rhs)) return set_error(WPCD_EINVAL, "tiled SpMM: even n_rhs and up to three channels");
    const float *v32 = P->val32 ? P->val32 : P->val32_copy;
    const SpmmConfig cfg{1, 32, 2, 4};
    wpcd_status st = launch_spmm_tile(pr, P, v32, (const float *)y, (float *)z, n_rhs, cfg, s);
    if (st != WPCD_OK) return st;
    LaunchTimer t(ms, s);
    t.start();
    st = launch_spmm_tile(pr, P, v32, (const float *)y, (float *)z, n_rhs, cfg, s);
    t.stop();
    return st;
  }
  SpmmConfig cfg;  // tune (which synchronises) before any timed launch
  wpcd_status st = tune_spmm(pr, P, n_rhs, fp32 ? 1 : 0, s, &cfg);
  if (st == WPCD_OK && cfg.tile) st = tile_prepare(pr, P, P->val32 ? P->val32 : P->val32_copy, cfg.tile, s);
  if (st != WPCD_OK) return st;
  LaunchTimer t(ms, s);
  t.start();
  st = fp32 ? spmm<float>(pr, P, (const float *)y, (float *)z, n_rhs, s)
            : spmm<double>(pr, P, (const double *)y, (double *)z, n_rhs, s);
  t.stop();
  return st;
}

// one channel-block product Y = A (G1 o X) of the K application
wpcd_status channel_gemm(wpcd_problem *pr, int which, int mode, const void *g, const void *x, void *y, int n_rhs,
                         float *ms, cudaStream_t s) {
  if (which != 0 && which != 1) return set_error(WPCD_EINVAL, "which must be 0 (Vt) or 1 (O)");
  if (!x || !y || x == y || n_rhs < 1) return set_error(WPCD_EINVAL, "bad vectors or n_rhs");
  WPCD_CUDA_TRY(cudaSetDevice(pr->device));
  const int N = pr->N;
  const int64_t ncol = 2LL * pr->M * n_rhs;
  dim3 grid((unsigned)((ncol + GB_N - 1) / GB_N), (N + GB_M - 1) / GB_M, pr->n_ch);
  if (mode == WPCD_GEMM_FF || mode == WPCD_GEMM_DIGITS)
    return df_gemm_op(pr, which == 1, mode == WPCD_GEMM_DIGITS, (const double *)g, (const double *)x, (double *)y,
                      n_rhs, ms, s);
  if (mode == WPCD_GEMM_TF32X3) {
    if (!tc_supported(pr)) return set_error(WPCD_EINVAL, "the tensor-core GEMM needs N <= 512");
    wpcd_status st = tc_prepare(pr, s);
    if (st == WPCD_OK) st = tc_clear(pr, s);
    if (st != WPCD_OK) return st;
    {
      LaunchTimer t(ms, s);
      t.start();
      st = tc_gemm(pr, which == 1, (const float *)g, (const float *)x, nullptr, (float *)y, ncol, s);
      t.stop();
    }
    if (st != WPCD_OK) return st;
    return tc_check(pr, s);
  }
  if (mode != WPCD_GEMM_FP64 && mode != WPCD_GEMM_FP32) return set_error(WPCD_EINVAL, "unknown GEMM mode");
  {
    LaunchTimer t(ms, s);
    t.start();
    if (mode == WPCD_GEMM_FP64) {
      const double *A = which ? pr->d.O : pr->d.Vt;
      if (g)
        gemm_kernel<double, true, false><<<grid, G_THREADS, 0, s>>>(N, ncol, A, (const double *)x,
                                                                    (const double *)g, nullptr, (double *)y);
      else
        gemm_kernel<double, false, false><<<grid, G_THREADS, 0, s>>>(N, ncol, A, (const double *)x, nullptr,
                                                                     nullptr, (double *)y);
    } else {
      const float *A = which ? pr->d.O32 : pr->d.Vt32;
      if (g)
        gemm_kernel<float, true, false><<<grid, G_THREADS, 0, s>>>(N, ncol, A, (const float *)x, (const float *)g,
                                                                   nullptr, (float *)y);
      else
        gemm_kernel<float, false, false><<<grid, G_THREADS, 0, s>>>(N, ncol, A, (const float *)x, nullptr,
                                                                    nullptr, (float *)y);
    }
    t.stop();
  }
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "channel gemm launch");
}

}  // namespace wpcd
