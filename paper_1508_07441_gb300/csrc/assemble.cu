// Step 2 of the numerical scheme (Sec. 3.3; Sec. 4.2): the lattice
// permutation matrix P0 of Eq. perm / Eq. gal, assembled on the device by
// quadrature-node binning, in two passes with no atomics.
//
//   count pass  one CTA per source cell c = (i, j).  Every GL node (a, b, x)
//               of the cell is mapped through the recoupled momenta
//                 p'^2 = fma((0.75 p) q, y, (p p) 0.25 + (q q) 0.5625)
//                 q'^2 = fma(-(p q),     y, (p p) + (q q) 0.25)
//               (FP64, each product rounded on its own) and binned by a
//               branch-free binary search over the squared edges held in
//               shared memory (compared as int64 bit patterns: the order of
//               non-negative doubles).  The packed keys (target << nb | node)
//               are sorted in shared memory (bitonic network), the distinct
//               targets counted (the paper's pre-selection), and the sorted
//               keys kept in global memory for the fill pass.
//   scan        exclusive scan of the counts -> row_ptr.
//   fill pass   one CTA per source cell.  The sorted keys are re-read; each
//               node's value w p^2 q^2 P_l(y) P_l'(y') is formed for every
//               (l, l') pair and summed per target by a block-wide segmented
//               scan (warp shuffles + a cross-warp carry), then normalised by
//               sqrt((2l+1)(2l'+1)) / sqrt(B_i Bq_j B_i' Bq_j') and written
//               to block-CSR (pair-major values).
//
// FP64 mode computes y' and the node values in FP64.  FP32C mode computes
// them in FP32 and accumulates with error-free transformations (TwoSum
// float-float pairs); only the binning uses FP64.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "wpcd_internal.h"

namespace wpcd {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kInvalid = 0xFFFFFFFFu;

struct AsmParams {
  int N, M, n_p, n_q, n_x, n_nodes, np2, nbits, n_ch, n_pairs;
  int pl[kMaxPairs], plp[kMaxPairs];
  double cnorm[kMaxPairs];  // sqrt((2l+1)(2l'+1))
  const double *pe2, *qe2, *pn, *wp, *qn, *wq, *yn, *wy, *rsb;
};

__device__ __forceinline__ int bin_search(const long long *e2, int n, long long x) {
  // number of interior squared edges e2[1..n-1] that are <= x
  int lo = 0;
  int step = 1;
  while (step * 2 <= n - 1) step *= 2;
  for (; step >= 1; step >>= 1) {
    int cand = lo + step;
    lo = (cand <= n - 1 && e2[cand] <= x) ? cand : lo;
  }
  return lo;
}

// p'^2 = A y + Bp and q'^2 = C y + D for one (p, q) node pair
struct BinConst {
  double A, Bp, C, D;
};

// Bitonic sort of n = E * blockDim.x keys (ascending) with the keys held in
// registers: thread t owns s[t E .. t E + E - 1].  A compare-exchange at
// distance j runs inside the thread for j < E, between lanes of a warp
// (shuffles) for j < 32 E, and through shared memory only beyond that.
template <int E>
__device__ void bitonic_sort_reg(uint32_t *s, int n) {
  const int t = threadIdx.x;
  uint32_t v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = s[t * E + e];
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j >= E; j >>= 1) {
      if (j < 32 * E) {
        const int d = j / E;  // partner lane distance
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const uint32_t p = __shfl_xor_sync(0xffffffffu, v[e], d);
          const int i = t * E + e;
          const bool keep_min = ((i & j) == 0) == ((i & k) == 0);
          v[e] = keep_min ? min(v[e], p) : max(v[e], p);
        }
      } else {
        __syncthreads();  // the previous exchange has been read
#pragma unroll
        for (int e = 0; e < E; ++e) s[t * E + e] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = t * E + e;
          const uint32_t p = s[i ^ j];
          const bool keep_min = ((i & j) == 0) == ((i & k) == 0);
          v[e] = keep_min ? min(v[e], p) : max(v[e], p);
        }
      }
    }
#pragma unroll
    for (int jj = E / 2; jj >= 1; jj >>= 1) {
      if (jj < k) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int f = e ^ jj;
          if (f > e) {
            const bool up = ((t * E + e) & k) == 0;
            const uint32_t a = v[e], b = v[f];
            if ((a > b) == up) {
              v[e] = b;
              v[f] = a;
            }
          }
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) s[t * E + e] = v[e];
  __syncthreads();
}

// shared-memory bitonic sort for any power-of-two n (used below 256 keys)
template <int NT>
__device__ void bitonic_sort(uint32_t *s, int n) {
  // n is a power of two; ascending
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < n / 2; t += NT) {
        int i = 2 * j * (t / j) + (t % j);
        int l = i + j;
        uint32_t a = s[i], b = s[l];
        bool up = (i & k) == 0;
        if ((a > b) == up) {
          s[i] = b;
          s[l] = a;
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kThreads) count_kernel(AsmParams P, int64_t *counts,
                                                         uint32_t *sorted) {
  extern __shared__ __align__(16) unsigned char smem[];
  long long *pe2 = reinterpret_cast<long long *>(smem);
  long long *qe2 = pe2 + (P.N + 1);
  BinConst *abk = reinterpret_cast<BinConst *>(qe2 + (P.M + 1));  // per (a, b)
  double *ys = reinterpret_cast<double *>(abk + P.n_p * P.n_q);
  uint32_t *keys = reinterpret_cast<uint32_t *>(ys + P.n_x);
  __shared__ int red[kThreads / 32];

  const int c = blockIdx.x;
  const int i = c / P.M, j = c % P.M;
  for (int k = threadIdx.x; k <= P.N; k += kThreads) pe2[k] = __double_as_longlong(P.pe2[k]);
  for (int k = threadIdx.x; k <= P.M; k += kThreads) qe2[k] = __double_as_longlong(P.qe2[k]);
  for (int ab = threadIdx.x; ab < P.n_p * P.n_q; ab += kThreads) {
    int a = ab / P.n_q, b = ab % P.n_q;
    double p = P.pn[i * P.n_p + a], q = P.qn[j * P.n_q + b];
    // canonical rounding order of the recoupled squares (no contraction)
    double A = __dmul_rn(__dmul_rn(0.75, p), q);
    double Bp = __dadd_rn(__dmul_rn(__dmul_rn(p, p), 0.25), __dmul_rn(__dmul_rn(q, q), 0.5625));
    double C = -__dmul_rn(p, q);
    double D = __dadd_rn(__dmul_rn(p, p), __dmul_rn(__dmul_rn(q, q), 0.25));
    abk[ab] = BinConst{A, Bp, C, D};
  }
  for (int x = threadIdx.x; x < P.n_x; x += kThreads) ys[x] = P.yn[x];
  __syncthreads();
  const long long pmax2 = pe2[P.N], qmax2 = qe2[P.M];
  for (int n = threadIdx.x; n < P.np2; n += kThreads) {
    uint32_t key = kInvalid;
    if (n < P.n_nodes) {
      const BinConst k = abk[n / P.n_x];
      const double y = ys[n % P.n_x];
      long long ip2 = __double_as_longlong(__fma_rn(k.A, y, k.Bp));
      long long iq2 = __double_as_longlong(__fma_rn(k.C, y, k.D));
      if (ip2 <= pmax2 && iq2 <= qmax2) {
        int ib = bin_search(pe2, P.N, ip2);
        int jb = bin_search(qe2, P.M, iq2);
        key = ((uint32_t)(ib * P.M + jb) << P.nbits) | (uint32_t)n;
      }
    }
    keys[n] = key;
  }
  __syncthreads();
  switch (P.np2 / kThreads) {  // keys per thread
    case 1: bitonic_sort_reg<1>(keys, P.np2); break;
    case 2: bitonic_sort_reg<2>(keys, P.np2); break;
    case 4: bitonic_sort_reg<4>(keys, P.np2); break;
    case 8: bitonic_sort_reg<8>(keys, P.np2); break;
    case 16: bitonic_sort_reg<16>(keys, P.np2); break;
    default: bitonic_sort<kThreads>(keys, P.np2); break;
  }
  int local = 0;
  for (int n = threadIdx.x; n < P.np2; n += kThreads) {
    uint32_t k = keys[n];
    if (k != kInvalid && (n == 0 || (keys[n - 1] >> P.nbits) != (k >> P.nbits))) ++local;
    sorted[(size_t)c * P.np2 + n] = k;
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    counts[c] = s;
  }
}

// single-CTA exclusive scan of n counts into row_ptr[n + 1]
__global__ void __launch_bounds__(1024) scan_kernel(const int64_t *counts, int n, int64_t *row_ptr) {
  __shared__ int64_t part[1024];
  const int T = 1024;
  int chunk = (n + T - 1) / T;
  int b = threadIdx.x * chunk, e = min(n, b + chunk);
  int64_t s = 0;
  for (int k = b; k < e; ++k) s += counts[k];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < T; off <<= 1) {
    int64_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = part[threadIdx.x] - s;
  for (int k = b; k < e; ++k) {
    row_ptr[k] = run;
    run += counts[k];
  }
  if (threadIdx.x == T - 1) row_ptr[n] = part[T - 1];
}

// ---- accumulators -----------------------------------------------------------
struct Acc64 {
  double v;
  __device__ void zero() { v = 0.0; }
  __device__ void fma(double a, double b) { v = ::fma(a, b, v); }
  __device__ void add(const Acc64 &o) { v += o.v; }
  __device__ double value() const { return v; }
  __device__ Acc64 shfl_up(int d) const { Acc64 r; r.v = __shfl_up_sync(0xffffffffu, v, d); return r; }
};

// float-float accumulator (Knuth TwoSum): hi + lo carries the sum exactly
// up to the rounding of lo
struct AccFF {
  float hi, lo;
  __device__ void zero() { hi = 0.f; lo = 0.f; }
  __device__ static void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  }
  __device__ void add(float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ void fma(float a, float b) { add(__fmul_rn(a, b)); }
  __device__ void add(const AccFF &o) {
    float s, e;
    two_sum(hi, o.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, o.lo));
    two_sum(s, e, hi, lo);
  }
  __device__ double value() const { return (double)hi + (double)lo; }
  __device__ AccFF shfl_up(int d) const {
    AccFF r;
    r.hi = __shfl_up_sync(0xffffffffu, hi, d);
    r.lo = __shfl_up_sync(0xffffffffu, lo, d);
    return r;
  }
};

template <bool F64>
struct NodeVal;
template <>
struct NodeVal<true> {
  using real = double;
  using Acc = Acc64;
};
template <>
struct NodeVal<false> {
  using real = float;
  using Acc = AccFF;
};

// P_0 .. P_{NCH-1} at y by the three-term recurrence
template <typename real, int NCH>
__device__ __forceinline__ void legendre_n(real y, real *P) {
  P[0] = real(1);
  if (NCH > 1) P[1] = y;
#pragma unroll
  for (int n = 1; n + 1 < NCH; ++n)
    P[n + 1] = (real(2 * n + 1) / real(n + 1)) * y * P[n] - (real(n) / real(n + 1)) * P[n - 1];
}

// Per (p, q) node pair constants of one source cell (FP64):
//   p'^2 = A y + Bp,  q'^2 = C y + D,  p'.q' = nA y + nB,  and the weight
//   wp wq.  Shared by the n_x y-nodes of the pair.
struct PairConst {
  double A, Bp, C, D, nA, nB, W;
};

template <bool F64, int NCH>
__global__ void __launch_bounds__(kThreads) fill_kernel(AsmParams P, const uint32_t *sorted,
                                                        const int64_t *row_ptr, int32_t *col,
                                                        typename NodeVal<F64>::real *val,
                                                        int64_t nnz) {
  using real = typename NodeVal<F64>::real;
  using Acc = typename NodeVal<F64>::Acc;
  constexpr int NPAIR = pair_count(NCH);
  extern __shared__ __align__(16) unsigned char smem[];
  PairConst *pc = reinterpret_cast<PairConst *>(smem);           // [n_p * n_q]
  real *Pyw = reinterpret_cast<real *>(pc + P.n_p * P.n_q);     // w_y P_l(y) [n_x][NCH]
  uint32_t *keys = reinterpret_cast<uint32_t *>(Pyw + P.n_x * NCH + 2);  // [np2]
  __shared__ Acc wtot[kThreads / 32][NPAIR];
  __shared__ int wflag[kThreads / 32];
  __shared__ int whead[kThreads / 32];

  const int c = blockIdx.x;
  const int i = c / P.M, j = c % P.M;
  const int R = P.np2 / kThreads;  // consecutive sorted elements per thread
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t mask = (1u << P.nbits) - 1u;
  const int nbits = P.nbits;

  for (int ab = threadIdx.x; ab < P.n_p * P.n_q; ab += kThreads) {
    int a = ab / P.n_q, b = ab % P.n_q;
    double p = P.pn[i * P.n_p + a], q = P.qn[j * P.n_q + b];
    PairConst k;
    k.A = __dmul_rn(__dmul_rn(0.75, p), q);
    k.Bp = __dadd_rn(__dmul_rn(__dmul_rn(p, p), 0.25), __dmul_rn(__dmul_rn(q, q), 0.5625));
    k.C = -__dmul_rn(p, q);
    k.D = __dadd_rn(__dmul_rn(p, p), __dmul_rn(__dmul_rn(q, q), 0.25));
    k.nA = -0.5 * p * q;
    k.nB = 0.375 * q * q - 0.5 * p * p;
    k.W = P.wp[i * P.n_p + a] * P.wq[j * P.n_q + b];
    pc[ab] = k;
  }
  for (int x = threadIdx.x; x < P.n_x; x += kThreads) {
    real Pl[NCH];
    legendre_n<real, NCH>((real)P.yn[x], Pl);
#pragma unroll
    for (int l = 0; l < NCH; ++l) Pyw[x * NCH + l] = (real)P.wy[x] * Pl[l];
  }
  for (int n = threadIdx.x; n < P.np2; n += kThreads) keys[n] = sorted[(size_t)c * P.np2 + n];
  __syncthreads();

  auto is_head = [&](int e) {
    uint32_t k = keys[e];
    return k != kInvalid && (e == 0 || (keys[e - 1] >> nbits) != (k >> nbits));
  };
  auto is_tail = [&](int e) {
    uint32_t k = keys[e];
    return k != kInvalid &&
           (e + 1 == P.np2 || keys[e + 1] == kInvalid || (keys[e + 1] >> nbits) != (k >> nbits));
  };
  // add the contributions of sorted element e to every (l, l') pair:
  // acc[m] += (W_pq w_y P_l(y)) P_l'(y'), the first factor per l
  auto accumulate = [&](int e, Acc *acc) {
    int node = (int)(keys[e] & mask);
    int x = node % P.n_x;
    const PairConst &k = pc[node / P.n_x];
    double y = P.yn[x];
    real yp;
    if (F64) {
      double p2 = fma(k.A, y, k.Bp), q2 = fma(k.C, y, k.D), num = fma(k.nA, y, k.nB);
      double den2 = p2 * q2;  // both >= 0 up to rounding; guarded below
      yp = den2 > 0.0 ? num * rsqrt(den2) : 0.0;
    } else {
      // recoupled squares and p'.q' in FP64 (three FMAs), the rest in FP32
      float p2 = (float)fma(k.A, y, k.Bp), q2 = (float)fma(k.C, y, k.D);
      float num = (float)fma(k.nA, y, k.nB);
      float den2 = p2 * q2;
      float cc = den2 > 0.f ? num * rsqrtf(den2) : 0.f;
      yp = (real)fminf(1.f, fmaxf(-1.f, cc));
    }
    real Pl2[NCH];
    legendre_n<real, NCH>(yp, Pl2);
    real wl[NCH];
    const real W = (real)k.W;
#pragma unroll
    for (int l = 0; l < NCH; ++l) wl[l] = W * Pyw[x * NCH + l];
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) acc[m].fma(wl[pair_first(NCH, m)], Pl2[pair_second(NCH, m)]);
  };

  // step A: segment ranks from an integer scan of the head flags
  const int e0 = threadIdx.x * R;
  int nhead = 0;
  for (int r = 0; r < R; ++r) nhead += is_head(e0 + r) ? 1 : 0;
  int hscan = nhead;
  for (int d = 1; d < 32; d <<= 1) {
    int hu = __shfl_up_sync(0xffffffffu, hscan, d);
    if (lane >= d) hscan += hu;
  }
  if (lane == 31) whead[warp] = hscan;
  __syncthreads();
  int hbase = 0;
  for (int w = 0; w < warp; ++w) hbase += whead[w];
  const int seg0 = hbase + hscan - nhead;  // heads before this thread
  const int64_t base = row_ptr[c];
  const int64_t lim = row_ptr[c + 1];
  const double rs_src = P.rsb[c];

  auto write_seg = [&](int seg, uint32_t k, const Acc *sum) {
    int64_t o = base + seg;
    if (o < lim) {
      int t = (int)(k >> nbits);
      col[o] = t;
      double nrm = rs_src * P.rsb[t];
#pragma unroll
      for (int m = 0; m < NPAIR; ++m) val[(size_t)m * nnz + o] = (real)(sum[m].value() * nrm * P.cnorm[m]);
    }
  };

  // step B: one pass over my elements; segments that open and close here are
  // written at once, the leading one (continuing from earlier threads) waits
  Acc run[NPAIR], lead[NPAIR];
#pragma unroll
  for (int m = 0; m < NPAIR; ++m) {
    run[m].zero();
    lead[m].zero();
  }
  int flag = 0, local_heads = 0, lead_tail = 0;
  uint32_t lead_key = 0;
  for (int r = 0; r < R; ++r) {
    const int e = e0 + r;
    const uint32_t k = keys[e];
    if (k == kInvalid) break;
    if (is_head(e)) {
      flag = 1;
      ++local_heads;
#pragma unroll
      for (int m = 0; m < NPAIR; ++m) run[m].zero();
    }
    accumulate(e, run);
    if (is_tail(e)) {
      if (flag) {
        write_seg(seg0 + local_heads - 1, k, run);
      } else {
#pragma unroll
        for (int m = 0; m < NPAIR; ++m) lead[m] = run[m];
        lead_tail = 1;
        lead_key = k;
      }
    }
  }
  // step C: segmented scan of (flag, sum of the segment open at my end)
  Acc agg[NPAIR];
#pragma unroll
  for (int m = 0; m < NPAIR; ++m) agg[m] = run[m];
  int f = flag;
  for (int d = 1; d < 32; d <<= 1) {
    int fu = __shfl_up_sync(0xffffffffu, f, d);
    Acc su[NPAIR];
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) su[m] = agg[m].shfl_up(d);
    if (lane >= d) {
      if (!f) {
#pragma unroll
        for (int m = 0; m < NPAIR; ++m) agg[m].add(su[m]);
      }
      f |= fu;
    }
  }
  if (lane == 31) {
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) wtot[warp][m] = agg[m];
    wflag[warp] = f;
  }
  __syncthreads();
  Acc carry[NPAIR];
#pragma unroll
  for (int m = 0; m < NPAIR; ++m) carry[m].zero();
  int cflag = 0;
  for (int w = warp - 1; w >= 0 && !cflag; --w) {
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) carry[m].add(wtot[w][m]);
    cflag = wflag[w];
  }
  if (!f) {
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) agg[m].add(carry[m]);
  }
  // exclusive value for this thread = inclusive value of the previous one
  Acc excl[NPAIR];
#pragma unroll
  for (int m = 0; m < NPAIR; ++m) excl[m] = agg[m].shfl_up(1);
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) excl[m] = carry[m];
  }
  // step D: close the leading segment with the carry from earlier threads
  if (lead_tail) {
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) lead[m].add(excl[m]);
    write_seg(seg0 - 1, lead_key, lead);
  }
}

template <bool F64, int NCH>
void launch_fill(const AsmParams &P, int n_cells, size_t smem, cudaStream_t s, const uint32_t *sorted,
                 const int64_t *row_ptr, int32_t *col, void *val, int64_t nnz) {
  using real = typename NodeVal<F64>::real;
  auto kern = fill_kernel<F64, NCH>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<n_cells, kThreads, smem, s>>>(P, sorted, row_ptr, col, reinterpret_cast<real *>(val), nnz);
}

template <bool F64>
wpcd_status dispatch_fill(const AsmParams &P, int n_cells, size_t smem, cudaStream_t s,
                          const uint32_t *sorted, const int64_t *row_ptr, int32_t *col, void *val,
                          int64_t nnz) {
  switch (P.n_ch) {
    case 1: launch_fill<F64, 1>(P, n_cells, smem, s, sorted, row_ptr, col, val, nnz); break;
    case 2: launch_fill<F64, 2>(P, n_cells, smem, s, sorted, row_ptr, col, val, nnz); break;
    case 3: launch_fill<F64, 3>(P, n_cells, smem, s, sorted, row_ptr, col, val, nnz); break;
    case 4: launch_fill<F64, 4>(P, n_cells, smem, s, sorted, row_ptr, col, val, nnz); break;
    case 5: launch_fill<F64, 5>(P, n_cells, smem, s, sorted, row_ptr, col, val, nnz); break;
    default: return set_error(WPCD_EINVAL, "unsupported number of channels");
  }
  return WPCD_OK;
}

}  // namespace

wpcd_status assemble(wpcd_grid *g, int n_ch, int prec, cudaStream_t s, wpcd_P **out) {
  if (prec != WPCD_FP64 && prec != WPCD_FP32C) return set_error(WPCD_EINVAL, "prec must be WPCD_FP64 or WPCD_FP32C");
  if (n_ch < 1 || n_ch > 5) return set_error(WPCD_EINVAL, "n_ch must be in [1, 5]");
  WPCD_CUDA_TRY(cudaSetDevice(g->device));
  AsmParams P{};
  P.N = g->N;
  P.M = g->M;
  P.n_p = g->n_p;
  P.n_q = g->n_q;
  P.n_x = g->n_x;
  P.n_nodes = g->n_p * g->n_q * g->n_x;
  int np2 = kThreads;
  while (np2 < P.n_nodes) np2 *= 2;
  P.np2 = np2;
  int nbits = 0;
  while ((1 << nbits) < np2) ++nbits;
  P.nbits = nbits;
  P.n_ch = n_ch;
  P.n_pairs = pair_count(n_ch);
  for (int m = 0; m < P.n_pairs; ++m) {
    P.pl[m] = pair_first(n_ch, m);
    P.plp[m] = pair_second(n_ch, m);
    P.cnorm[m] = sqrt((2.0 * P.pl[m] + 1.0) * (2.0 * P.plp[m] + 1.0));
  }
  P.pe2 = g->pe2;
  P.qe2 = g->qe2;
  P.pn = g->pn;
  P.wp = g->wp;
  P.qn = g->qn;
  P.wq = g->wq;
  P.yn = g->yn;
  P.wy = g->wy;
  P.rsb = g->rsb;
  const int n_cells = P.N * P.M;
  if (np2 > 8192) return set_error(WPCD_EINVAL, "too many quadrature nodes per cell (max 8192)");
  if ((int64_t)n_cells << nbits >= (int64_t)1 << 32)
    return set_error(WPCD_EINVAL, "lattice too large for 32-bit packed node keys");

  cudaEvent_t ev0, ev1, evc, evs;
  WPCD_CUDA_TRY(cudaEventCreate(&ev0));
  WPCD_CUDA_TRY(cudaEventCreate(&ev1));
  WPCD_CUDA_TRY(cudaEventCreate(&evc));
  WPCD_CUDA_TRY(cudaEventCreate(&evs));
  int64_t *counts = nullptr;
  uint32_t *sorted = nullptr;
  wpcd_P *Pm = new wpcd_P();
  Pm->grid = g;
  Pm->device = g->device;
  Pm->n_ch = n_ch;
  Pm->prec = prec;
  Pm->n_pairs = P.n_pairs;
  Pm->work = (int64_t)n_cells * P.n_nodes;  // every node of every cell mapped once
  auto fail = [&](wpcd_status st) {
    dev_free(counts);
    dev_free(sorted);
    dev_free(Pm->row_ptr);
    dev_free(Pm->col);
    dev_free(Pm->val64);
    dev_free(Pm->val32);
    delete Pm;
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaEventDestroy(evc);
    cudaEventDestroy(evs);
    return st;
  };
  cudaError_t e;
  if ((e = dev_malloc(&counts, sizeof(int64_t) * n_cells)) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc counts"));
  if ((e = dev_malloc(&sorted, sizeof(uint32_t) * (size_t)n_cells * np2)) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc sorted keys"));
  if ((e = dev_malloc(&Pm->row_ptr, sizeof(int64_t) * (n_cells + 1))) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc row_ptr"));

  cudaEventRecord(ev0, s);
  size_t smem_count = sizeof(long long) * (P.N + P.M + 2) + sizeof(BinConst) * P.n_p * P.n_q +
                      sizeof(double) * P.n_x + sizeof(uint32_t) * np2;
  cudaFuncSetAttribute(count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_count);
  count_kernel<<<n_cells, kThreads, smem_count, s>>>(P, counts, sorted);
  cudaEventRecord(evc, s);
  scan_kernel<<<1, 1024, 0, s>>>(counts, n_cells, Pm->row_ptr);
  cudaEventRecord(evs, s);
  count_launches(2);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_error(e, "count/scan launch"));
  int64_t nnz = 0;
  if ((e = cudaMemcpyAsync(&nnz, Pm->row_ptr + n_cells, sizeof(int64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail(cuda_error(e, "nnz readback"));
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(cuda_error(e, "count pass"));
  Pm->nnz = nnz;
  size_t nz = nnz > 0 ? (size_t)nnz : 1;
  if ((e = dev_malloc(&Pm->col, sizeof(int32_t) * nz)) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc col"));
  void *val = nullptr;
  if (prec == WPCD_FP64) {
    if ((e = dev_malloc(&Pm->val64, sizeof(double) * nz * P.n_pairs)) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc val"));
    val = Pm->val64;
  } else {
    if ((e = dev_malloc(&Pm->val32, sizeof(float) * nz * P.n_pairs)) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc val"));
    val = Pm->val32;
  }
  size_t rsz = prec == WPCD_FP64 ? sizeof(double) : sizeof(float);
  size_t smem_fill = sizeof(double) * 7 * (size_t)P.n_p * P.n_q +
                     rsz * ((size_t)P.n_x * P.n_ch + 2) + sizeof(uint32_t) * np2;
  smem_fill = (smem_fill + 15) & ~(size_t)15;
  wpcd_status st = prec == WPCD_FP64
                       ? dispatch_fill<true>(P, n_cells, smem_fill, s, sorted, Pm->row_ptr, Pm->col, val, nnz)
                       : dispatch_fill<false>(P, n_cells, smem_fill, s, sorted, Pm->row_ptr, Pm->col, val, nnz);
  if (st != WPCD_OK) return fail(st);
  count_launches(1);
  cudaEventRecord(ev1, s);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_error(e, "fill launch"));
  if ((e = cudaEventSynchronize(ev1)) != cudaSuccess) return fail(cuda_error(e, "fill pass"));
  cudaEventElapsedTime(&Pm->ms, ev0, ev1);
  cudaEventElapsedTime(&Pm->ms_phase[0], ev0, evc);
  cudaEventElapsedTime(&Pm->ms_phase[1], evc, evs);
  cudaEventElapsedTime(&Pm->ms_phase[2], evs, ev1);
  dev_free(counts);
  dev_free(sorted);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  cudaEventDestroy(evc);
  cudaEventDestroy(evs);
  grid_retain(g);  // P0 keeps its lattice alive
  *out = Pm;
  return WPCD_OK;
}

}  // namespace wpcd
