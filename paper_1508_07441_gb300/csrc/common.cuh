// Device pieces shared by the single-problem batched solver (solve.cu) and
// the grouped solver over problems of uneven size (group.cu): complex and
// accumulator types, the dense block-GEMM tile, the per-system Givens /
// back-substitution kernels of the Krylov least-squares problem, and the
// autotuner's candidate SpMM launch shapes.  Everything sits in an unnamed
// namespace, so each translation unit gets its own copy of the kernels.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "wpcd_internal.h"

namespace wpcd {
namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// FP64 <-> FP32 conversions by integer operations.  On GB300 a conversion
// instruction occupies an FP64-pipe slot like a multiply-add, and the
// splitting kernels below are bound by that pipe; these take the integer
// pipe instead.  f64_to_f32_rn rounds to nearest, ties to even (IEEE 754),
// for results in the float normal range; |v| below 2^-126 gives a signed
// zero (no float subnormals: those magnitudes are far below every value these
// kernels handle), beyond the float range an infinity, a NaN stays a NaN.
__device__ __forceinline__ float f64_to_f32_rn(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (e < 897) return __uint_as_float(sign);
  if (e == 2047) return __uint_as_float(sign | (m ? 0x7FC00000u : 0x7F800000u));
  if (e > 1150) return __uint_as_float(sign | 0x7F800000u);
  // the float's exponent and mantissa fields before rounding; the 29 bits
  // dropped decide the rounding, and a carry out of the mantissa raises the
  // exponent (to infinity past the largest float)
  unsigned r = ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29);
  const unsigned rem = (unsigned)(m & 0x1FFFFFFFull);
  r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
  return __uint_as_float(sign | r);
}

// exact widening of a float that f64_to_f32_rn produced (zero or normal;
// infinities and NaNs keep their class)
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned fe = (u >> 23) & 0xFFu;
  const unsigned long long man = (unsigned long long)(u & 0x7FFFFFu) << 29;
  if (fe == 0) return __longlong_as_double((long long)sign);
  if (fe == 255) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull | man));
  return __longlong_as_double((long long)(sign | ((unsigned long long)(fe + 896) << 52) | man));
}

template <typename T>
struct Cx;
template <>
struct Cx<double> {
  using t = double2;
};
template <>
struct Cx<float> {
  using t = float2;
};

// one block-CSR P0 and the SpMM launch shape (rows per warp, energy lanes)
struct SpmmParams {
  int n_cells, B, rpw, el;
  const int64_t *row_ptr;
  const int32_t *col;
  int64_t nnz;
};

// SpMM accumulators: plain FP64 sums, or FP32 compensated sums (Knuth's
// TwoSum on the running sum, the rounding errors gathered in lo)
struct AccD {
  double v;
  __device__ void zero() { v = 0.0; }
  __device__ void add(double x) { v += x; }
  __device__ void add_shfl(int off) { v += __shfl_xor_sync(0xffffffffu, v, off); }
  __device__ double value() const { return v; }
};

struct AccF {
  float hi, lo;
  __device__ void zero() { hi = 0.f; lo = 0.f; }
  __device__ void add(float x) {
    float s = __fadd_rn(hi, x);
    float bb = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ void add_shfl(int off) {
    float ohi = __shfl_xor_sync(0xffffffffu, hi, off);
    float olo = __shfl_xor_sync(0xffffffffu, lo, off);
    add(ohi);
    lo = __fadd_rn(lo, olo);
  }
  __device__ float value() const { return __fadd_rn(hi, lo); }
};

// the same compensated sums held in shared memory, for a lane whose
// registers are better spent on loads in flight than on accumulators
// touched once per block of nonzeros: slot k = ((l EPT + t) 2 + q) of the
// thread keeps hi at base[2 k S] and lo at base[(2 k + 1) S], S the block
// size (thread-major, so a warp's accesses hit distinct banks)
constexpr int kAccSmStride = 256;
struct AccFSView {
  float *base;  // the thread's first slot
  __device__ void add_slot(int k, float x) {
    float *h = base + 2 * k * kAccSmStride;
    const float hi = h[0];
    float s = __fadd_rn(hi, x);
    float bb = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    h[0] = s;
    h[kAccSmStride] = __fadd_rn(h[kAccSmStride], e);
  }
};

// add x to accumulator (l, t, q): register accumulators, or the shared view
template <int EPT, typename A, int NCH, typename X>
__device__ __forceinline__ void acc_add(A (&acc)[NCH][EPT][2], int l, int t, int q, X x) {
  acc[l][t][q].add(x);
}
template <int EPT>
__device__ __forceinline__ void acc_add(AccFSView &v, int l, int t, int q, float x) {
  v.add_slot((l * EPT + t) * 2 + q, x);
}

template <typename T>
struct AccOf;
template <>
struct AccOf<double> {
  using t = AccD;
};
template <>
struct AccOf<float> {
  using t = AccF;
};

// nonzeros a lane keeps in flight in the SpMM (fewer for wide channel sets,
// whose value blocks take more registers; measured: halving it for
// several energies per lane buys occupancy but loses more in memory
// parallelism)
template <int NCH, int EPT>
struct SpmmUnroll {
  static constexpr int value = NCH <= 3 ? 4 : 2;
};

// groups of U nonzeros per block partial: FP32 blocks of 4 U nonzeros (one
// compensated add per 16 nonzeros for U = 4), FP64 blocks of U
template <typename T>
struct SpmmGroups {
  static constexpr int value = sizeof(T) == 4 ? 4 : 1;
};

// The sums of one block-CSR row for the SpMM kernels.  A lane takes the
// nonzeros o = b + nl, b + nl + nl_count, ... of its row, U at a time (their
// column and value loads issued together), and for each of its EPT energies
// forms the block partial of G such groups (G U nonzeros) with plain FMAs
// and adds it to the accumulator.  For FP32 this is blocked summation with a
// compensated sum of the block partials (FABsum, Blanchard, Higham and Mary,
// SIAM J. Sci. Comput. 2020, block size b = 16): the error grows with the
// number of blocks only through the float-float accumulator, and inside a
// block with its b terms.  FP64 sums the block partials plainly.  y points at the problem's own vector
// block ([n_ch][n_cells][B] complex).  The lane's energies are en0 +
// estride * t; with VEC (FP32, EPT and B even, en0 even) the pair t, t + 1
// starts at en0 + estride * t and comes in one 16-byte load.
template <typename VT, typename T, int NCH, int EPT, bool VEC, typename Acc>
__device__ __forceinline__ void spmm_row(int64_t b, int64_t e, int nl, int nl_count, const int32_t *__restrict__ col,
                                         const VT *__restrict__ val, int64_t nnz,
                                         const typename Cx<T>::t *__restrict__ y, int n_cells, int B, int en0,
                                         int estride, Acc &acc) {
  using C2 = typename Cx<T>::t;
  constexpr int NPAIR = pair_count(NCH);
  constexpr int U = SpmmUnroll<NCH, EPT>::value;
  constexpr int TS = VEC ? 2 : 1;  // energies per load
  static_assert(!VEC || (sizeof(T) == 4 && EPT % 2 == 0), "vector loads need FP32 and an even EPT");
  constexpr int G = SpmmGroups<T>::value;
  for (int64_t ob = b + nl; ob < e; ob += (int64_t)G * U * nl_count) {
    T part[NCH][EPT][2];
#pragma unroll
    for (int l = 0; l < NCH; ++l)
#pragma unroll
      for (int t = 0; t < EPT; ++t) part[l][t][0] = part[l][t][1] = T(0);
#pragma unroll 1
    for (int gi = 0; gi < G; ++gi) {
      const int64_t o0 = ob + (int64_t)gi * U * nl_count;
      if (o0 >= e) break;
      int tc[U];
      T v[U][NPAIR];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t o = o0 + (int64_t)u * nl_count;
        const bool ok = o < e;
        tc[u] = ok ? __ldg(col + o) : -1;
#pragma unroll
        for (int m = 0; m < NPAIR; ++m) v[u][m] = ok ? (T)__ldg(val + (size_t)m * nnz + o) : T(0);
      }
#pragma unroll
      for (int t0 = 0; t0 < EPT; t0 += TS) {
        const int en = en0 + estride * t0;
        if (en < B) {
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if (tc[u] >= 0) {
              T yr[NCH][TS], yi[NCH][TS];
#pragma unroll
              for (int l = 0; l < NCH; ++l) {
                const C2 *p = y + ((size_t)l * n_cells + tc[u]) * B + en;
                if constexpr (VEC) {
                  const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
                  yr[l][0] = q.x;
                  yi[l][0] = q.y;
                  yr[l][TS - 1] = q.z;
                  yi[l][TS - 1] = q.w;
                } else {
                  const C2 q = __ldg(p);
                  yr[l][0] = q.x;
                  yi[l][0] = q.y;
                }
              }
#pragma unroll
              for (int m = 0; m < NPAIR; ++m) {
                const int l = pair_first(NCH, m), lp = pair_second(NCH, m);
#pragma unroll
                for (int q = 0; q < TS; ++q) {
                  part[l][t0 + q][0] = fma(v[u][m], yr[lp][q], part[l][t0 + q][0]);
                  part[l][t0 + q][1] = fma(v[u][m], yi[lp][q], part[l][t0 + q][1]);
                }
              }
            }
          }
        }
      }
    }
#pragma unroll
    for (int l = 0; l < NCH; ++l)
#pragma unroll
      for (int t = 0; t < EPT; ++t) {
        acc_add<EPT>(acc, l, t, 0, part[l][t][0]);
        acc_add<EPT>(acc, l, t, 1, part[l][t][1]);
      }
  }
}

// a row's sums into the register accumulators acc (zeroed here): summed in
// place, or with SACC (FP32) in shared memory (acc_sm: the block's 4 NCH EPT
// slots per thread, thread-major) and read back, which leaves the lane's
// registers to the loads in flight
template <typename VT, typename T, int NCH, int EPT, bool VEC, bool SACC>
__device__ __forceinline__ void spmm_row_sums(int64_t b, int64_t e, int nl, int nl_count,
                                              const int32_t *__restrict__ col, const VT *__restrict__ val,
                                              int64_t nnz, const typename Cx<T>::t *__restrict__ y, int n_cells,
                                              int B, int en0, int estride, typename AccOf<T>::t (&acc)[NCH][EPT][2],
                                              float *acc_sm) {
  if constexpr (SACC) {
    static_assert(sizeof(T) == 4, "shared-memory accumulators are FP32 compensated sums");
    AccFSView sacc{acc_sm + threadIdx.x};
#pragma unroll
    for (int k = 0; k < 4 * NCH * EPT; ++k) sacc.base[k * kAccSmStride] = 0.f;
    spmm_row<VT, T, NCH, EPT, VEC>(b, e, nl, nl_count, col, val, nnz, y, n_cells, B, en0, estride, sacc);
#pragma unroll
    for (int l = 0; l < NCH; ++l)
#pragma unroll
      for (int t = 0; t < EPT; ++t)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int k = (l * EPT + t) * 2 + q;
          acc[l][t][q].hi = sacc.base[2 * k * kAccSmStride];
          acc[l][t][q].lo = sacc.base[(2 * k + 1) * kAccSmStride];
        }
  } else {
#pragma unroll
    for (int l = 0; l < NCH; ++l)
#pragma unroll
      for (int t = 0; t < EPT; ++t) {
        acc[l][t][0].zero();
        acc[l][t][1].zero();
      }
    spmm_row<VT, T, NCH, EPT, VEC>(b, e, nl, nl_count, col, val, nnz, y, n_cells, B, en0, estride, acc);
  }
}

// dynamic shared memory of the shared-accumulator SpMM kernels (hi and lo
// of 2 NCH EPT sums per thread of a 256-thread block); kernel K opts in
// once above 48 KB (extra: its static shared memory)
template <int NCH, int EPT, typename K>
cudaError_t sacc_smem(K kernel, size_t *bytes, bool &opted_in, size_t extra = 0) {
  *bytes = (size_t)4 * NCH * EPT * kAccSmStride * sizeof(float);
  if (*bytes + extra <= 48 * 1024 || opted_in) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*bytes);
  opted_in = e == cudaSuccess;
  return e;
}

int grid_for(int64_t n, int threads, int cap = 152 * 8) {
  int64_t g = (n + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// ---------------------------------------------------------------------------
// dense block GEMM tile:  C (n x ncol) = A (n x n) * B' (n x ncol), rows
// row0..row0+31, columns col0..col0+63; B' = B, or the G1-scaled complex
// block (complex pairs along the columns, re at even columns); epilogue
// C = out, or C = S - out.  All pointers are at the block's origin; ncol is
// even, so complex pairs never straddle a row.
// ---------------------------------------------------------------------------
// 32 x 64 output tiles: 7 x 7 x 3 = 147 CTAs for the 200-bin, 3-channel,
// one-energy blocks, close to one wave over the 152 SMs (FP64 work is
// issue-bound, so SM coverage matters more than data reuse there)
constexpr int GB_M = 32, GB_N = 64, GB_K = 16, G_THREADS = 256;

template <typename T>
struct GemmSmem {
  T As[GB_K][GB_M + 1];
  T Bs[GB_K][GB_N];
};

template <typename T, bool SCALE_G, bool SUB>
__device__ __forceinline__ void gemm_tile(int n, int64_t ncol, const T *__restrict__ A, const T *__restrict__ B,
                                          const T *__restrict__ G, const T *__restrict__ S, T *__restrict__ C,
                                          int row0, int64_t col0, GemmSmem<T> &sm) {
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 2 x 4 outputs each
  T acc[2][4] = {};
  for (int k0 = 0; k0 < n; k0 += GB_K) {
    for (int t = threadIdx.x; t < GB_M * GB_K; t += G_THREADS) {
      int r = t / GB_K, kk = t % GB_K;
      int gr = row0 + r, gk = k0 + kk;
      sm.As[kk][r] = (gr < n && gk < n) ? A[(size_t)gr * n + gk] : T(0);
    }
    for (int t = threadIdx.x; t < GB_K * GB_N; t += G_THREADS) {
      int kk = t / GB_N, cc = t % GB_N;
      int gk = k0 + kk;
      int64_t gc = col0 + cc;
      T v = T(0);
      if (gk < n && gc < ncol) {
        size_t o = (size_t)gk * ncol + gc;
        if (SCALE_G) {
          size_t oc = o & ~(size_t)1;  // complex pair (re at even column)
          T xr = B[oc], xi = B[oc + 1], gr_ = G[oc], gi = G[oc + 1];
          v = (gc & 1) ? (gr_ * xi + gi * xr) : (gr_ * xr - gi * xi);
        } else {
          v = B[o];
        }
      }
      sm.Bs[kk][cc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      T a[2], bb[4];
#pragma unroll
      for (int u = 0; u < 2; ++u) a[u] = sm.As[kk][ty + 16 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u) bb[u] = sm.Bs[kk][tx + 16 * u];
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
      int gr = row0 + ty + 16 * u;
      int64_t gc = col0 + tx + 16 * v;
      if (gr < n && gc < ncol) {
        size_t o = (size_t)gr * ncol + gc;
        C[o] = SUB ? S[o] - acc[u][v] : acc[u][v];
      }
    }
}

// device time of the launches between start() and stop() (optional)
struct LaunchTimer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s;
  float *out;
  LaunchTimer(float *ms, cudaStream_t st) : s(st), out(ms) {
    if (out) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
    }
  }
  void start() {
    if (out) cudaEventRecord(a, s);
  }
  void stop() {
    if (out) cudaEventRecord(b, s);
  }
  ~LaunchTimer() {
    if (out) {
      cudaEventSynchronize(b);
      cudaEventElapsedTime(out, a, b);
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  }
};

// ---------------------------------------------------------------------------
// Krylov least squares, one thread per system (energy)
// ---------------------------------------------------------------------------
// Givens least-squares update of column k for every energy (thread e).
// Layout per energy e: H + e*(m+1)*m column-major (ld m+1), cs/sn + e*m,
// bet + e*(m+1); h[i * B + e], hn2[e].
__global__ void bgivens_kernel(int B, int m, int k, const double2 *h, const double2 *hn2, double2 *Hb,
                               double2 *csb, double2 *snb, double2 *betb, double *resid,
                               const double *bnorm) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  double2 *H = Hb + (size_t)e * (m + 1) * m, *cs = csb + (size_t)e * m, *sn = snb + (size_t)e * m;
  double2 *bet = betb + (size_t)e * (m + 1);
  double2 *col = H + (size_t)k * (m + 1);
  for (int i = 0; i <= k; ++i) col[i] = h[(size_t)i * B + e];
  col[k + 1] = make_double2(sqrt(fmax(hn2[e].x, 0.0)), 0.0);
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
  resid[e] = sqrt(bet[k + 1].x * bet[k + 1].x + bet[k + 1].y * bet[k + 1].y) / bnorm[e];
}

// c[j * S + s] = y[j * S + s] * sqrt(nrm2[s].x) (or y with nrm2 NULL) in the
// basis precision T: the coefficients of the correction V c, so that the
// elementwise update does no FP64 arithmetic but the final add
template <typename T>
__global__ void bupdate_coef_kernel(int k, int S, const double2 *__restrict__ y, const double2 *__restrict__ nrm2,
                                    typename Cx<T>::t *__restrict__ c) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= k * S) return;
  const int s = idx % S;
  const double sc = nrm2 ? sqrt(fmax(nrm2[s].x, 0.0)) : 1.0;
  c[idx].x = (T)(y[idx].x * sc);
  c[idx].y = (T)(y[idx].y * sc);
}

// back substitution H y = bet per energy; y[j * B + e]
__global__ void bbacksub_kernel(int B, int m, int k, const double2 *Hb, const double2 *betb, double2 *y) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  const double2 *H = Hb + (size_t)e * (m + 1) * m, *bet = betb + (size_t)e * (m + 1);
  for (int i = k - 1; i >= 0; --i) {
    double2 s = bet[i];
    for (int j = i + 1; j < k; ++j) {
      double2 h = H[(size_t)j * (m + 1) + i], yj = y[(size_t)j * B + e];
      s.x -= h.x * yj.x - h.y * yj.y;
      s.y -= h.x * yj.y + h.y * yj.x;
    }
    double2 d = H[(size_t)i * (m + 1) + i];
    double dd = d.x * d.x + d.y * d.y;
    y[(size_t)i * B + e] = dd > 0.0 ? make_double2((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd)
                                    : make_double2(0.0, 0.0);
  }
  for (int i = k; i < m; ++i) y[(size_t)i * B + e] = make_double2(0.0, 0.0);
}

// r = b - u + t  (FP64)
__global__ void bresid_kernel(int64_t n, const double2 *b, const double2 *u, const double2 *t, double2 *r) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n;
       f += (int64_t)gridDim.x * blockDim.x)
    r[f] = make_double2(b[f].x - u[f].x + t[f].x, b[f].y - u[f].y + t[f].y);
}

// warm-start fallback: energies flagged get u = 0, r = b
__global__ void bfallback_kernel(int64_t n, int B, const int *flag, const double2 *b, double2 *u, double2 *r) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(f % B);
    if (flag[e]) {
      u[f] = make_double2(0.0, 0.0);
      r[f] = b[f];
    }
  }
}

// Steps of a mixed-solve refinement cycle after the first: the previous
// cycle (mm_prev steps) took the worst relative residual from worst_prev to
// worst; at that per-step reduction, the steps to a tenth of tol, at least 2
// and at most m (m when there is no reduction to go by)
inline int next_cycle_steps(double worst, double worst_prev, int mm_prev, int m, double tol) {
  if (mm_prev <= 0 || !(worst_prev > 0.0) || !(worst > 0.0) || !(worst < worst_prev)) return m;
  const double rate = std::pow(worst / worst_prev, 1.0 / mm_prev);
  const double need = std::log(0.1 * tol / worst) / std::log(rate);
  return need < m ? std::max(2, (int)std::ceil(need)) : m;
}

// launch shapes tried by the autotuner for a batch of B energies
std::vector<SpmmConfig> candidates(int B) {
  std::vector<SpmmConfig> c;
  if (B == 1) {  // the one-right-hand-side SpMV (spmv.cu): ept = chunks per step
    for (int cps : {1, 2})
      for (int rpw : {2, 4, 8, 16}) c.push_back(SpmmConfig{rpw, 1, cps});
    return c;
  }
  int el = 1;
  while (el < B && el < 32) el *= 2;
  for (int ept : {1, 2, 4}) {
    if (ept > 1 && el * ept / 2 >= B) continue;  // tile wider than the batch
    c.push_back(SpmmConfig{1, el, ept});
    if (el <= 16) c.push_back(SpmmConfig{2, el, ept});
  }
  if (el > 1) c.push_back(SpmmConfig{1, el / 2, 1});
  // narrower energy lanes with more energies each (for FP32 these load two
  // adjacent energies at a time) leave two nonzero lanes per row
  if (el >= 8 && B % 2 == 0)
    for (int ept : {2, 4}) {
      if (el / 2 * ept / 2 >= B) continue;
      c.push_back(SpmmConfig{1, el / 2, ept});
    }
  return c;
}

}  // namespace
}  // namespace wpcd
