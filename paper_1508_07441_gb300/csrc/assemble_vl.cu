// P0 with variable limits (Sec. 3.2, after Eq. gal: the element of Eq. perm
// reduced to an integral with variable limits, "calculated numerically").
//
// For a GL node (p, q) of the source cell the recoupled squares are linear
// in y = p.q / (|p| |q|):
//   p'^2 = A y + Bp,  A = 3 p q / 4 > 0;   q'^2 = C y + Dq,  C = -p q < 0,
// so the theta functions of Eq. perm hold on one y-interval per target cell
// (i', j'): [yp(i'), yp(i'+1)] from the p edges, yp(k) = (e_k^2 - Bp) / A,
// intersected with [yq(j'+1), yq(j')] from the q edges, yq(k) =
// (f_k^2 - Dq) / C, and with [-1, 1].  P_l(y) P_l'(y') is integrated over the
// interval with the n_x-point GL rule mapped onto it; the p and q integrals
// keep the cell's GL rule.  Against node binning the theta functions are
// exact in y, so the element converges faster to the exact cell overlap.
//
// Kernels (FP64 throughout; the limits are IEEE divisions of values rounded
// in the canonical order, so identical inputs give identical limits):
//   vl_rows_kernel   one CTA per source cell: every (p, q) node walks its
//                    targets in increasing y (the next limit is the smaller
//                    of the next p limit and the next q limit) and inserts
//                    the non-empty ones into a shared-memory hash set of
//                    the row's targets, which is compacted and sorted: the
//                    row length, or (second launch) the row's ascending
//                    columns;
//   vl_value_kernel  one thread per nonzero element (the paper's own
//                    decomposition, Sec. 4.2): the sum over the source
//                    cell's nodes, in a fixed order, of the GL integral over
//                    the element's interval, normalised as in Eq. perm.
// The row lengths are summed into row pointers on the host (one copy each
// way); no atomics on values, so the result is bit-reproducible.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "wpcd_internal.h"

namespace wpcd {
namespace {

constexpr int VL_THREADS = 128;
constexpr int VL_MAX_SLOTS = 8192;  // hash slots for one row's distinct targets, at most
constexpr int VL_EMPTY = INT_MAX;

struct VlParams {
  int N, M, n_p, n_q, n_x, n_ch, n_pairs;
  int slot_bits, max_row;  // the row hash set: 2^slot_bits slots, filled to 3/4 at most
  int pl[kMaxPairs], plp[kMaxPairs];
  double cnorm[kMaxPairs];  // sqrt((2l+1)(2l'+1))
  const double *pe2, *qe2, *pn, *wp, *qn, *wq, *yn, *wy, *rsb;
};

// the linear coefficients of node (p, q), each product and sum rounded
// separately (no contraction), in the canonical order of the node-binned P0
struct VlNode {
  double A, Bp, C, Dq;
  __device__ VlNode(double p, double q) {
    A = __dmul_rn(__dmul_rn(0.75, p), q);
    Bp = __dadd_rn(__dmul_rn(__dmul_rn(p, p), 0.25), __dmul_rn(__dmul_rn(q, q), 0.5625));
    C = -__dmul_rn(p, q);
    Dq = __dadd_rn(__dmul_rn(p, p), __dmul_rn(__dmul_rn(q, q), 0.25));
  }
  // y limits of p edge k and q edge k (k beyond the grid: +-infinity)
  __device__ double yp(const VlParams &P, int k) const {
    return k > P.N ? INFINITY : __ddiv_rn(__dsub_rn(P.pe2[k], Bp), A);
  }
  __device__ double yq(const VlParams &P, int k) const {
    return k > P.M ? -INFINITY : __ddiv_rn(__dsub_rn(P.qe2[k], Dq), C);
  }
};

// the y-interval of target (it, jt) for the node; true if not empty
__device__ __forceinline__ bool vl_interval(const VlParams &P, const VlNode &nd, int it, int jt, double &lo,
                                            double &hi) {
  lo = fmax(-1.0, fmax(nd.yp(P, it), nd.yq(P, jt + 1)));
  hi = fmin(1.0, fmin(nd.yp(P, it + 1), nd.yq(P, jt)));
  return hi > lo;
}

// insert a target into the shared hash set of the row (multiplicative
// hash, linear probing): 1 new, 0 already present, -1 table full
__device__ __forceinline__ int vl_insert(int *table, int bits, int key) {
  const uint32_t mask = (1u << bits) - 1;
  uint32_t h = ((uint32_t)key * 2654435761u) >> (32 - bits);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const int old = atomicCAS(&table[h], VL_EMPTY, key);
    if (old == VL_EMPTY) return 1;
    if (old == key) return 0;
    h = (h + 1) & mask;
  }
  return -1;
}

// row lengths (cols == nullptr: counts[c]) or the row's ascending columns.
// The nodes' pieces overlap heavily (neighbouring nodes cross nearly the
// same targets), so each piece goes into a hash set of the row's distinct
// targets at once; the set is then compacted and sorted.
__global__ void __launch_bounds__(VL_THREADS) vl_rows_kernel(VlParams P, int64_t *counts, const int64_t *row_ptr,
                                                            int32_t *cols, int *err,
                                                            unsigned long long *pieces) {
  extern __shared__ int vl_smem[];
  const int slots = 1 << P.slot_bits;
  int *table = vl_smem, *keys = vl_smem + slots;
  __shared__ int n_distinct, n_fill, overflow;
  __shared__ unsigned long long n_pieces;
  const int c = blockIdx.x, i = c / P.M, j = c % P.M;
  for (int k = threadIdx.x; k < slots; k += blockDim.x) table[k] = VL_EMPTY;
  if (threadIdx.x == 0) {
    n_distinct = n_fill = overflow = 0;
    n_pieces = 0;
  }
  __syncthreads();
  unsigned long long my_pieces = 0;
  for (int node = threadIdx.x; node < P.n_p * P.n_q; node += blockDim.x) {
    const int a = node / P.n_q, b = node % P.n_q;
    const VlNode nd(P.pn[i * P.n_p + a], P.qn[j * P.n_q + b]);
    // the p bin and the q bin at y just above -1 (bin N, M: beyond the grid)
    int it = 0;
    while (it < P.N && !(nd.yp(P, it + 1) > -1.0)) ++it;
    int jt = P.M;
    while (jt > 0 && !(nd.yq(P, jt) > -1.0)) --jt;
    // walk up in y: from one target to the next across the nearer limit
    for (int guard = 0; guard < 2 * (P.N + P.M) + 4; ++guard) {
      double lo, hi;
      const bool in = it < P.N && jt < P.M;
      if (vl_interval(P, nd, it, jt, lo, hi) && in) {
        ++my_pieces;
        const int r = vl_insert(table, P.slot_bits, it * P.M + jt);
        if (r > 0)
          atomicAdd(&n_distinct, 1);
        else if (r < 0)
          overflow = 1;
      }
      const double up = nd.yp(P, it + 1), uq = nd.yq(P, jt);
      const double top = fmin(up, uq);
      if (!(top < 1.0) || it >= P.N || jt < 0) break;
      if (up <= uq) ++it;
      if (uq <= up) --jt;
      if (jt < 0) break;
    }
  }
  if (my_pieces) atomicAdd(&n_pieces, my_pieces);
  __syncthreads();
  const int n = n_distinct;
  if (pieces && threadIdx.x == 0) atomicAdd(pieces, n_pieces);
  if (overflow || n > P.max_row) {
    if (threadIdx.x == 0) atomicOr(err, 1);
    return;  // uniform over the CTA
  }
  // compact the set (any order), pad to a power of two, sort ascending
  for (int k = threadIdx.x; k < slots; k += blockDim.x) {
    const int v = table[k];
    if (v != VL_EMPTY) keys[atomicAdd(&n_fill, 1)] = v;
  }
  int np2 = 1;
  while (np2 < n) np2 <<= 1;
  __syncthreads();
  for (int k = n + threadIdx.x; k < np2; k += blockDim.x) keys[k] = INT_MAX;
  __syncthreads();
  for (int k = 2; k <= np2; k <<= 1)
    for (int d = k >> 1; d > 0; d >>= 1) {
      for (int x = threadIdx.x; x < np2; x += blockDim.x) {
        const int y = x ^ d;
        if (y > x) {
          const int u = keys[x], v = keys[y];
          if ((u > v) == ((x & k) == 0)) {
            keys[x] = v;
            keys[y] = u;
          }
        }
      }
      __syncthreads();
    }
  if (!cols) {
    if (threadIdx.x == 0) counts[c] = n;
  } else {
    const int64_t o = row_ptr[c];
    for (int k = threadIdx.x; k < n; k += blockDim.x) cols[o + k] = keys[k];
  }
}

// P_0 .. P_{NCH-1} at x by the three-term recurrence (constant coefficients)
template <int NCH>
__device__ __forceinline__ void legendre_t(double x, double *Pl) {
  Pl[0] = 1.0;
  if (NCH > 1) Pl[1] = x;
#pragma unroll
  for (int n = 1; n + 1 < NCH; ++n)
    Pl[n + 1] = (double(2 * n + 1) / double(n + 1)) * x * Pl[n] - (double(n) / double(n + 1)) * Pl[n - 1];
}

// 1/sqrt(d) for d > 0: an FP32 seed refined by one Newton-Raphson step in
// FP64 (relative error about 1.5 e^2 for the seed's e < 3e-7: below 2e-13);
// the seed's float is cut from d's bits and the result widened by integer
// operations (no conversion on the FP64 pipe); d outside 2^-99 .. 2^99 takes
// the FP64 rsqrt
__device__ __forceinline__ double vl_rsqrt(double d) {
  const long long b = __double_as_longlong(d);
  const int ex = (int)((b >> 52) & 0x7ff) - 1023;
  if (ex < -99 || ex > 99) return rsqrt(d);
  const unsigned fb = ((unsigned)(ex + 127) << 23) | (unsigned)((b >> 29) & 0x7fffff);
  const unsigned rb = __float_as_uint(rsqrtf(__uint_as_float(fb)));
  const double r = __longlong_as_double(((long long)((int)((rb >> 23) & 0xff) - 127 + 1023) << 52) |
                                        ((long long)(rb & 0x7fffff) << 29));
  const double e = fma(-(d * r), r, 1.0);
  // r / 2 by decrementing the exponent (r is normal): no FP64 multiply
  const double half_r = __longlong_as_double(__double_as_longlong(r) - (1LL << 52));
  return fma(half_r, e, r);
}

// one thread per nonzero of row c (CTA c): sum over the cell's nodes, in a
// fixed order, of the GL integral over the node's y-interval for the target
template <int NCH>
__global__ void __launch_bounds__(VL_THREADS) vl_value_kernel(VlParams P, const int64_t *row_ptr,
                                                             const int32_t *cols, int64_t nnz, double *val) {
  constexpr int NPAIR = pair_count(NCH);
  const int c = blockIdx.x, i = c / P.M, j = c % P.M;
  const int64_t b0 = row_ptr[c], b1 = row_ptr[c + 1];
  for (int64_t o = b0 + threadIdx.x; o < b1; o += blockDim.x) {
    const int t = cols[o], it = t / P.M, jt = t % P.M;
    double sum[NPAIR];
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) sum[m] = 0.0;
    for (int a = 0; a < P.n_p; ++a)
      for (int b = 0; b < P.n_q; ++b) {
        const double p = P.pn[i * P.n_p + a], q = P.qn[j * P.n_q + b];
        const VlNode nd(p, q);
        double lo, hi;
        if (!vl_interval(P, nd, it, jt, lo, hi)) continue;
        const double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
        const double hW = P.wp[i * P.n_p + a] * P.wq[j * P.n_q + b] * half;
        // p'.q' = nA y + nB = -p^2/2 - p q y / 2 + 3 q^2 / 8
        const double nA = -0.5 * p * q, nB = 0.375 * q * q - 0.5 * p * p;
        for (int x = 0; x < P.n_x; ++x) {
          const double y = fma(half, P.yn[x], mid);
          const double W = hW * P.wy[x];
          const double p2 = fma(nd.A, y, nd.Bp), q2 = fma(nd.C, y, nd.Dq), num = fma(nA, y, nB);
          const double den2 = fmax(p2, 0.0) * fmax(q2, 0.0);
          const double yp = den2 > 0.0 ? fmin(1.0, fmax(-1.0, num * vl_rsqrt(den2))) : 0.0;
          double Py[NCH], Pyp[NCH];
          legendre_t<NCH>(y, Py);
          legendre_t<NCH>(yp, Pyp);
#pragma unroll
          for (int l = 0; l < NCH; ++l) Py[l] *= W;
#pragma unroll
          for (int m = 0; m < NPAIR; ++m) sum[m] = fma(Py[pair_first(NCH, m)], Pyp[pair_second(NCH, m)], sum[m]);
        }
      }
    const double nrm = P.rsb[c] * P.rsb[t];
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) val[(size_t)m * nnz + o] = sum[m] * nrm * P.cnorm[m];
  }
}

template <int NCH>
void launch_vl_value(const VlParams &P, int n_cells, cudaStream_t s, const int64_t *row_ptr, const int32_t *cols,
                     int64_t nnz, double *val) {
  vl_value_kernel<NCH><<<n_cells, VL_THREADS, 0, s>>>(P, row_ptr, cols, nnz, val);
}

}  // namespace

wpcd_status assemble_vl(wpcd_grid *g, int n_ch, cudaStream_t s, wpcd_P **out) {
  if (n_ch < 1 || n_ch > 5) return set_error(WPCD_EINVAL, "n_ch must be in [1, 5]");
  WPCD_CUDA_TRY(cudaSetDevice(g->device));
  VlParams P{};
  P.N = g->N;
  P.M = g->M;
  P.n_p = g->n_p;
  P.n_q = g->n_q;
  P.n_x = g->n_x;
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
  // a row's targets lie near the paths of its nodes, each a monotone walk of
  // at most N + M + 1 cells: the hash set starts with 4 (N + M) slots (a
  // power of two) and doubles, up to VL_MAX_SLOTS, while a row overflows it
  P.slot_bits = 6;
  while ((1 << P.slot_bits) < 4 * (P.N + P.M) && (1 << P.slot_bits) < VL_MAX_SLOTS) ++P.slot_bits;
  const int n_cells = P.N * P.M;
  cudaEvent_t ev0, ev1, evc, evs;
  WPCD_CUDA_TRY(cudaEventCreate(&ev0));
  WPCD_CUDA_TRY(cudaEventCreate(&ev1));
  WPCD_CUDA_TRY(cudaEventCreate(&evc));
  WPCD_CUDA_TRY(cudaEventCreate(&evs));
  int64_t *counts = nullptr;
  int *err = nullptr;  // err[0] overflow flag, err[2..3] piece count (8-byte aligned)
  wpcd_P *Pm = new wpcd_P();
  Pm->grid = g;
  Pm->device = g->device;
  Pm->n_ch = n_ch;
  Pm->prec = WPCD_FP64;
  Pm->n_pairs = P.n_pairs;
  auto fail = [&](wpcd_status st) {
    dev_free(counts);
    dev_free(err);
    dev_free(Pm->row_ptr);
    dev_free(Pm->col);
    dev_free(Pm->val64);
    delete Pm;
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaEventDestroy(evc);
    cudaEventDestroy(evs);
    return st;
  };
  cudaError_t e;
  if ((e = dev_malloc(&counts, sizeof(int64_t) * n_cells)) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc counts"));
  if ((e = dev_malloc(&err, 4 * sizeof(int))) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc flag"));
  if ((e = dev_malloc(&Pm->row_ptr, sizeof(int64_t) * (n_cells + 1))) != cudaSuccess)
    return fail(cuda_error(e, "cudaMalloc row_ptr"));
  unsigned long long *d_pieces = reinterpret_cast<unsigned long long *>(err + 2);
  std::vector<int64_t> rp(n_cells + 1, 0);
  int herr[4] = {0, 0, 0, 0};
  size_t vl_smem = 0;
  cudaEventRecord(ev0, s);
  for (;;) {
    P.max_row = 3 * (1 << P.slot_bits) / 4;
    vl_smem = 2 * sizeof(int) * ((size_t)1 << P.slot_bits);  // hash set + sort buffer
    if ((e = cudaFuncSetAttribute(vl_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vl_smem)) !=
        cudaSuccess)
      return fail(cuda_error(e, "variable-limit rows kernel attribute"));
    cudaMemsetAsync(err, 0, 4 * sizeof(int), s);
    vl_rows_kernel<<<n_cells, VL_THREADS, vl_smem, s>>>(P, counts, nullptr, nullptr, err, d_pieces);
    count_launches(1);
    cudaEventRecord(evc, s);
    // row pointers: prefix sum of the row lengths on the host
    if ((e = cudaMemcpyAsync(rp.data() + 1, counts, sizeof(int64_t) * n_cells, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(herr, err, 4 * sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return fail(cuda_error(e, "variable-limit row lengths"));
    if (!herr[0]) break;
    if ((1 << P.slot_bits) >= VL_MAX_SLOTS) {
      char msg[96];
      std::snprintf(msg, sizeof msg, "variable-limit assembly: a row has more than %d targets", P.max_row);
      return fail(set_error(WPCD_EINVAL, msg));
    }
    ++P.slot_bits;
  }
  unsigned long long n_pieces = 0;
  std::memcpy(&n_pieces, herr + 2, sizeof(n_pieces));
  Pm->work = (int64_t)n_pieces * P.n_x;  // y points integrated
  for (int c = 0; c < n_cells; ++c) rp[c + 1] += rp[c];
  const int64_t nz = rp[n_cells];
  Pm->nnz = nz;
  if ((e = cudaMemcpyAsync(Pm->row_ptr, rp.data(), sizeof(int64_t) * (n_cells + 1), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return fail(cuda_error(e, "row_ptr upload"));
  cudaEventRecord(evs, s);
  if ((e = dev_malloc(&Pm->col, sizeof(int32_t) * (nz > 0 ? nz : 1))) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc col"));
  if ((e = dev_malloc(&Pm->val64, sizeof(double) * (nz > 0 ? nz : 1) * P.n_pairs)) != cudaSuccess)
    return fail(cuda_error(e, "cudaMalloc val"));
  vl_rows_kernel<<<n_cells, VL_THREADS, vl_smem, s>>>(P, nullptr, Pm->row_ptr, Pm->col, err, nullptr);
  switch (n_ch) {
    case 1: launch_vl_value<1>(P, n_cells, s, Pm->row_ptr, Pm->col, nz, Pm->val64); break;
    case 2: launch_vl_value<2>(P, n_cells, s, Pm->row_ptr, Pm->col, nz, Pm->val64); break;
    case 3: launch_vl_value<3>(P, n_cells, s, Pm->row_ptr, Pm->col, nz, Pm->val64); break;
    case 4: launch_vl_value<4>(P, n_cells, s, Pm->row_ptr, Pm->col, nz, Pm->val64); break;
    default: launch_vl_value<5>(P, n_cells, s, Pm->row_ptr, Pm->col, nz, Pm->val64); break;
  }
  count_launches(2);
  cudaEventRecord(ev1, s);
  if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventSynchronize(ev1)) != cudaSuccess)
    return fail(cuda_error(e, "variable-limit assembly"));
  cudaEventElapsedTime(&Pm->ms, ev0, ev1);
  cudaEventElapsedTime(&Pm->ms_phase[0], ev0, evc);
  cudaEventElapsedTime(&Pm->ms_phase[1], evc, evs);
  cudaEventElapsedTime(&Pm->ms_phase[2], evs, ev1);
  dev_free(counts);
  dev_free(err);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  cudaEventDestroy(evc);
  cudaEventDestroy(evs);
  grid_retain(g);  // P0 keeps its lattice alive
  *out = Pm;
  return WPCD_OK;
}

}  // namespace wpcd
