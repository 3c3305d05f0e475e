// Grouped solve over problems of uneven size: the iteration of the matrix
// Faddeev equation (Sec. 3.3, Eq. m_pvg, with K = O P0 Vt G1 of Eq. kernel)
// for n_prob problems whose packet grids differ, each with its own energies,
// run as ONE launch per operation over all of them.  The paper reuses one
// P0 for many energies; here many P0 matrices of different sizes share every
// launch as well, so small grids do not leave the GPU idle.
//
//   ggemm_kernel  persistent CTAs walk one list of 32 x 64 output tiles over
//                 (problem, channel, row tile, column tile) of the Vt and O
//                 block products
//   gspmm_kernel  warps walk the concatenated row space of all P0 matrices;
//                 each row finds its problem by binary search over the row
//                 offsets (held in shared memory)
//   ggemm_df_kernel / gspmm_df_kernel  the same two walks in float-float
//                 (hi + lo floats) for the refinement residual
//   gdot / gaxpy / gscale / gupdate ...  Krylov vector kernels over the
//                 concatenated segments; an element finds its system
//                 (problem, energy) by binary search over segment offsets
//
// Device layout: problem g's segment starts at complex element eoff[g] and
// holds its dim_g x B_g block with the energy index innermost (r * B_g + e,
// r = ch*N*M + k*M + j), the single-problem batched layout.  Systems
// (problem, energy) are numbered sys[g] + e; each keeps its own G1, Krylov
// basis and least-squares state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "df_common.cuh"
#include "wpcd_internal.h"

namespace wpcd {
namespace {

constexpr int kMaxGroup = WPCD_GROUP_MAX;
constexpr int kMaxGroupE = WPCD_GROUP_MAX_E;  // energies per problem (one warp of lanes)
constexpr int GV_THREADS = 256;
constexpr int GJC = 8;  // basis vectors per pass of the dot kernel

// offsets of the group (device memory, read into shared memory by kernels)
struct GMeta {
  int n = 0, S = 0;                 // problems, systems
  int64_t eoff[kMaxGroup + 1];      // complex element offset of each segment
  int B[kMaxGroup];                 // energies per problem
  int sys[kMaxGroup + 1];           // first system of each problem
  int tile_off[kMaxGroup + 1];      // first GEMM tile of each problem
  int dtile_off[kMaxGroup + 1];     // first float-float GEMM tile (32 x 128) of each problem
  int cell_off[kMaxGroup + 1];      // first P0 row of each problem
  int blk_off[kMaxGroup + 1];       // first dot-product block of each problem
};

// one problem's operands (device pointers)
struct alignas(16) GProb {
  int N, M, B, n_cells, rt, ct;     // grid, energies, cells, GEMM tiles per channel
  int dct, pad_;                    // float-float GEMM column tiles per channel
  int64_t eoff, nnz;
  const int64_t *row_ptr;
  const int32_t *col;
  const double *val64;              // FP64 P0 values (FP64 assembly) or NULL
  const float *val32;               // FP32 P0 values (FP32C assembly, or the FP32 copy)
  const double *O, *Vt;
  const float *O32, *Vt32;
  const float *O_h, *O_l, *Vt_h, *Vt_l;  // float-float splits of O and Vt
  const float *val_h, *val_l;            // float-float P0 values (val_l NULL for FP32C values)
};

// largest g in [0, n) with off[g] <= x
template <typename I>
__device__ __forceinline__ int seg_of(const I *off, int n, I x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// segment offsets, energies and first systems in shared memory
struct SegSmem {
  int64_t off[kMaxGroup + 1];
  int B[kMaxGroup];
  int sys[kMaxGroup];
};

__device__ __forceinline__ void load_segs(const GMeta *__restrict__ gm, SegSmem &sm) {
  const int n = gm->n;
  for (int i = threadIdx.x; i <= n; i += blockDim.x) {
    sm.off[i] = gm->eoff[i];
    if (i < n) {
      sm.B[i] = gm->B[i];
      sm.sys[i] = gm->sys[i];
    }
  }
  __syncthreads();
}

// system of complex element f of a concatenated vector
__device__ __forceinline__ int system_of(const SegSmem &sm, int n, int64_t f) {
  const int g = seg_of(sm.off, n, f);
  return sm.sys[g] + (int)((f - sm.off[g]) % sm.B[g]);
}

template <typename T>
__device__ __forceinline__ const T *mat_of(const GProb &P, bool O);
template <>
__device__ __forceinline__ const double *mat_of<double>(const GProb &P, bool O) {
  return O ? P.O : P.Vt;
}
template <>
__device__ __forceinline__ const float *mat_of<float>(const GProb &P, bool O) {
  return O ? P.O32 : P.Vt32;
}

// ---------------------------------------------------------------------------
// grouped block GEMM: for every (problem, channel) C = A B' (A = Vt or O)
// ---------------------------------------------------------------------------
template <typename T, bool SCALE_G, bool SUB>
__global__ void __launch_bounds__(G_THREADS) ggemm_kernel(const GMeta *__restrict__ gm,
                                                             const GProb *__restrict__ gp, int use_O,
                                                             const T *__restrict__ X, const T *__restrict__ G,
                                                             const T *__restrict__ S, T *__restrict__ C) {
  __shared__ GemmSmem<T> sm;
  __shared__ int toff[kMaxGroup + 1];
  const int n = gm->n;
  for (int i = threadIdx.x; i <= n; i += blockDim.x) toff[i] = gm->tile_off[i];
  __syncthreads();
  const int total = toff[n];
  // the loop bound is the same for the whole CTA (gemm_tile synchronises)
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int g = seg_of(toff, n, t);
    const GProb &P = gp[g];
    const int N = P.N, ct = P.ct;
    const int lt = t - toff[g];
    const int per_ch = P.rt * ct;
    const int ch = lt / per_ch, rem = lt % per_ch;
    const int64_t ncol = 2LL * P.M * P.B;
    const T *A = mat_of<T>(P, use_O != 0) + (size_t)ch * N * N;
    const size_t base = 2 * (size_t)P.eoff + (size_t)ch * N * ncol;
    gemm_tile<T, SCALE_G, SUB>(N, ncol, A, X + base, SCALE_G ? G + base : nullptr, SUB ? S + base : nullptr,
                               C + base, (rem / ct) * GB_M, (int64_t)(rem % ct) * GB_N, sm);
  }
}

// ---------------------------------------------------------------------------
// grouped block-CSR SpMM: Z[l][c][e] = sum P0[(l,c),(l',c')] Y[l'][c'][e] for
// every problem; the lane layout of a warp is the single-problem one (rows
// per warp, energy lanes, nonzero lanes, energies per lane)
// ---------------------------------------------------------------------------
template <typename VT>
__device__ __forceinline__ const VT *vals_of(const GProb &P);
template <>
__device__ __forceinline__ const double *vals_of<double>(const GProb &P) {
  return P.val64;
}
template <>
__device__ __forceinline__ const float *vals_of<float>(const GProb &P) {
  return P.val32;
}

// SACC (FP32): compensated sums in dynamic shared memory, as in the
// single-problem SpMM
template <typename VT, typename T, int NCH, int EPT, bool VEC, bool SACC>
__device__ __forceinline__ void gspmm_body(const GMeta *__restrict__ gm, const GProb *__restrict__ gp, int rpw,
                                           int el_n, const typename Cx<T>::t *__restrict__ y,
                                           typename Cx<T>::t *__restrict__ z, float *acc_sm) {
  using C2 = typename Cx<T>::t;
  using Acc = typename AccOf<T>::t;
  __shared__ int coff[kMaxGroup + 1];
  __shared__ GProb sp[kMaxGroup];
  const int n = gm->n;
  for (int i = threadIdx.x; i <= n; i += blockDim.x) {
    coff[i] = gm->cell_off[i];
    if (i < n) sp[i] = gp[i];
  }
  __syncthreads();
  const int total = coff[n];
  const int lane = threadIdx.x & 31;
  const int lpr = 32 / rpw;         // lanes per row
  const int nl_count = lpr / el_n;  // nonzero lanes per row
  const int r_in = lane / lpr, sub = lane % lpr;
  const int el = sub % el_n, nl = sub / el_n;
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int n_warps = gridDim.x * blockDim.x / 32;
  const int e_base = blockIdx.y * el_n * EPT;
  // the loop bound depends on the warp only, so every lane reaches the
  // full-mask shuffles below; the rows of one warp may belong to two problems
  for (int base = warp_global * rpw; base < total; base += n_warps * rpw) {
    const int R = base + r_in;
    const bool active = R < total;
    const int g = active ? seg_of(coff, n, R) : 0;
    const GProb &P = sp[g];
    const int c = R - coff[g];
    const int B = P.B, n_cells = P.n_cells;
    const C2 *yg = y + P.eoff;
    const VT *val = vals_of<VT>(P);
    Acc acc[NCH][EPT][2];
    const int64_t b = active ? P.row_ptr[c] : 0, e = active ? P.row_ptr[c + 1] : 0;
    // lane energies: strided (el + el_n t); with VEC in adjacent pairs
    // (2 el + el_n (t - t % 2) + t % 2), one 16-byte gather covering 16 el_n
    // contiguous bytes of a vector row
    const int en0 = VEC ? e_base + 2 * el : e_base + el, estride = el_n;
    spmm_row_sums<VT, T, NCH, EPT, VEC, SACC>(b, e, nl, nl_count, P.col, val, P.nnz, yg, n_cells, B, en0, estride,
                                              acc, acc_sm);
    for (int off = el_n; off < lpr; off <<= 1)
#pragma unroll
      for (int l = 0; l < NCH; ++l)
#pragma unroll
        for (int t = 0; t < EPT; ++t) {
          acc[l][t][0].add_shfl(off);
          acc[l][t][1].add_shfl(off);
        }
    if (active && nl == 0) {
      C2 *zg = z + P.eoff;
#pragma unroll
      for (int t = 0; t < EPT; ++t) {
        const int en = VEC ? e_base + 2 * el + el_n * (t & ~1) + (t & 1) : e_base + el + el_n * t;
        if (en < B)
#pragma unroll
          for (int l = 0; l < NCH; ++l) {
            C2 out;
            out.x = (T)acc[l][t][0].value();
            out.y = (T)acc[l][t][1].value();
            zg[((size_t)l * n_cells + c) * B + en] = out;
          }
      }
    }
  }
}

template <typename VT, typename T, int NCH, int EPT, bool VEC>
__global__ void __launch_bounds__(256) gspmm_kernel(const GMeta *__restrict__ gm, const GProb *__restrict__ gp,
                                                    int rpw, int el_n, const typename Cx<T>::t *__restrict__ y,
                                                    typename Cx<T>::t *__restrict__ z) {
  gspmm_body<VT, T, NCH, EPT, VEC, false>(gm, gp, rpw, el_n, y, z, nullptr);
}

template <int NCH, int EPT, bool VEC>
__global__ void __launch_bounds__(256, 2)
    gspmm_sacc_kernel(const GMeta *__restrict__ gm, const GProb *__restrict__ gp, int rpw, int el_n,
                      const float2 *__restrict__ y, float2 *__restrict__ z) {
  extern __shared__ float acc_sm[];
  gspmm_body<float, float, NCH, EPT, VEC, true>(gm, gp, rpw, el_n, y, z, acc_sm);
}

template <int NCH, int EPT, bool VEC>
cudaError_t gspmm_sacc_smem(size_t *bytes) {
  static bool opted_in = false;
  return sacc_smem<NCH, EPT>(gspmm_sacc_kernel<NCH, EPT, VEC>, bytes, opted_in,
                             sizeof(int) * (kMaxGroup + 1) + sizeof(GProb) * kMaxGroup);
}

// ---------------------------------------------------------------------------
// grouped float-float operators for the refinement residual: the same tile
// list and row walk, with hi + lo float operands (exact splits of the FP64
// values) and float-float accumulation
// ---------------------------------------------------------------------------
template <bool OUT_DF>
__global__ void __launch_bounds__(G_THREADS) ggemm_df_kernel(const GMeta *__restrict__ gm,
                                                                const GProb *__restrict__ gp, int use_O,
                                                                const float *__restrict__ Xh,
                                                                const float *__restrict__ Xl, double *__restrict__ C,
                                                                float *__restrict__ Ch, float *__restrict__ Cl) {
  __shared__ DfGemmSmem sm;
  __shared__ int toff[kMaxGroup + 1];
  const int n = gm->n;
  for (int i = threadIdx.x; i <= n; i += blockDim.x) toff[i] = gm->dtile_off[i];
  __syncthreads();
  const int total = toff[n];
  for (int t = blockIdx.x; t < total; t += gridDim.x) {  // uniform per CTA
    const int g = seg_of(toff, n, t);
    const GProb &P = gp[g];
    const int N = P.N, ct = P.dct;
    const int lt = t - toff[g];
    const int per_ch = P.rt * ct;
    const int ch = lt / per_ch, rem = lt % per_ch;
    const int64_t ncol = 2LL * P.M * P.B;
    const size_t ao = (size_t)ch * N * N;
    const float *Ah = (use_O ? P.O_h : P.Vt_h) + ao, *Al = (use_O ? P.O_l : P.Vt_l) + ao;
    const size_t base = 2 * (size_t)P.eoff + (size_t)ch * N * ncol;
    gemm_df_tile<OUT_DF>(N, ncol, Ah, Al, Xh + base, Xl + base, OUT_DF ? nullptr : C + base,
                         OUT_DF ? Ch + base : nullptr, OUT_DF ? Cl + base : nullptr, (rem / ct) * GB_M,
                         (int64_t)(rem % ct) * DF_N, sm);
  }
}

template <int NCH, int EPT>
__global__ void __launch_bounds__(256) gspmm_df_kernel(const GMeta *__restrict__ gm, const GProb *__restrict__ gp,
                                                       int rpw, int el_n, const float2 *__restrict__ yh,
                                                       const float2 *__restrict__ yl, float2 *__restrict__ zh,
                                                       float2 *__restrict__ zl) {
  __shared__ int coff[kMaxGroup + 1];
  __shared__ GProb sp[kMaxGroup];
  const int n = gm->n;
  for (int i = threadIdx.x; i <= n; i += blockDim.x) {
    coff[i] = gm->cell_off[i];
    if (i < n) sp[i] = gp[i];
  }
  __syncthreads();
  const int total = coff[n];
  const int lane = threadIdx.x & 31;
  const int lpr = 32 / rpw, nl_count = lpr / el_n;
  const int r_in = lane / lpr, sub = lane % lpr;
  const int el = sub % el_n, nl = sub / el_n;
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int n_warps = gridDim.x * blockDim.x / 32;
  const int e_base = blockIdx.y * el_n * EPT;
  // warp-uniform loop bound: every lane reaches the full-mask shuffles
  for (int base = warp_global * rpw; base < total; base += n_warps * rpw) {
    const int R = base + r_in;
    const bool active = R < total;
    const int g = active ? seg_of(coff, n, R) : 0;
    const GProb &P = sp[g];
    const int c = R - coff[g];
    float ah[NCH][EPT][2], al[NCH][EPT][2];
#pragma unroll
    for (int l = 0; l < NCH; ++l)
#pragma unroll
      for (int t = 0; t < EPT; ++t) ah[l][t][0] = ah[l][t][1] = al[l][t][0] = al[l][t][1] = 0.f;
    const int64_t b = active ? P.row_ptr[c] : 0, e = active ? P.row_ptr[c + 1] : 0;
    spmm_df_row<NCH, EPT>(b, e, nl, nl_count, P.col, P.val_h, P.val_l, P.nnz, yh + P.eoff, yl + P.eoff, P.n_cells,
                          P.B, e_base + el, el_n, ah, al);
    spmm_df_finish<NCH, EPT>(el_n, lpr, active && nl == 0, ah, al, zh + P.eoff, zl + P.eoff, P.n_cells, c, P.B,
                             e_base + el, el_n);
  }
}

// Vt e0 for every system in float-float (the splits of gborn_vt_kernel's values)
__global__ void gborn_vt_df_kernel(const GMeta *__restrict__ gm, const GProb *__restrict__ gp, int64_t len,
                                   const int *__restrict__ j0, float2 *__restrict__ yh, float2 *__restrict__ yl) {
  __shared__ SegSmem sm;
  load_segs(gm, sm);
  const int n = gm->n;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < len; f += (int64_t)gridDim.x * blockDim.x) {
    const int g = seg_of(sm.off, n, f);
    const int B = sm.B[g];
    const int64_t loc = f - sm.off[g];
    const int e = (int)(loc % B);
    const int64_t r = loc / B;
    const int N = gp[g].N, M = gp[g].M;
    float h = 0.f, l = 0.f;
    if (r < (int64_t)N * M && (int)(r % M) == j0[sm.sys[g] + e]) {
      h = gp[g].Vt_h[(r / M) * N];
      l = gp[g].Vt_l[(r / M) * N];
    }
    yh[f] = make_float2(h, 0.f);
    yl[f] = make_float2(l, 0.f);
  }
}

// ---------------------------------------------------------------------------
// segmented Krylov vector kernels (scalars per system in FP64)
// ---------------------------------------------------------------------------
// partial[((j * NBT) + blk) * 32 + e] = sum over blk's rows of conj(V_j) w,
// blocks blk_off[g] .. blk_off[g+1]-1 serve problem g; block (EL, RB) with
// EL >= the problem's energies
// partial[blk * kMaxGroupE + e] = (sum over blk's rows of |x|^2, 0): the norm
// pass of gdot_kernel, one vector read once, four rows in flight per thread
template <typename T>
__global__ void __launch_bounds__(GV_THREADS) gnorm_kernel(const GMeta *__restrict__ gm,
                                                           const typename Cx<T>::t *__restrict__ x,
                                                           double2 *__restrict__ partial) {
  __shared__ double red[GV_THREADS];
  const int EL = blockDim.x, RB = blockDim.y;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * EL + tx;
  const int n = gm->n;
  const int g = seg_of(gm->blk_off, n, (int)blockIdx.x);
  const int nb = gm->blk_off[g + 1] - gm->blk_off[g], lb = blockIdx.x - gm->blk_off[g];
  const int B = gm->B[g];
  const int64_t off = gm->eoff[g];
  const int rows = (int)((gm->eoff[g + 1] - off) / B);
  const int stride = nb * RB;
  T acc = T(0);
  if (tx < B) {
    int r = lb * RB + ty;
    for (; r + 3 * stride < rows; r += 4 * stride) {
      typename Cx<T>::t a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = x[(size_t)off + (size_t)(r + u * stride) * B + tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc = fma(a[u].x, a[u].x, fma(a[u].y, a[u].y, acc));
    }
    for (; r < rows; r += stride) {
      const auto a = x[(size_t)off + (size_t)r * B + tx];
      acc = fma(a.x, a.x, fma(a.y, a.y, acc));
    }
  }
  red[tid] = (double)acc;
  __syncthreads();
  for (int h = RB / 2; h > 0; h >>= 1) {
    if (ty < h) red[tid] += red[(ty + h) * EL + tx];
    __syncthreads();
  }
  if (ty == 0 && tx < B) partial[(size_t)blockIdx.x * kMaxGroupE + tx] = make_double2(red[tx], 0.0);
}

template <typename T>
__global__ void __launch_bounds__(GV_THREADS) gdot_kernel(const GMeta *__restrict__ gm, int nv,
                                                          const typename Cx<T>::t *__restrict__ V, size_t ld,
                                                          const typename Cx<T>::t *__restrict__ w,
                                                          double2 *__restrict__ partial) {
  __shared__ double2 red[GJC][GV_THREADS];
  const int EL = blockDim.x, RB = blockDim.y;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * EL + tx;
  const int n = gm->n;
  const int g = seg_of(gm->blk_off, n, (int)blockIdx.x);
  const int nb = gm->blk_off[g + 1] - gm->blk_off[g], lb = blockIdx.x - gm->blk_off[g];
  const int B = gm->B[g];
  const int64_t off = gm->eoff[g];
  const int rows = (int)((gm->eoff[g + 1] - off) / B);
  const int NBT = gridDim.x;
  for (int j0 = 0; j0 < nv; j0 += GJC) {
    T sx[GJC], sy[GJC];
#pragma unroll
    for (int c = 0; c < GJC; ++c) sx[c] = sy[c] = T(0);
    if (tx < B) {
      for (int r = lb * RB + ty; r < rows; r += nb * RB) {
        const size_t f = (size_t)off + (size_t)r * B + tx;
        const auto b = w[f];
#pragma unroll
        for (int c = 0; c < GJC; ++c) {
          if (j0 + c < nv) {
            const auto a = V[(size_t)(j0 + c) * ld + f];
            sx[c] = fma(a.x, b.x, fma(a.y, b.y, sx[c]));
            sy[c] = fma(a.x, b.y, fma(-a.y, b.x, sy[c]));
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < GJC; ++c) red[c][tid] = make_double2((double)sx[c], (double)sy[c]);
    __syncthreads();
    for (int h = RB / 2; h > 0; h >>= 1) {
      if (ty < h)
#pragma unroll
        for (int c = 0; c < GJC; ++c) {
          double2 o = red[c][(ty + h) * EL + tx];
          red[c][tid].x += o.x;
          red[c][tid].y += o.y;
        }
      __syncthreads();
    }
    if (ty == 0 && tx < B)
#pragma unroll
      for (int c = 0; c < GJC; ++c)
        if (j0 + c < nv) partial[((size_t)(j0 + c) * NBT + blockIdx.x) * kMaxGroupE + tx] = red[c][tx];
    __syncthreads();
  }
}

// out[j * S + s] (+)= sum of system s's block partials; also, in the vector
// precision T, coef = sign * (this pass's sum) and, for a norm pass,
// inv = 1 / sqrt(sum.x) (0 for a zero norm)
template <typename T>
__global__ void greduce_kernel(const GMeta *__restrict__ gm, int nv, int NBT, const double2 *__restrict__ partial,
                               double2 *__restrict__ out, int accumulate, typename Cx<T>::t *coef, double sign,
                               T *inv) {
  // one warp per output (j, s): the lanes stride over the problem's blocks
  const int S = gm->S;
  const int idx = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (idx >= nv * S) return;  // warp-uniform
  const int j = idx / S, s = idx % S;
  const int g = seg_of(gm->sys, gm->n, s);
  const int e = s - gm->sys[g];
  double sx = 0.0, sy = 0.0;
  for (int b = gm->blk_off[g] + lane; b < gm->blk_off[g + 1]; b += 32) {
    const double2 p = partial[((size_t)j * NBT + b) * kMaxGroupE + e];
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

// w[f] += sum_j c[j * S + s(f)] V_j[f]   (coefficients in the vector precision)
template <typename T>
__global__ void gaxpy_kernel(const GMeta *__restrict__ gm, int64_t len, int nv,
                             const typename Cx<T>::t *__restrict__ V, size_t ld,
                             const typename Cx<T>::t *__restrict__ c, typename Cx<T>::t *__restrict__ w) {
  __shared__ SegSmem sm;
  load_segs(gm, sm);
  const int n = gm->n, S = gm->S;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < len; f += (int64_t)gridDim.x * blockDim.x) {
    const int s = system_of(sm, n, f);
    T ax = w[f].x, ay = w[f].y;
    for (int j = 0; j < nv; ++j) {
      const auto a = V[(size_t)j * ld + f];
      const auto cj = c[(size_t)j * S + s];
      ax = fma(cj.x, a.x, fma(-cj.y, a.y, ax));
      ay = fma(cj.x, a.y, fma(cj.y, a.x, ay));
    }
    w[f].x = ax;
    w[f].y = ay;
  }
}

// the FP32 axpy of an even group (every B_g and segment offset even): two
// adjacent energies of one row per thread in 16-byte loads; len2 = len / 2
// (NVT > 0: at most NVT vectors, every vector's load for the element issued
// before the multiply-adds, the sums in the same order)
template <int NVT>
__global__ void gaxpy2_kernel(const GMeta *__restrict__ gm, int64_t len2, int nv, const float4 *__restrict__ V,
                              size_t ld2, const float4 *__restrict__ c, float4 *__restrict__ w) {
  __shared__ SegSmem sm;
  load_segs(gm, sm);
  const int n = gm->n, S2 = gm->S / 2;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < len2;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int s2 = system_of(sm, n, 2 * f) / 2;  // even system of the pair
    float4 a = w[f];
    const auto mac = [&](const float4 &v, const float4 &cj) {
      a.x = fmaf(cj.x, v.x, fmaf(-cj.y, v.y, a.x));
      a.y = fmaf(cj.x, v.y, fmaf(cj.y, v.x, a.y));
      a.z = fmaf(cj.z, v.z, fmaf(-cj.w, v.w, a.z));
      a.w = fmaf(cj.z, v.w, fmaf(cj.w, v.z, a.w));
    };
    if constexpr (NVT > 0) {
      float4 v[NVT];
#pragma unroll
      for (int j = 0; j < NVT; ++j) v[j] = j < nv ? V[(size_t)j * ld2 + f] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 0; j < NVT; ++j)
        if (j < nv) mac(v[j], c[(size_t)j * S2 + s2]);
    } else {
      for (int j = 0; j < nv; ++j) mac(V[(size_t)j * ld2 + f], c[(size_t)j * S2 + s2]);
    }
    w[f] = a;
  }
}

// dst[f] = src[f] * inv[s(f)]
template <typename T>
__global__ void gscale_kernel(const GMeta *__restrict__ gm, int64_t len, const typename Cx<T>::t *src,
                              const T *__restrict__ inv, typename Cx<T>::t *dst) {
  __shared__ SegSmem sm;
  load_segs(gm, sm);
  const int n = gm->n;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < len; f += (int64_t)gridDim.x * blockDim.x) {
    const T sc = inv[system_of(sm, n, f)];
    dst[f].x = src[f].x * sc;
    dst[f].y = src[f].y * sc;
  }
}

// dst32[f] = (float)(src[f] * inv[s(f)])
__global__ void gnormalize_f32_kernel(const GMeta *__restrict__ gm, int64_t len, const double2 *__restrict__ src,
                                      const double *__restrict__ inv, float2 *__restrict__ dst) {
  __shared__ SegSmem sm;
  load_segs(gm, sm);
  const int n = gm->n;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < len; f += (int64_t)gridDim.x * blockDim.x) {
    const double sc = inv[system_of(sm, n, f)];
    dst[f] = make_float2(f64_to_f32_rn(src[f].x * sc), f64_to_f32_rn(src[f].y * sc));
  }
}

// u[f] += sum_j c[j * S + s] V_j[f]: the correction formed in the basis
// precision T (coefficients from bupdate_coef_kernel), added to u in FP64
template <typename T>
__global__ void gupdate_kernel(const GMeta *__restrict__ gm, int64_t len, int k,
                               const typename Cx<T>::t *__restrict__ V, size_t ld,
                               const typename Cx<T>::t *__restrict__ c, double2 *__restrict__ u) {
  __shared__ SegSmem sm;
  load_segs(gm, sm);
  const int n = gm->n, S = gm->S;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < len; f += (int64_t)gridDim.x * blockDim.x) {
    const int s = system_of(sm, n, f);
    T ax = T(0), ay = T(0);
    for (int j = 0; j < k; ++j) {
      const auto a = V[(size_t)j * ld + f];
      const auto cj = c[(size_t)j * S + s];
      ax = fma(cj.x, a.x, fma(-cj.y, a.y, ax));
      ay = fma(cj.x, a.y, fma(cj.y, a.x, ay));
    }
    u[f].x += (double)ax;
    u[f].y += (double)ay;
  }
}

// Vt e0 for every system: column 0 of the problem's Vt_0 at (channel 0, q-bin j0)
__global__ void gborn_vt_kernel(const GMeta *__restrict__ gm, const GProb *__restrict__ gp, int64_t len,
                                const int *__restrict__ j0, double2 *__restrict__ y) {
  __shared__ SegSmem sm;
  load_segs(gm, sm);
  const int n = gm->n;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < len; f += (int64_t)gridDim.x * blockDim.x) {
    const int g = seg_of(sm.off, n, f);
    const int B = sm.B[g];
    const int64_t loc = f - sm.off[g];
    const int e = (int)(loc % B);
    const int64_t r = loc / B;  // ch*N*M + i*M + j
    const int N = gp[g].N, M = gp[g].M;
    double v = 0.0;
    if (r < (int64_t)N * M && (int)(r % M) == j0[sm.sys[g] + e]) v = gp[g].Vt[(r / M) * N];
    y[f] = make_double2(v, 0.0);
  }
}

__global__ void gd2f_kernel(int64_t n, const double *__restrict__ src, float *__restrict__ dst) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x)
    dst[f] = f64_to_f32_rn(src[f]);
}

// S = 1 - 2 pi i U00 / D and the paper's A per system; out[s * 6 + ...]
__global__ void gamplitude_kernel(int S, const double2 *__restrict__ u, const int64_t *__restrict__ idx0,
                                  const double *__restrict__ D, const double *__restrict__ pref, double *out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double2 U = u[idx0[s]];
  double *o = out + 6 * (size_t)s;
  o[0] = U.x;
  o[1] = U.y;
  o[2] = 1.0 + 2.0 * kPi * U.y / D[s];
  o[3] = -2.0 * kPi * U.x / D[s];
  o[4] = pref[s] * U.x;
  o[5] = pref[s] * U.y;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// device memory from the library's stream-ordered pool, allocated and freed
// on the solve's stream
struct DevFree {
  std::vector<void *> p;
  cudaStream_t st = nullptr;
  template <typename T>
  cudaError_t alloc(T **out, size_t bytes) {
    void *q = nullptr;
    cudaError_t e = pool_malloc(&q, bytes, st);
    if (e == cudaSuccess) {
      p.push_back(q);
      *out = static_cast<T *>(q);
    }
    return e;
  }
  ~DevFree() {
    for (void *q : p) pool_free(q, st);
  }
};

struct Group {
  int n = 0, n_ch = 0, S = 0, prec = WPCD_FP64, Bmax = 1;
  bool even = true;        // every B_g and every segment offset even
  bool tc = false;         // FP32 block products on the tensor cores (tc_gemm_group)
  std::vector<TcGroupProb> tcp;
  int64_t L = 0;           // complex elements of one concatenated vector
  GMeta meta;              // host copy
  std::vector<GProb> probs;
  GMeta *d_meta = nullptr;
  GProb *d_probs = nullptr;
  SpmmConfig cfg64, cfg32, cfgff;
  dim3 dot_block() const {
    int el = 1;
    while (el < Bmax) el *= 2;
    return dim3(el, GV_THREADS / el);
  }
  int nbt() const { return meta.blk_off[n]; }
  int tiles() const { return meta.tile_off[n]; }
  int dtiles() const { return meta.dtile_off[n]; }
};

int gemm_grid(const Group &gr) { return std::max(1, std::min(gr.tiles(), 152 * 4)); }

// C = A X' per (problem, channel) in float-float; OUT_DF: C as (Ch, Cl)
template <bool OUT_DF>
void ggemm_df(const Group &gr, bool use_O, const float *Xh, const float *Xl, double *C, float *Ch, float *Cl,
              cudaStream_t s) {
  const int grid = std::max(1, std::min(gr.dtiles(), 152 * 2));
  ggemm_df_kernel<OUT_DF><<<grid, G_THREADS, 0, s>>>(gr.d_meta, gr.d_probs, use_O, Xh, Xl, C, Ch, Cl);
  count_launches(1);
}

wpcd_status gspmm_df_cfg(const Group &gr, const float *yh, const float *yl, float *zh, float *zl,
                         const SpmmConfig &cfg, cudaStream_t s) {
  const float2 *y2h = reinterpret_cast<const float2 *>(yh), *y2l = reinterpret_cast<const float2 *>(yl);
  float2 *z2h = reinterpret_cast<float2 *>(zh), *z2l = reinterpret_cast<float2 *>(zl);
  dim3 grid(grid_for((int64_t)gr.meta.cell_off[gr.n], 8 * cfg.rpw, 152 * 16),
            (gr.Bmax + cfg.el * cfg.ept - 1) / (cfg.el * cfg.ept));
#define WPCD_GDF_EPT(NCH, EPT) \
  gspmm_df_kernel<NCH, EPT><<<grid, 256, 0, s>>>(gr.d_meta, gr.d_probs, cfg.rpw, cfg.el, y2h, y2l, z2h, z2l)
#define WPCD_GDF_CASE(NCH)  \
  case NCH:                 \
    if (cfg.ept == 1)       \
      WPCD_GDF_EPT(NCH, 1); \
    else if (cfg.ept == 2)  \
      WPCD_GDF_EPT(NCH, 2); \
    else                    \
      WPCD_GDF_EPT(NCH, 4); \
    break;
  switch (gr.n_ch) {
    WPCD_GDF_CASE(1)
    WPCD_GDF_CASE(2)
    WPCD_GDF_CASE(3)
    WPCD_GDF_CASE(4)
    WPCD_GDF_CASE(5)
    default:
      return set_error(WPCD_EINVAL, "unsupported channel count for the SpMM");
  }
#undef WPCD_GDF_CASE
#undef WPCD_GDF_EPT
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "grouped float-float spmm launch");
}

template <typename T>
void ggemm(const Group &gr, bool use_O, bool scale_g, bool sub, const T *X, const T *G, const T *S, T *C,
           cudaStream_t s) {
  const int grid = gemm_grid(gr);
  if (scale_g)
    ggemm_kernel<T, true, false><<<grid, G_THREADS, 0, s>>>(gr.d_meta, gr.d_probs, use_O, X, G, nullptr, C);
  else if (sub)
    ggemm_kernel<T, false, true><<<grid, G_THREADS, 0, s>>>(gr.d_meta, gr.d_probs, use_O, X, nullptr, S, C);
  else
    ggemm_kernel<T, false, false><<<grid, G_THREADS, 0, s>>>(gr.d_meta, gr.d_probs, use_O, X, nullptr, nullptr, C);
  count_launches(1);
}

template <typename VT, typename T>
wpcd_status gspmm_cfg(const Group &gr, const T *y, T *z, const SpmmConfig &cfg, cudaStream_t s) {
  using C2 = typename Cx<T>::t;
  const C2 *yy = reinterpret_cast<const C2 *>(y);
  C2 *zz = reinterpret_cast<C2 *>(z);
  const int rows_per_block = 8 * cfg.rpw;
  dim3 grid(grid_for((int64_t)gr.meta.cell_off[gr.n], rows_per_block, 152 * 16),
            (gr.Bmax + cfg.el * cfg.ept - 1) / (cfg.el * cfg.ept));
  // FP32 vectors, every batch even and every segment 16-byte aligned: two
  // adjacent energies per load
  const bool vec = sizeof(T) == 4 && gr.even;
  // FP32 (values and vectors): compensated sums in shared memory
  constexpr bool sacc = sizeof(T) == 4 && sizeof(VT) == 4;
#define WPCD_GSPMM_EPT(NCH, EPT, VEC)                                                                        \
  do {                                                                                                       \
    if constexpr (sacc) {                                                                                    \
      size_t smem = 0;                                                                                       \
      cudaError_t ae = gspmm_sacc_smem<NCH, EPT, VEC>(&smem);                                                \
      if (ae != cudaSuccess) return cuda_error(ae, "grouped spmm shared-memory attribute");                  \
      gspmm_sacc_kernel<NCH, EPT, VEC><<<grid, 256, smem, s>>>(gr.d_meta, gr.d_probs, cfg.rpw, cfg.el,       \
                                                               reinterpret_cast<const float2 *>(yy),         \
                                                               reinterpret_cast<float2 *>(zz));              \
    } else {                                                                                                 \
      gspmm_kernel<VT, T, NCH, EPT, VEC><<<grid, 256, 0, s>>>(gr.d_meta, gr.d_probs, cfg.rpw, cfg.el, yy, zz); \
    }                                                                                                        \
  } while (0)
#define WPCD_GSPMM_CASE(NCH)                                                         \
  case NCH:                                                                          \
    if (cfg.ept == 1)                                                                \
      WPCD_GSPMM_EPT(NCH, 1, false);                                                 \
    else if (cfg.ept == 2) {                                                         \
      if (vec)                                                                       \
        WPCD_GSPMM_EPT(NCH, 2, sizeof(T) == 4);                                      \
      else                                                                           \
        WPCD_GSPMM_EPT(NCH, 2, false);                                               \
    } else {                                                                         \
      if (vec)                                                                       \
        WPCD_GSPMM_EPT(NCH, 4, sizeof(T) == 4);                                      \
      else                                                                           \
        WPCD_GSPMM_EPT(NCH, 4, false);                                               \
    }                                                                                \
    break;
  switch (gr.n_ch) {
    WPCD_GSPMM_CASE(1)
    WPCD_GSPMM_CASE(2)
    WPCD_GSPMM_CASE(3)
    WPCD_GSPMM_CASE(4)
    WPCD_GSPMM_CASE(5)
    default:
      return set_error(WPCD_EINVAL, "unsupported channel count for the SpMM");
  }
#undef WPCD_GSPMM_CASE
#undef WPCD_GSPMM_EPT
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "grouped spmm launch");
}

// FP64 vectors use the group's own P0 precision; FP32 vectors the FP32 values
template <typename T>
wpcd_status gspmm(const Group &gr, const T *y, T *z, const SpmmConfig &cfg, cudaStream_t s) {
  if (sizeof(T) == 4) return gspmm_cfg<float, float>(gr, (const float *)y, (float *)z, cfg, s);
  if (gr.prec == WPCD_FP64) return gspmm_cfg<double, double>(gr, (const double *)y, (double *)z, cfg, s);
  return gspmm_cfg<float, double>(gr, (const double *)y, (double *)z, cfg, s);
}

// tuned launch shapes, keyed by the group's shape
std::mutex g_gtune_mutex;
std::map<std::string, SpmmConfig> g_gtuned;

std::string group_key(const Group &gr, int mode) {
  std::string k = std::to_string(gr.n_ch) + "/" + std::to_string(gr.prec) + "/" + std::to_string(mode);
  for (int g = 0; g < gr.n; ++g)
    k += ":" + std::to_string(gr.probs[g].N) + "x" + std::to_string(gr.probs[g].M) + "b" +
         std::to_string(gr.probs[g].B) + "n" + std::to_string(gr.probs[g].nnz);
  return k;
}

// time every candidate shape on the whole group (3 launches each, CUDA
// events, the minimum kept) with run(cfg); mode 0 FP64, 1 FP32, 2
// float-float; the caller zeroes the input vectors; outside stream capture
template <typename Run>
wpcd_status gtune(const Group &gr, int mode, Run run, cudaStream_t s, SpmmConfig *out) {
  std::lock_guard<std::mutex> lock(g_gtune_mutex);
  const std::string key = group_key(gr, mode);
  auto it = g_gtuned.find(key);
  if (it != g_gtuned.end()) {
    *out = it->second;
    return WPCD_OK;
  }
  cudaEvent_t a, b;
  WPCD_CUDA_TRY(cudaEventCreate(&a));
  WPCD_CUDA_TRY(cudaEventCreate(&b));
  float best = 1e30f;
  SpmmConfig pick;
  wpcd_status st = WPCD_OK;
  for (const SpmmConfig &c : candidates(gr.Bmax)) {
    float tmin = 1e30f;
    for (int rep = 0; rep < 3 && st == WPCD_OK; ++rep) {
      cudaEventRecord(a, s);
      st = run(c);
      cudaEventRecord(b, s);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      tmin = std::min(tmin, ms);
    }
    if (st != WPCD_OK) break;
    if (tmin < best) {
      best = tmin;
      pick = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != WPCD_OK) return st;
  g_gtuned[key] = pick;
  *out = pick;
  return WPCD_OK;
}

// out = O P0 Vt (g o x)  or  out = sub - O P0 Vt (g o x) for every system
template <typename T>
wpcd_status gkapply(const Group &gr, const T *g, const T *x, T *out, const T *sub, T *wy, T *wz,
                    cudaStream_t s) {
  if (sizeof(T) == 4 && gr.tc) {  // FP32: both block products on the tensor cores, one launch each
    const float *gf = reinterpret_cast<const float *>(g), *xf = reinterpret_cast<const float *>(x);
    wpcd_status st = tc_gemm_group(gr.tcp.data(), gr.n, false, gf, xf, nullptr, reinterpret_cast<float *>(wy), s);
    if (st == WPCD_OK) st = gspmm<T>(gr, wy, wz, gr.cfg32, s);
    if (st == WPCD_OK)
      st = tc_gemm_group(gr.tcp.data(), gr.n, true, nullptr, reinterpret_cast<const float *>(wz),
                         reinterpret_cast<const float *>(sub), reinterpret_cast<float *>(out), s);
    return st;
  }
  ggemm<T>(gr, false, g != nullptr, false, x, g, nullptr, wy, s);
  wpcd_status st = gspmm<T>(gr, wy, wz, sizeof(T) == 4 ? gr.cfg32 : gr.cfg64, s);
  if (st != WPCD_OK) return st;
  ggemm<T>(gr, true, false, sub != nullptr, wz, nullptr, sub, out, s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "grouped kapply launch");
}

// float-float work vectors of the grouped residual (2 L floats each)
struct GDf {
  float *xh = nullptr, *xl = nullptr, *yh = nullptr, *yl = nullptr;
};

// out = O P0 Vt (g o x) for every system in float-float, FP64 in and out
wpcd_status gkapply_df(const Group &gr, const double *g, const double *x, double *out, const GDf &w,
                       cudaStream_t s) {
  df_split_scaled_kernel<<<grid_for(gr.L, 256), 256, 0, s>>>(gr.L, reinterpret_cast<const double2 *>(x),
                                                            reinterpret_cast<const double2 *>(g), w.xh, w.xl);
  count_launches(1);
  ggemm_df<true>(gr, false, w.xh, w.xl, nullptr, w.yh, w.yl, s);
  wpcd_status st = gspmm_df_cfg(gr, w.yh, w.yl, w.xh, w.xl, gr.cfgff, s);
  if (st != WPCD_OK) return st;
  ggemm_df<false>(gr, true, w.xh, w.xl, out, nullptr, nullptr, s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "grouped float-float kapply launch");
}

// Krylov bases and least-squares state of all systems
template <typename T>
struct GKrylov {
  using C2 = typename Cx<T>::t;
  const Group *gr = nullptr;
  int m = 0, S = 0;
  int64_t L = 0;
  T *V = nullptr, *w = nullptr;  // [(m+1)][L], [L] complex
  double2 *H = nullptr, *cs = nullptr, *sn = nullptr, *bet = nullptr;
  double2 *h = nullptr, *h2 = nullptr, *nrm = nullptr, *y = nullptr, *partial = nullptr;
  double *resid = nullptr, *bnorm = nullptr;
  C2 *hc = nullptr;  // axpy / update coefficients in T [(m+1)][S]
  T *inv = nullptr;  // 1 / norm per system in T [S]
  DevFree mem;
  cudaError_t alloc(const Group &g, int m_, cudaStream_t s, bool vectors = true) {
    gr = &g;
    mem.st = s;
    m = m_;
    S = g.S;
    L = g.L;
    cudaError_t e;
    if (vectors) {
      if ((e = mem.alloc(&V, 2 * sizeof(T) * (size_t)L * (m + 1))) != cudaSuccess) return e;
      if ((e = mem.alloc(&w, 2 * sizeof(T) * (size_t)L)) != cudaSuccess) return e;
    }
    if ((e = mem.alloc(&H, sizeof(double2) * (size_t)S * (m + 1) * m)) != cudaSuccess) return e;
    if ((e = mem.alloc(&cs, sizeof(double2) * (size_t)S * m)) != cudaSuccess) return e;
    if ((e = mem.alloc(&sn, sizeof(double2) * (size_t)S * m)) != cudaSuccess) return e;
    if ((e = mem.alloc(&bet, sizeof(double2) * (size_t)S * (m + 1))) != cudaSuccess) return e;
    if ((e = mem.alloc(&h, sizeof(double2) * (size_t)S * (m + 1))) != cudaSuccess) return e;
    if ((e = mem.alloc(&h2, sizeof(double2) * (size_t)S * (m + 1))) != cudaSuccess) return e;
    if ((e = mem.alloc(&nrm, sizeof(double2) * (size_t)S)) != cudaSuccess) return e;
    if ((e = mem.alloc(&y, sizeof(double2) * (size_t)S * m)) != cudaSuccess) return e;
    if ((e = mem.alloc(&partial, sizeof(double2) * (size_t)(m + 1) * g.nbt() * kMaxGroupE)) != cudaSuccess)
      return e;
    if ((e = mem.alloc(&resid, sizeof(double) * S)) != cudaSuccess) return e;
    if ((e = mem.alloc(&hc, sizeof(C2) * (size_t)S * (m + 1))) != cudaSuccess) return e;
    if ((e = mem.alloc(&inv, sizeof(T) * (size_t)S)) != cudaSuccess) return e;
    return mem.alloc(&bnorm, sizeof(double) * S);
  }
  C2 *vec(int j) { return reinterpret_cast<C2 *>(V) + (size_t)j * L; }
  C2 *wv() { return reinterpret_cast<C2 *>(w); }
  // out[j * S + s] = <V_j, x>; with hcoef also hc = -out in T
  template <typename U>
  void dots(int nv, const typename Cx<U>::t *base, size_t ld, const typename Cx<U>::t *x, double2 *out,
            int accumulate, cudaStream_t s, bool hcoef = false, bool scale = false) {
    gdot_kernel<U><<<gr->nbt(), gr->dot_block(), 0, s>>>(gr->d_meta, nv, base, ld, x, partial);
    greduce_kernel<T><<<(nv * S * 32 + 255) / 256, 256, 0, s>>>(gr->d_meta, nv, gr->nbt(), partial, out, accumulate,
                                                           hcoef ? hc : nullptr, -1.0, scale ? inv : nullptr);
    count_launches(2);
  }
  // nrm[s] = |x_s|^2 (and inv = 1 / |x_s| in T with scale)
  template <typename U>
  void norms(const typename Cx<U>::t *x, cudaStream_t s, bool scale = false) {
    gnorm_kernel<U><<<gr->nbt(), gr->dot_block(), 0, s>>>(gr->d_meta, x, partial);
    greduce_kernel<T><<<(S * 32 + 255) / 256, 256, 0, s>>>(gr->d_meta, 1, gr->nbt(), partial, nrm, 0, nullptr, -1.0,
                                                          scale ? inv : nullptr);
    count_launches(2);
  }
  // w += sum_{j < nv} hc_j V_j (FP32 in an even group: two energies per thread)
  void axpy(int nv, cudaStream_t s) {
    if (sizeof(T) == 4 && gr->even) {
      const float4 *Vv = reinterpret_cast<const float4 *>(V), *cc = reinterpret_cast<const float4 *>(hc);
      float4 *ww = reinterpret_cast<float4 *>(w);
      const int g = grid_for(L / 2, 256);
      if (nv <= 2)
        gaxpy2_kernel<2><<<g, 256, 0, s>>>(gr->d_meta, L / 2, nv, Vv, (size_t)L / 2, cc, ww);
      else if (nv <= 4)
        gaxpy2_kernel<4><<<g, 256, 0, s>>>(gr->d_meta, L / 2, nv, Vv, (size_t)L / 2, cc, ww);
      else if (nv <= 8)
        gaxpy2_kernel<8><<<g, 256, 0, s>>>(gr->d_meta, L / 2, nv, Vv, (size_t)L / 2, cc, ww);
      else if (nv <= 12)
        gaxpy2_kernel<12><<<g, 256, 0, s>>>(gr->d_meta, L / 2, nv, Vv, (size_t)L / 2, cc, ww);
      else
        gaxpy2_kernel<0><<<g, 256, 0, s>>>(gr->d_meta, L / 2, nv, Vv, (size_t)L / 2, cc, ww);
    } else {
      gaxpy_kernel<T><<<grid_for(L, 256), 256, 0, s>>>(gr->d_meta, L, nv, vec(0), (size_t)L, hc, wv());
    }
  }
  // one Arnoldi step from column k (w = (I - K) v_k on entry); classical
  // Gram-Schmidt with a second pass (reorth) or a single pass
  void step(int k, cudaStream_t s, bool reorth) {
    const int vg = grid_for(L, 256);
    const size_t ld = (size_t)L;
    dots<T>(k + 1, vec(0), ld, wv(), h, 0, s, true);
    axpy(k + 1, s);
    if (reorth) {
      dots<T>(k + 1, vec(0), ld, wv(), h2, 0, s, true);
      axpy(k + 1, s);
      // h += h2: the second pass's coefficients, summed from its partials
      greduce_kernel<T><<<((k + 1) * S * 32 + 255) / 256, 256, 0, s>>>(gr->d_meta, k + 1, gr->nbt(), partial, h, 1,
                                                                   nullptr, 0.0, nullptr);
      count_launches(2);
    }
    norms<T>(wv(), s, true);
    gscale_kernel<T><<<vg, 256, 0, s>>>(gr->d_meta, L, wv(), inv, vec(k + 1));
    bgivens_kernel<<<(S + 127) / 128, 128, 0, s>>>(S, m, k, h, nrm, H, cs, sn, bet, resid, bnorm);
    count_launches(3);
  }
};

struct GCtx {
  double *g = nullptr, *b = nullptr, *u = nullptr, *r = nullptr, *t = nullptr, *wy = nullptr, *wz = nullptr;
  float *g32 = nullptr, *wy32 = nullptr, *wz32 = nullptr;
  GDf df;               // float-float residual work (WPCD_SOLVE_MIXED)
  int *j0 = nullptr;
  int64_t *idx0 = nullptr;
  double *D = nullptr, *pref = nullptr, *amp = nullptr;
  DevFree mem;
};

// plain FP64 Krylov on every system from u = 0; conv[s] = steps to tolerance
wpcd_status gsolve_fp64(const Group &gr, const wpcd_solve_opts &o, GCtx &cx, GKrylov<double> &kr,
                        std::vector<int> &status, std::vector<double> &relres, std::vector<int> &conv, int &n_apply,
                        cudaStream_t s) {
  const int S = gr.S, m = kr.m;
  const int64_t L = gr.L;
  const int vg = grid_for(L, 256);
  n_apply = 0;
  WPCD_CUDA_TRY(cudaMemsetAsync(cx.u, 0, 16 * L, s));
  kr.norms<double>((const double2 *)cx.b, s);
  std::vector<double2> nb(S);
  WPCD_CUDA_TRY(cudaMemcpyAsync(nb.data(), kr.nrm, sizeof(double2) * S, cudaMemcpyDeviceToHost, s));
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<double> bn(S);
  std::vector<double2> bet0((size_t)S * (m + 1), make_double2(0.0, 0.0));
  for (int e = 0; e < S; ++e) {
    bn[e] = std::sqrt(nb[e].x);
    if (!(bn[e] > 0.0)) return set_error(WPCD_EBREAKDOWN, "Born term is zero");
    bet0[(size_t)e * (m + 1)] = make_double2(bn[e], 0.0);
  }
  kr.norms<double>((const double2 *)cx.b, s, true);  // inv = 1 / |b| for v0
  gscale_kernel<double><<<vg, 256, 0, s>>>(gr.d_meta, L, (const double2 *)cx.b, kr.inv, kr.vec(0));
  count_launches(1);
  WPCD_CUDA_TRY(cudaMemsetAsync(kr.H, 0, sizeof(double2) * (size_t)S * (m + 1) * m, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(kr.bet, bet0.data(), sizeof(double2) * bet0.size(), cudaMemcpyHostToDevice, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(kr.bnorm, bn.data(), sizeof(double) * S, cudaMemcpyHostToDevice, s));
  status.assign(S, WPCD_ENOCONV);
  relres.assign(S, 1.0);
  conv.assign(S, m + 1);
  std::vector<double> res(S);
  bool done = false;
  int k = 0;
  for (k = 0; k < m && !done; ++k) {
    wpcd_status st = gkapply<double>(gr, cx.g, (double *)kr.vec(k), kr.w, (double *)kr.vec(k), cx.wy, cx.wz, s);
    if (st != WPCD_OK) return st;
    ++n_apply;
    kr.step(k, s, true);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_error(ce, "grouped krylov step launch");
    if (((k + 1) % std::max(o.check_every, 1) == 0) || k + 1 == m) {
      WPCD_CUDA_TRY(cudaMemcpyAsync(res.data(), kr.resid, sizeof(double) * S, cudaMemcpyDeviceToHost, s));
      WPCD_CUDA_TRY(cudaStreamSynchronize(s));
      done = true;
      for (int e = 0; e < S; ++e) {
        if (status[e] == WPCD_OK) continue;
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
  bbacksub_kernel<<<(S + 127) / 128, 128, 0, s>>>(S, m, k, kr.H, kr.bet, kr.y);
  bupdate_coef_kernel<double><<<std::max(1, (k * S + 255) / 256), 256, 0, s>>>(k, S, kr.y, nullptr, kr.hc);
  gupdate_kernel<double><<<vg, 256, 0, s>>>(gr.d_meta, L, k, kr.vec(0), (size_t)L, kr.hc, (double2 *)cx.u);
  count_launches(3);
  return WPCD_OK;
}

// mixed precision: FP64 refinement around FP32 inner cycles (graph-replayed)
wpcd_status gsolve_mixed(const Group &gr, const wpcd_solve_opts &o, GCtx &cx, GKrylov<float> &kr,
                         GKrylov<double> &k64, std::vector<int> &status, std::vector<double> &relres, int &n64,
                         int &n32, int &n_outer, cudaStream_t s) {
  const int S = gr.S, m = kr.m;
  const int64_t L = gr.L;
  const int vg = grid_for(L, 256);
  n64 = n32 = n_outer = 0;
  WPCD_CUDA_TRY(cudaMemsetAsync(cx.u, 0, 16 * L, s));
  k64.norms<double>((const double2 *)cx.b, s);
  std::vector<double2> nb(S);
  WPCD_CUDA_TRY(cudaMemcpyAsync(nb.data(), k64.nrm, sizeof(double2) * S, cudaMemcpyDeviceToHost, s));
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<double> bn(S);
  for (int e = 0; e < S; ++e) {
    bn[e] = std::sqrt(nb[e].x);
    if (!(bn[e] > 0.0)) return set_error(WPCD_EBREAKDOWN, "Born term is zero");
  }
  std::vector<double> ones(S, 1.0);
  std::vector<double2> bet0((size_t)S * (m + 1), make_double2(0.0, 0.0));
  for (int e = 0; e < S; ++e) bet0[(size_t)e * (m + 1)] = make_double2(1.0, 0.0);
  DevFree tmp;
  tmp.st = s;
  double2 *d_bet0 = nullptr;
  WPCD_CUDA_TRY(tmp.alloc(&d_bet0, sizeof(double2) * bet0.size()));
  WPCD_CUDA_TRY(cudaMemcpyAsync(kr.bnorm, ones.data(), sizeof(double) * S, cudaMemcpyHostToDevice, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(d_bet0, bet0.data(), sizeof(double2) * bet0.size(), cudaMemcpyHostToDevice, s));
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  // the inner cycle of mm <= m steps (the full one captured as a graph)
  auto inner_cycle = [&](int mm) -> wpcd_status {
    cudaMemsetAsync(kr.H, 0, sizeof(double2) * (size_t)S * (m + 1) * m, s);
    cudaMemcpyAsync(kr.bet, d_bet0, sizeof(double2) * bet0.size(), cudaMemcpyDeviceToDevice, s);
    for (int k = 0; k < mm; ++k) {
      wpcd_status st =
          gkapply<float>(gr, cx.g32, (float *)kr.vec(k), kr.w, (float *)kr.vec(k), cx.wy32, cx.wz32, s);
      if (st != WPCD_OK) return st;
      // single-pass Gram-Schmidt: the FP64 refinement residual judges the cycle
      kr.step(k, s, false);
    }
    bbacksub_kernel<<<(S + 127) / 128, 128, 0, s>>>(S, m, mm, kr.H, kr.bet, kr.y);
    bupdate_coef_kernel<float><<<(mm * S + 255) / 256, 256, 0, s>>>(mm, S, kr.y, k64.nrm, kr.hc);
    gupdate_kernel<float><<<vg, 256, 0, s>>>(gr.d_meta, L, mm, kr.vec(0), (size_t)L, kr.hc, (double2 *)cx.u);
    count_launches(3);
    return WPCD_OK;
  };
  cudaGraphExec_t exec = nullptr;
  int graph_kernels = 0;
  status.assign(S, WPCD_ENOCONV);
  relres.assign(S, 1.0);
  std::vector<double2> nr(S);
  const int max_outer = o.max_outer > 0 ? o.max_outer : 12;
  wpcd_status result = WPCD_OK;
  // cycle lengths after the first from the previous cycle's per-step
  // reduction of the worst residual, as in the single-problem solve
  double worst_prev = 0.0;
  int mm_prev = 0;
  for (int outer = 0; outer <= max_outer; ++outer) {
    if (outer > 0) {  // r = b - (I - K) u in FP64
      wpcd_status st = cx.df.xh ? gkapply_df(gr, cx.g, cx.u, cx.t, cx.df, s)
                                : gkapply<double>(gr, cx.g, cx.u, cx.t, nullptr, cx.wy, cx.wz, s);
      if (st != WPCD_OK) {
        result = st;
        break;
      }
      ++n64;
      bresid_kernel<<<vg, 256, 0, s>>>(L, (double2 *)cx.b, (double2 *)cx.u, (double2 *)cx.t, (double2 *)cx.r);
      count_launches(1);
    } else {
      cudaMemcpyAsync(cx.r, cx.b, 16 * L, cudaMemcpyDeviceToDevice, s);
    }
    k64.norms<double>((const double2 *)cx.r, s, true);  // |r|^2 and 1 / |r|
    cudaMemcpyAsync(nr.data(), k64.nrm, sizeof(double2) * S, cudaMemcpyDeviceToHost, s);
    cudaError_t ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
      result = cuda_error(ce, "grouped refinement residual");
      break;
    }
    bool done = true;
    double worst = 0.0;
    for (int e = 0; e < S; ++e) {
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
    gnormalize_f32_kernel<<<vg, 256, 0, s>>>(gr.d_meta, L, (const double2 *)cx.r, k64.inv, kr.vec(0));
    count_launches(1);
    if (o.use_graph && s != nullptr && mm == m) {  // the legacy default stream cannot be captured
      if (!exec) {
        cudaGraph_t graph;
        const int64_t launches0 = wpcd_launch_count();
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
  return result;
}

}  // namespace

wpcd_status solve_group(int n_prob, wpcd_problem *const *prs, const wpcd_P *const *Ps, const double *const *E,
                        const int *n_E, const wpcd_solve_opts *o, double *const *U00, wpcd_solve_stats *const *st_out,
                        cudaStream_t s) {
  wpcd_solve_opts opt{};
  opt.method = WPCD_SUM_KRYLOV;
  opt.max_iter = 100;
  opt.min_iter = 4;
  opt.tol = 1e-10;
  opt.check_every = 4;
  opt.precision = WPCD_SOLVE_FP64;
  opt.use_graph = 1;
  if (o) opt = *o;
  if (n_prob < 1 || n_prob > kMaxGroup) return set_error(WPCD_EINVAL, "n_prob must be in [1, WPCD_GROUP_MAX]");
  if (!prs || !Ps || !E || !n_E || !U00) return set_error(WPCD_EINVAL, "NULL group arrays");
  if (opt.method != WPCD_SUM_KRYLOV) return set_error(WPCD_EINVAL, "the grouped solve uses the Krylov summation");
  if (opt.precision != WPCD_SOLVE_FP64 && opt.precision != WPCD_SOLVE_MIXED &&
      opt.precision != WPCD_SOLVE_MIXED_FP64)
    return set_error(WPCD_EINVAL, "unknown precision");
  if (opt.u_init || opt.u_out) return set_error(WPCD_EINVAL, "the grouped solve takes no vectors");
  if (opt.batch != 0) return set_error(WPCD_EINVAL, "the grouped solve takes every energy in one batch (batch 0)");
  if (opt.max_iter < 2 || opt.max_iter > 512) return set_error(WPCD_EINVAL, "max_iter must be in [2, 512]");
  if (!(opt.tol > 0.0)) return set_error(WPCD_EINVAL, "tol must be positive");
  if (opt.inner_iter < 0 || opt.inner_iter > 128) return set_error(WPCD_EINVAL, "inner_iter must be in [0, 128]");
  Group gr;
  gr.n = n_prob;
  for (int g = 0; g < n_prob; ++g) {
    const wpcd_problem *pr = prs[g];
    const wpcd_P *P = Ps[g];
    if (!pr || !P || !E[g] || !U00[g]) return set_error(WPCD_EINVAL, "NULL problem, P, energies or output");
    if (!P_fits(P, pr)) return set_error(WPCD_EINVAL, "P was assembled on another lattice or for another channel count");
    if (n_E[g] < 1 || n_E[g] > kMaxGroupE) return set_error(WPCD_EINVAL, "n_E must be in [1, WPCD_GROUP_MAX_E]");
    if (g > 0 && (pr->device != prs[0]->device || pr->n_ch != prs[0]->n_ch || P->prec != Ps[0]->prec))
      return set_error(WPCD_EINVAL, "grouped problems must share device, channel count and P precision");
    const int64_t seg = (int64_t)pr->n_ch * pr->N * pr->M * n_E[g];
    if (seg > (int64_t)1 << 30) return set_error(WPCD_EINVAL, "problem segment too large for the grouped solve");
    for (int e = 0; e < n_E[g]; ++e) {
      int j0;
      double lo, hi;
      wpcd_status st = onshell(pr, E[g][e], &j0, &lo, &hi, nullptr);
      if (st != WPCD_OK) return st;
    }
  }
  WPCD_CUDA_TRY(cudaSetDevice(prs[0]->device));
  const bool mixed = opt.precision != WPCD_SOLVE_FP64;
  // WPCD_SOLVE_MIXED: float-float residual and Born term; WPCD_SOLVE_MIXED_FP64: native FP64
  const bool ff = opt.precision == WPCD_SOLVE_MIXED;
  gr.n_ch = prs[0]->n_ch;
  gr.prec = Ps[0]->prec;
  if (ff)
    for (int g = 0; g < n_prob; ++g) {
      // the grouped residual runs its own float-float products: no digit planes
      wpcd_status st = df_prepare(const_cast<wpcd_problem *>(prs[g]), const_cast<wpcd_P *>(Ps[g]), s, false);
      if (st != WPCD_OK) return st;
    }
  // FP32 values of FP64-assembled matrices for the inner cycles
  for (int g = 0; g < n_prob; ++g) {
    wpcd_P *P = const_cast<wpcd_P *>(Ps[g]);
    if (mixed && !P->val32 && !P->val32_copy) {
      WPCD_CUDA_TRY(dev_malloc(&P->val32_copy, sizeof(float) * (size_t)P->nnz * P->n_pairs + 4));
      const int64_t nv = (int64_t)P->nnz * P->n_pairs;
      gd2f_kernel<<<grid_for(nv, 256), 256, 0, s>>>(nv, P->val64, P->val32_copy);
      count_launches(1);
    }
  }
  // offsets and descriptors
  GMeta &mt = gr.meta;
  mt.n = n_prob;
  mt.eoff[0] = 0;
  mt.sys[0] = mt.tile_off[0] = mt.dtile_off[0] = mt.cell_off[0] = 0;
  for (int g = 0; g < n_prob; ++g) {
    const wpcd_problem *pr = prs[g];
    const wpcd_P *P = Ps[g];
    const int B = n_E[g];
    GProb q{};
    q.N = pr->N;
    q.M = pr->M;
    q.B = B;
    q.n_cells = pr->N * pr->M;
    q.rt = (pr->N + GB_M - 1) / GB_M;
    q.ct = (int)((2LL * pr->M * B + GB_N - 1) / GB_N);
    q.dct = (int)((2LL * pr->M * B + DF_N - 1) / DF_N);
    q.eoff = mt.eoff[g];
    q.nnz = P->nnz;
    q.row_ptr = P->row_ptr;
    q.col = P->col;
    q.val64 = P->val64;
    q.val32 = P->val32 ? P->val32 : P->val32_copy;
    q.O = pr->d.O;
    q.Vt = pr->d.Vt;
    q.O32 = pr->d.O32;
    q.Vt32 = pr->d.Vt32;
    q.O_h = pr->d.O_h;
    q.O_l = pr->d.O_l;
    q.Vt_h = pr->d.Vt_h;
    q.Vt_l = pr->d.Vt_l;
    q.val_h = P->prec == WPCD_FP64 ? P->val_h : P->val32;
    q.val_l = P->prec == WPCD_FP64 ? P->val_l : nullptr;
    gr.probs.push_back(q);
    mt.B[g] = B;
    mt.eoff[g + 1] = mt.eoff[g] + (int64_t)pr->n_ch * pr->N * pr->M * B;
    mt.sys[g + 1] = mt.sys[g] + B;
    mt.tile_off[g + 1] = mt.tile_off[g] + pr->n_ch * q.rt * q.ct;
    mt.dtile_off[g + 1] = mt.dtile_off[g] + pr->n_ch * q.rt * q.dct;
    mt.cell_off[g + 1] = mt.cell_off[g] + q.n_cells;
    gr.Bmax = std::max(gr.Bmax, B);
    gr.even = gr.even && B % 2 == 0 && mt.eoff[g] % 2 == 0;
  }
  // FP32 block products of the inner cycles on the tensor cores when every
  // problem fits (N <= 512) and every segment is 16-byte aligned
  if (mixed && tc_enabled() && gr.even) {
    bool ok = true;
    for (int g = 0; g < n_prob; ++g) ok = ok && tc_supported(prs[g]);
    if (ok) {
      for (int g = 0; g < n_prob; ++g) {
        wpcd_status st = tc_prepare(const_cast<wpcd_problem *>(prs[g]), s);
        if (st != WPCD_OK) return st;
        gr.tcp.push_back(TcGroupProb{prs[g], 2 * mt.eoff[g], 2LL * prs[g]->M * n_E[g]});
      }
      if (wpcd_status st = tc_clear(prs[0], s); st != WPCD_OK) return st;
      gr.tc = true;
    }
  }
  gr.S = mt.S = mt.sys[n_prob];
  gr.L = mt.eoff[n_prob];
  // dot-product blocks: about two per SM, split in proportion to segment size
  const int target = 152 * 2;
  mt.blk_off[0] = 0;
  for (int g = 0; g < n_prob; ++g) {
    const double share = (double)(mt.eoff[g + 1] - mt.eoff[g]) / (double)gr.L;
    mt.blk_off[g + 1] = mt.blk_off[g] + std::max(1, (int)std::lround(share * target));
  }
  GCtx cx;
  cx.mem.st = s;
  WPCD_CUDA_TRY(cx.mem.alloc(&gr.d_meta, sizeof(GMeta)));
  WPCD_CUDA_TRY(cx.mem.alloc(&gr.d_probs, sizeof(GProb) * n_prob));
  WPCD_CUDA_TRY(cudaMemcpyAsync(gr.d_meta, &mt, sizeof(GMeta), cudaMemcpyHostToDevice, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(gr.d_probs, gr.probs.data(), sizeof(GProb) * n_prob, cudaMemcpyHostToDevice, s));
  const size_t nb = 16 * (size_t)gr.L;
  WPCD_CUDA_TRY(cx.mem.alloc(&cx.g, nb));
  WPCD_CUDA_TRY(cx.mem.alloc(&cx.b, nb));
  WPCD_CUDA_TRY(cx.mem.alloc(&cx.u, nb));
  WPCD_CUDA_TRY(cx.mem.alloc(&cx.r, nb));
  WPCD_CUDA_TRY(cx.mem.alloc(&cx.t, nb));
  WPCD_CUDA_TRY(cx.mem.alloc(&cx.wy, nb));
  WPCD_CUDA_TRY(cx.mem.alloc(&cx.wz, nb));
  if (mixed) {
    WPCD_CUDA_TRY(cx.mem.alloc(&cx.g32, nb / 2));
    WPCD_CUDA_TRY(cx.mem.alloc(&cx.wy32, nb / 2));
    WPCD_CUDA_TRY(cx.mem.alloc(&cx.wz32, nb / 2));
  }
  if (ff) {
    WPCD_CUDA_TRY(cx.mem.alloc(&cx.df.xh, nb / 2));
    WPCD_CUDA_TRY(cx.mem.alloc(&cx.df.xl, nb / 2));
    WPCD_CUDA_TRY(cx.mem.alloc(&cx.df.yh, nb / 2));
    WPCD_CUDA_TRY(cx.mem.alloc(&cx.df.yl, nb / 2));
  }
  const int S = gr.S;
  WPCD_CUDA_TRY(cx.mem.alloc(&cx.j0, sizeof(int) * S));
  WPCD_CUDA_TRY(cx.mem.alloc(&cx.idx0, sizeof(int64_t) * S));
  WPCD_CUDA_TRY(cx.mem.alloc(&cx.D, sizeof(double) * S));
  WPCD_CUDA_TRY(cx.mem.alloc(&cx.pref, sizeof(double) * S));
  WPCD_CUDA_TRY(cx.mem.alloc(&cx.amp, sizeof(double) * 6 * S));
  // per-system on-shell data (host) and the launch shapes, before the clock
  std::vector<int> j0(S);
  std::vector<int64_t> idx0(S);
  std::vector<double> Dh(S), prefh(S);
  for (int g = 0; g < n_prob; ++g)
    for (int e = 0; e < n_E[g]; ++e) {
      const int si = mt.sys[g] + e;
      double lo, hi, q0;
      onshell(prs[g], E[g][e], &j0[si], &lo, &hi, &q0);
      Dh[si] = hi - lo;
      prefh[si] = 2.0 / (3.0 * q0) / (prs[g]->qe[j0[si] + 1] - prs[g]->qe[j0[si]]);
      idx0[si] = mt.eoff[g] + (int64_t)j0[si] * n_E[g] + e;  // channel 0, k = 0, q-bin j0
    }
  WPCD_CUDA_TRY(cudaMemcpyAsync(cx.j0, j0.data(), sizeof(int) * S, cudaMemcpyHostToDevice, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(cx.idx0, idx0.data(), sizeof(int64_t) * S, cudaMemcpyHostToDevice, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(cx.D, Dh.data(), sizeof(double) * S, cudaMemcpyHostToDevice, s));
  WPCD_CUDA_TRY(cudaMemcpyAsync(cx.pref, prefh.data(), sizeof(double) * S, cudaMemcpyHostToDevice, s));
  WPCD_CUDA_TRY(cudaMemsetAsync(cx.wy, 0, nb, s));
  wpcd_status st = gtune(
      gr, 0, [&](const SpmmConfig &c) { return gspmm<double>(gr, cx.wy, cx.wz, c, s); }, s, &gr.cfg64);
  if (st == WPCD_OK && mixed) {
    WPCD_CUDA_TRY(cudaMemsetAsync(cx.wy32, 0, nb / 2, s));
    st = gtune(
        gr, 1, [&](const SpmmConfig &c) { return gspmm<float>(gr, cx.wy32, cx.wz32, c, s); }, s, &gr.cfg32);
  }
  if (st == WPCD_OK && ff) {
    WPCD_CUDA_TRY(cudaMemsetAsync(cx.df.yh, 0, nb / 2, s));
    WPCD_CUDA_TRY(cudaMemsetAsync(cx.df.yl, 0, nb / 2, s));
    st = gtune(
        gr, 2, [&](const SpmmConfig &c) { return gspmm_df_cfg(gr, cx.df.yh, cx.df.yl, cx.df.xh, cx.df.xl, c, s); },
        s, &gr.cfgff);
  }
  if (st != WPCD_OK) return st;
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));  // host staging vectors

  struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  WPCD_CUDA_TRY(cudaEventCreate(&ev.a));
  WPCD_CUDA_TRY(cudaEventCreate(&ev.b));
  cudaEventRecord(ev.a, s);
  // G1 of every system (one launch per problem: the per-bin energy averages
  // are the problem's own), then the Born terms u0 = O P0 Vt e0
  for (int g = 0; g < n_prob && st == WPCD_OK; ++g)
    st = resolvent_minor(prs[g], E[g], n_E[g], cx.g + 2 * mt.eoff[g], s);
  if (st != WPCD_OK) return st;
  if (mixed) {
    gd2f_kernel<<<grid_for(2 * gr.L, 256), 256, 0, s>>>(2 * gr.L, cx.g, cx.g32);
    count_launches(1);
  }
  if (ff) {
    gborn_vt_df_kernel<<<grid_for(gr.L, 256), 256, 0, s>>>(gr.d_meta, gr.d_probs, gr.L, cx.j0, (float2 *)cx.df.yh,
                                                           (float2 *)cx.df.yl);
    count_launches(1);
    st = gspmm_df_cfg(gr, cx.df.yh, cx.df.yl, cx.df.xh, cx.df.xl, gr.cfgff, s);
    if (st != WPCD_OK) return st;
    ggemm_df<false>(gr, true, cx.df.xh, cx.df.xl, cx.b, nullptr, nullptr, s);
  } else {
    gborn_vt_kernel<<<grid_for(gr.L, 256), 256, 0, s>>>(gr.d_meta, gr.d_probs, gr.L, cx.j0, (double2 *)cx.wy);
    count_launches(1);
    st = gspmm<double>(gr, cx.wy, cx.wz, gr.cfg64, s);
    if (st != WPCD_OK) return st;
    ggemm<double>(gr, true, false, false, cx.wz, nullptr, nullptr, cx.b, s);
  }
  std::vector<int> status, conv;
  std::vector<double> relres;
  int n64 = 0, n32 = 0, n_outer = 0;
  if (mixed) {
    GKrylov<float> kr;
    GKrylov<double> k64;
    WPCD_CUDA_TRY(kr.alloc(gr, opt.inner_iter > 0 ? opt.inner_iter : kDefaultInner, s));
    WPCD_CUDA_TRY(k64.alloc(gr, 1, s, false));  // norms only
    st = gsolve_mixed(gr, opt, cx, kr, k64, status, relres, n64, n32, n_outer, s);
  } else {
    GKrylov<double> kr;
    WPCD_CUDA_TRY(kr.alloc(gr, opt.max_iter, s));
    st = gsolve_fp64(gr, opt, cx, kr, status, relres, conv, n64, s);
  }
  if (st != WPCD_OK) return st;
  if (gr.tc && (st = tc_check(prs[0], s)) != WPCD_OK) return st;
  n64 += 1;  // the Born term
  gamplitude_kernel<<<(S + 127) / 128, 128, 0, s>>>(S, (const double2 *)cx.u, cx.idx0, cx.D, cx.pref, cx.amp);
  count_launches(1);
  cudaEventRecord(ev.b, s);
  std::vector<double> amp(6 * (size_t)S);
  WPCD_CUDA_TRY(cudaMemcpyAsync(amp.data(), cx.amp, sizeof(double) * 6 * S, cudaMemcpyDeviceToHost, s));
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev.a, ev.b);
  wpcd_status worst = WPCD_OK;
  for (int g = 0; g < n_prob; ++g)
    for (int e = 0; e < n_E[g]; ++e) {
      const int si = mt.sys[g] + e;
      U00[g][2 * e] = amp[6 * si];
      U00[g][2 * e + 1] = amp[6 * si + 1];
      if (st_out && st_out[g]) {
        wpcd_solve_stats &so = st_out[g][e];
        so = wpcd_solve_stats{};
        so.status = status[si];
        so.n_kapply = conv.empty() ? n64 : std::min(conv[si], n64) + 1;
        so.n_kapply32 = n32;
        so.n_outer = n_outer;
        so.j0 = j0[si];
        so.D = Dh[si];
        so.relres = relres[si];
        for (int i = 0; i < 2; ++i) {
          so.U00[i] = amp[6 * si + i];
          so.S[i] = amp[6 * si + 2 + i];
          so.A[i] = amp[6 * si + 4 + i];
        }
        so.ms = ms / S;
      }
      if (status[si] < worst) worst = status[si];
    }
  if (worst != WPCD_OK)
    set_error(worst, worst == WPCD_ENOCONV ? "summation did not reach the tolerance for some energy"
                                           : "Krylov breakdown for some energy");
  return worst;
}

}  // namespace wpcd
