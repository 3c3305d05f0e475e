// Row-tiled FP32 SpMM of the inner cycles, Z = P0 Y over a batch of
// energies (Sec. 3.3 Eq. kernel, the sparse step; P0 of Sec. 3.2 Eq. perm).
//
// The permutation conserves p^2 + 3/4 q^2, so the nonzeros of a row of P0
// lie on one energy shell, and rows of neighbouring cells share many of
// their columns: for the 3-channel 200 x 200 lattice a column of a 2 x 1
// tile of cells (two neighbouring p-bins, one q-bin) is used by 1.44 of its
// 2 rows on average, of a 2 x 2 tile by 2.19 of 4 (consecutive cells of one
// p-bin share less: 2.46 of 16).  The warp-per-row SpMM gathers the y row of
// a column once per nonzero; here a warp takes a tile of R cells and gathers
// the y row of each column of the tile once, into registers, and applies it
// to all R rows.  The tile structure is built once per matrix on the device
// (a counting pass, a host prefix sum, a filling pass: tile2_merge_warp_kernel
// for 2-cell tiles, tile_merge_kernel for 4-cell ones): for tile t the
// merged, ascending column list of its rows, and per column an R-row block
// of values for every (l, l') pair, zero where a row lacks the column.
//
// A warp covers 32 lanes x EPT energies (two adjacent energies per 16-byte
// load, lanes interleaved as in the warp-per-row kernel); per column of a
// tile it loads the column index and the R x n_pairs values (broadcast), the
// NCH y rows of its energies, and does R n_pairs EPT complex multiply-adds.
// Sums as in the other FP32 SpMM (FABsum, Blanchard, Higham and Mary 2020):
// plain FMAs over blocks of 32 or 64 columns of the tile (the autotuner's
// choice), each block added with TwoSum to a compensated accumulator held in
// shared memory.  (Packed fma.rn.f32x2 multiply-adds, with the values stored
// as {v, v} pairs, measured slower: 0.67 against 0.60 ms at 128 energies.)
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "common.cuh"
#include "wpcd_internal.h"

namespace wpcd {
namespace {

constexpr int TL_THREADS = 128;  // 4 warps: 4 CTAs per SM (2% faster than 8-warp CTAs)

// floats of one column's value block: R rows x n_pairs, padded to 4
__host__ __device__ constexpr int tile_vs(int R, int npair) { return (R * npair + 3) & ~3; }

// rows of tile t (-1 where the lattice ends): R = 2 tiles span p-bins
// (2 i', 2 i' + 1) at one q-bin, R = 4 tiles p-bins (2 i', 2 i' + 1) and
// q-bins (2 j', 2 j' + 1); tiles are numbered q fastest
template <int R>
__host__ __device__ inline void tile_rows(int t, int N, int M, int (&r)[R]) {
  if constexpr (R == 2) {
    const int ip = t / M, j = t % M;
    r[0] = 2 * ip * M + j;
    r[1] = 2 * ip + 1 < N ? (2 * ip + 1) * M + j : -1;
  } else {
    const int Mh = (M + 1) / 2, ip = t / Mh, jp = t % Mh;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = 2 * ip + (k >> 1), j = 2 * jp + (k & 1);
      r[k] = i < N && j < M ? i * M + j : -1;
    }
  }
}

template <int R>
__host__ __device__ inline int tile_count(int N, int M) {
  return R == 2 ? ((N + 1) / 2) * M : ((N + 1) / 2) * ((M + 1) / 2);
}

// merge of the tile's R ascending column lists: count (fill = false) or
// write the merged columns and value blocks (fill = true)
template <int R, bool FILL>
__global__ void __launch_bounds__(TL_THREADS) tile_merge_kernel(int N, int M, int npair, const int64_t *__restrict__ row_ptr,
                                                               const int32_t *__restrict__ col,
                                                               const float *__restrict__ val, int64_t nnz,
                                                               int64_t *__restrict__ cnt_or_ptr,
                                                               int32_t *__restrict__ ucol, float *__restrict__ tval) {
  const int n_tiles = tile_count<R>(N, M);
  const int vs = tile_vs(R, npair);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x) {
    int r[R];
    tile_rows<R>(t, N, M, r);
    int64_t p[R], e[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      p[k] = r[k] >= 0 ? row_ptr[r[k]] : 0;
      e[k] = r[k] >= 0 ? row_ptr[r[k] + 1] : 0;
    }
    int64_t u = FILL ? cnt_or_ptr[t] : 0;
    while (true) {
      int cmin = INT32_MAX;
#pragma unroll
      for (int k = 0; k < R; ++k)
        if (p[k] < e[k]) cmin = min(cmin, col[p[k]]);
      if (cmin == INT32_MAX) break;
      if (FILL) {
        ucol[u] = cmin;
        float *v = tval + u * vs;
        for (int q = R * npair; q < vs; ++q) v[q] = 0.f;
      }
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const bool has = p[k] < e[k] && col[p[k]] == cmin;
        if (FILL)
          for (int m = 0; m < npair; ++m) tval[u * vs + m * R + k] = has ? val[(size_t)m * nnz + p[k]] : 0.f;
        if (has) ++p[k];
      }
      ++u;
    }
    if (!FILL) cnt_or_ptr[t] = u;
  }
}

// the same merge for 2-cell tiles, a warp per tile: the merged position of
// a column of one row is its index there plus the number of the other row's
// columns below it (a binary search) less the number of shared columns
// before it (a warp prefix count); shared columns are written from the first
// row.  The result is the thread-per-tile kernel's, element for element.
__device__ __forceinline__ int t2_lower_bound(const int32_t *__restrict__ a, int n, int x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <bool FILL>
__global__ void __launch_bounds__(TL_THREADS) tile2_merge_warp_kernel(int N, int M, int npair,
                                                                     const int64_t *__restrict__ row_ptr,
                                                                     const int32_t *__restrict__ col,
                                                                     const float *__restrict__ val, int64_t nnz,
                                                                     int64_t *__restrict__ cnt_or_ptr,
                                                                     int32_t *__restrict__ ucol,
                                                                     float *__restrict__ tval) {
  const int n_tiles = tile_count<2>(N, M);
  const int vs = tile_vs(2, npair);
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_tiles; t += (gridDim.x * blockDim.x) >> 5) {
    int r[2];
    tile_rows<2>(t, N, M, r);
    const int64_t a0 = row_ptr[r[0]], na = row_ptr[r[0] + 1] - a0;
    const int64_t b0 = r[1] >= 0 ? row_ptr[r[1]] : 0, nb = r[1] >= 0 ? row_ptr[r[1] + 1] - b0 : 0;
    const int32_t *A = col + a0, *Bc = col + b0;
    const int64_t u0 = FILL ? cnt_or_ptr[t] : 0;
    // the first row's columns (and the shared ones)
    int common = 0;
    for (int i0 = 0; i0 < na; i0 += 32) {
      const int i = i0 + lane;
      const bool in = i < na;
      const int x = in ? __ldg(A + i) : 0;
      const int lb = in ? t2_lower_bound(Bc, (int)nb, x) : 0;
      const bool shared_col = in && lb < nb && __ldg(Bc + lb) == x;
      const unsigned m = __ballot_sync(0xffffffffu, shared_col);
      if (FILL && in) {
        const int64_t u = u0 + i + lb - (common + __popc(m & below));
        ucol[u] = x;
        float *v = tval + u * vs;
        for (int q = 0; q < npair; ++q) {
          v[q * 2] = val[(size_t)q * nnz + a0 + i];
          v[q * 2 + 1] = shared_col ? val[(size_t)q * nnz + b0 + lb] : 0.f;
        }
        for (int q = 2 * npair; q < vs; ++q) v[q] = 0.f;
      }
      common += __popc(m);
    }
    // the second row's columns that the first row lacks
    int common_b = 0;
    for (int j0 = 0; j0 < nb; j0 += 32) {
      const int j = j0 + lane;
      const bool in = j < nb;
      const int x = in ? __ldg(Bc + j) : 0;
      const int lb = in ? t2_lower_bound(A, (int)na, x) : 0;
      const bool shared_col = in && lb < na && __ldg(A + lb) == x;
      const unsigned m = __ballot_sync(0xffffffffu, shared_col);
      if (FILL && in && !shared_col) {
        const int64_t u = u0 + j + lb - (common_b + __popc(m & below));
        ucol[u] = x;
        float *v = tval + u * vs;
        for (int q = 0; q < npair; ++q) {
          v[q * 2] = 0.f;
          v[q * 2 + 1] = val[(size_t)q * nnz + b0 + j];
        }
        for (int q = 2 * npair; q < vs; ++q) v[q] = 0.f;
      }
      common_b += __popc(m);
    }
    if (!FILL && lane == 0) cnt_or_ptr[t] = na + nb - common;
  }
}

struct TileParams {
  int n_cells, n_tiles, N, M, B;
  const int64_t *tptr;
  const int32_t *ucol;
  const float *tval;
};

// compensated sums in shared memory: sum j of a thread keeps hi in row 2 j
// and lo in row 2 j + 1 of TL_THREADS floats (thread-major, so a warp's
// accesses hit distinct banks); base points at the thread's column
__device__ __forceinline__ void tl_add(float *base, int j, float x) {
  float *h = base + (size_t)(2 * j) * TL_THREADS;
  const float hi = h[0];
  const float sum = __fadd_rn(hi, x);
  const float bb = __fsub_rn(sum, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(x, bb));
  h[0] = sum;
  h[TL_THREADS] = __fadd_rn(h[TL_THREADS], err);
}

// Lane energies: pairs (2 lane, 2 lane + 1) + 64 h for h < EPT / 2.  FAB:
// columns of the tile per plain block.
template <int NCH, int R, int EPT, int FAB>
__global__ void __launch_bounds__(TL_THREADS, 4) spmm_tile_kernel(TileParams T, const float2 *__restrict__ y,
                                                                 float2 *__restrict__ z) {
  constexpr int NPAIR = pair_count(NCH);
  constexpr int VS = tile_vs(R, NPAIR);
  constexpr int H = EPT / 2;                      // 16-byte loads per channel
  constexpr int NSLOT = R * NCH * EPT * 2;        // real sums per lane
  extern __shared__ float tl_sm[];
  float *acc_sm = tl_sm + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n_warps = (gridDim.x * blockDim.x) >> 5;
  const int e_base = blockIdx.y * 32 * EPT;
  const int B = T.B;
  bool eok[H];
#pragma unroll
  for (int h = 0; h < H; ++h) eok[h] = e_base + 2 * lane + 64 * h < B;  // B even: the pair is whole
  for (int t = warp_global; t < T.n_tiles; t += n_warps) {
    int r[R];
    tile_rows<R>(t, T.N, T.M, r);
#pragma unroll
    for (int s = 0; s < 2 * NSLOT; ++s) acc_sm[(size_t)s * TL_THREADS] = 0.f;
    float part[R][NCH][EPT][2];
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
      for (int l = 0; l < NCH; ++l)
#pragma unroll
        for (int q = 0; q < EPT; ++q) part[k][l][q][0] = part[k][l][q][1] = 0.f;
    const int64_t u0 = T.tptr[t], u1 = T.tptr[t + 1];
    int nb = 0;
    // unrolled so that the next columns' value and y loads issue before this
    // column's FMAs (2-row tiles: 4 columns; 4-row tiles have no registers
    // to spare)
    constexpr int UNR = R == 2 ? 4 : 1;
#pragma unroll UNR
    for (int64_t u = u0; u < u1; ++u) {
      const int c = __ldg(T.ucol + u);
      float v[VS];
#pragma unroll
      for (int q = 0; q < VS; q += 4) {
        const float4 w = __ldg(reinterpret_cast<const float4 *>(T.tval + u * VS + q));
        v[q] = w.x, v[q + 1] = w.y, v[q + 2] = w.z, v[q + 3] = w.w;
      }
      float yr[NCH][EPT], yi[NCH][EPT];
#pragma unroll
      for (int l = 0; l < NCH; ++l)
#pragma unroll
        for (int h = 0; h < H; ++h) {
          float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
          if (eok[h])
            w = __ldg(reinterpret_cast<const float4 *>(y + ((size_t)l * T.n_cells + c) * B + e_base + 2 * lane +
                                                        64 * h));
          yr[l][2 * h] = w.x, yi[l][2 * h] = w.y, yr[l][2 * h + 1] = w.z, yi[l][2 * h + 1] = w.w;
        }
#pragma unroll
      for (int m = 0; m < NPAIR; ++m) {
        const int l = pair_first(NCH, m), lp = pair_second(NCH, m);
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
          for (int q = 0; q < EPT; ++q) {
            part[k][l][q][0] = fmaf(v[m * R + k], yr[lp][q], part[k][l][q][0]);
            part[k][l][q][1] = fmaf(v[m * R + k], yi[lp][q], part[k][l][q][1]);
          }
      }
      if (++nb == FAB || u + 1 == u1) {
        nb = 0;
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
          for (int l = 0; l < NCH; ++l)
#pragma unroll
            for (int q = 0; q < EPT; ++q)
#pragma unroll
              for (int x = 0; x < 2; ++x) {
                tl_add(acc_sm, ((k * NCH + l) * EPT + q) * 2 + x, part[k][l][q][x]);
                part[k][l][q][x] = 0.f;
              }
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (r[k] < 0) continue;
#pragma unroll
      for (int l = 0; l < NCH; ++l)
#pragma unroll
        for (int h = 0; h < H; ++h) {
          if (!eok[h]) continue;
          float o[4];
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int q = 2 * h + (w >> 1), x = w & 1;
            const int j = ((k * NCH + l) * EPT + q) * 2 + x;
            o[w] = __fadd_rn(acc_sm[(size_t)(2 * j) * TL_THREADS], acc_sm[(size_t)(2 * j + 1) * TL_THREADS]);
          }
          *reinterpret_cast<float4 *>(z + ((size_t)l * T.n_cells + r[k]) * B + e_base + 2 * lane + 64 * h) =
              make_float4(o[0], o[1], o[2], o[3]);
        }
    }
  }
}

template <int R>
wpcd_status tile_prepare_r(const wpcd_problem *pr, wpcd_P *P, const float *v32, cudaStream_t s) {
  const int idx = R == 2 ? 0 : 1;
  if (P->tile_ptr[idx]) return WPCD_OK;
  const int N = pr->N, M = pr->M, npair = pr->n_pairs;
  const int n_tiles = tile_count<R>(N, M);
  int64_t *ptr = nullptr;
  WPCD_CUDA_TRY(dev_malloc(&ptr, sizeof(int64_t) * (n_tiles + 1)));
  const int grid = grid_for(n_tiles, TL_THREADS);
  // 2-cell tiles: a warp per tile (640 K threads at 200 x 200, against 20 K)
  const int wgrid = grid_for((int64_t)n_tiles * 32, TL_THREADS, 152 * 16);
  if constexpr (R == 2)
    tile2_merge_warp_kernel<false><<<wgrid, TL_THREADS, 0, s>>>(N, M, npair, P->row_ptr, P->col, v32, P->nnz, ptr,
                                                                 nullptr, nullptr);
  else
    tile_merge_kernel<R, false><<<grid, TL_THREADS, 0, s>>>(N, M, npair, P->row_ptr, P->col, v32, P->nnz, ptr,
                                                             nullptr, nullptr);
  count_launches(1);
  // exclusive prefix sum of the tile sizes on the host (once per matrix)
  std::vector<int64_t> h(n_tiles + 1, 0);
  cudaError_t e = cudaMemcpyAsync(h.data() + 1, ptr, sizeof(int64_t) * n_tiles, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    dev_free(ptr);
    return cuda_error(e, "tile sizes");
  }
  for (int t = 0; t < n_tiles; ++t) h[t + 1] += h[t];
  const int64_t total = h[n_tiles];
  int32_t *ucol = nullptr;
  float *tval = nullptr;
  e = cudaMemcpyAsync(ptr, h.data(), sizeof(int64_t) * (n_tiles + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = dev_malloc(&ucol, sizeof(int32_t) * std::max<int64_t>(total, 1));
  if (e == cudaSuccess) e = dev_malloc(&tval, sizeof(float) * tile_vs(R, npair) * std::max<int64_t>(total, 1));
  if (e == cudaSuccess) {
    if constexpr (R == 2)
      tile2_merge_warp_kernel<true><<<wgrid, TL_THREADS, 0, s>>>(N, M, npair, P->row_ptr, P->col, v32, P->nnz, ptr,
                                                                  ucol, tval);
    else
      tile_merge_kernel<R, true><<<grid, TL_THREADS, 0, s>>>(N, M, npair, P->row_ptr, P->col, v32, P->nnz, ptr, ucol,
                                                              tval);
    count_launches(1);
    e = cudaGetLastError();
  }
  // the host vector goes when this returns: the copy from it must be done
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    dev_free(ptr);
    dev_free(ucol);
    dev_free(tval);
    return cuda_error(e, "tile build");
  }
  P->tile_ptr[idx] = ptr;
  P->tile_col[idx] = ucol;
  P->tile_val[idx] = tval;
  P->tile_n[idx] = total;
  return WPCD_OK;
}

template <int NCH, int R, int EPT, int FAB>
wpcd_status launch_tile_t(int device, const TileParams &T, const float2 *y, float2 *z, cudaStream_t s) {
  constexpr int NSLOT = R * NCH * EPT * 2;
  const size_t smem = sizeof(float) * 2 * NSLOT * TL_THREADS;
  static bool opted_in = false;  // once per kernel instance, before any graph capture (the tuner's launches)
  if (!opted_in) {
    WPCD_CUDA_TRY(cudaFuncSetAttribute(spmm_tile_kernel<NCH, R, EPT, FAB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    opted_in = true;
  }
  // one tile per warp: the scheduler balances the tiles' uneven column
  // counts (a persistent grid of 8 warps per SM measured 3% slower)
  const int gx = std::max(1, (T.n_tiles + TL_THREADS / 32 - 1) / (TL_THREADS / 32));
  dim3 grid(gx, (T.B + 32 * EPT - 1) / (32 * EPT));
  spmm_tile_kernel<NCH, R, EPT, FAB><<<grid, TL_THREADS, smem, s>>>(T, y, z);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "tile spmm launch");
}

template <int R, int EPT, int FAB>
wpcd_status launch_tile_nch(int device, int n_ch, const TileParams &T, const float2 *y, float2 *z, cudaStream_t s) {
  switch (n_ch) {
    case 1: return launch_tile_t<1, R, EPT, FAB>(device, T, y, z, s);
    case 2: return launch_tile_t<2, R, EPT, FAB>(device, T, y, z, s);
    case 3: return launch_tile_t<3, R, EPT, FAB>(device, T, y, z, s);
    default: return set_error(WPCD_EINVAL, "tile SpMM: up to three channels");
  }
}

}  // namespace

bool tile_supported(const wpcd_problem *pr, int B) { return pr->n_ch <= 3 && B % 2 == 0 && B >= 2; }

wpcd_status tile_prepare(const wpcd_problem *pr, wpcd_P *P, const float *v32, int tile, cudaStream_t s) {
  if (tile == 2) return tile_prepare_r<2>(pr, P, v32, s);
  if (tile == 4) return tile_prepare_r<4>(pr, P, v32, s);
  return set_error(WPCD_EINVAL, "tile SpMM: tiles of 2 or 4 cells");
}

wpcd_status launch_spmm_tile(const wpcd_problem *pr, wpcd_P *P, const float *v32, const float *y, float *z, int B,
                             const SpmmConfig &cfg, cudaStream_t s) {
  if (!tile_supported(pr, B)) return set_error(WPCD_EINVAL, "tile SpMM: even batch and up to three channels");
  if (cfg.tile != 2 && cfg.tile != 4) return set_error(WPCD_EINVAL, "tile SpMM: tiles of 2 or 4 cells");
  wpcd_status st = cfg.tile == 2 ? tile_prepare_r<2>(pr, P, v32, s) : tile_prepare_r<4>(pr, P, v32, s);
  if (st != WPCD_OK) return st;
  const int idx = cfg.tile == 2 ? 0 : 1;
  TileParams T{pr->N * pr->M,
               cfg.tile == 2 ? tile_count<2>(pr->N, pr->M) : tile_count<4>(pr->N, pr->M),
               pr->N,
               pr->M,
               B,
               P->tile_ptr[idx],
               P->tile_col[idx],
               P->tile_val[idx]};
  const float2 *yy = reinterpret_cast<const float2 *>(y);
  float2 *zz = reinterpret_cast<float2 *>(z);
  // tiles of two cells with 4 or 2 energies per lane, of four cells with 2
  // (four rows of 4 energies would need more registers than two CTAs per SM
  // leave); plain blocks of 32 columns, or 64 (cfg.rpw = 2)
  const int d = pr->device, nc = pr->n_ch;
  if (cfg.rpw == 2) {
    if (cfg.tile == 2)
      return cfg.ept == 4 ? launch_tile_nch<2, 4, 64>(d, nc, T, yy, zz, s) : launch_tile_nch<2, 2, 64>(d, nc, T, yy, zz, s);
    return launch_tile_nch<4, 2, 64>(d, nc, T, yy, zz, s);
  }
  if (cfg.tile == 2)
    return cfg.ept == 4 ? launch_tile_nch<2, 4, 32>(d, nc, T, yy, zz, s) : launch_tile_nch<2, 2, 32>(d, nc, T, yy, zz, s);
  return launch_tile_nch<4, 2, 32>(d, nc, T, yy, zz, s);
}

}  // namespace wpcd
