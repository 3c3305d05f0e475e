// Row-block FP32 SpMM of the inner cycles, z = P0 y (Sec. 3.2 Eq. perm,
// applied as in Sec. 3.3), with the gathered rows of y staged in shared
// memory.
//
// Neighbouring rows of P0 share most of their columns: the permutation
// conserves p^2 + 3/4 q^2, so the nonzeros of a row lie on that shell, and
// the 16 rows of a block (one p-bin, 16 consecutive q-bins) hit about 0.41
// distinct columns per nonzero.  A CTA takes one block of 16 rows and a tile
// of 32 energies: it copies the y rows of the block's distinct columns into
// shared memory once, in chunks of 128 columns with coalesced loads, and its
// 16 warps (one row each, one energy per lane) then read them from there.
// The block structure (the sorted distinct columns of each block and, per
// nonzero, the index of its column among them) is built once per matrix by
// spmm_blk_prep_kernel: a shared-memory bitonic sort of the block's column
// indices, a flag-and-scan compaction and a binary search per nonzero.
//
// Sums: each lane forms blocks of 16 nonzeros with plain FMAs and adds them
// to a compensated (TwoSum) accumulator, the FABsum scheme of the other
// FP32 SpMM.
//
// Measured against the warp-per-row kernel (spmm_kernel, tuned shapes) on
// the 3-channel 200 x 200 lattice: 2.03 against 0.92 ms at 128 energies,
// 0.59 against 0.28 ms at 32 (same results to 2e-7).  Staging and use of a
// chunk do not overlap, and a warp keeps only four nonzeros' column and
// value loads in flight, so the kernel is latency-bound; it stays an
// explicit alternative (WPCD_SPMM_FP32_BLOCKED) that the solves do not use.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "common.cuh"
#include "wpcd_internal.h"

namespace wpcd {
namespace {

constexpr int SB_R = 16;        // rows per block (one warp each)
constexpr int SB_T = 32 * SB_R;
constexpr int SB_CAP = 4096;    // column entries of a block sorted in shared memory
constexpr int SB_ET = 32;       // energies per tile (one per lane)
constexpr int SB_UC = 128;      // distinct columns per shared-memory chunk
constexpr int SB_U = 4;         // nonzeros a warp loads together
constexpr int SB_FAB = 16;      // nonzeros per compensated add

// per block b of SB_R rows: nu[b] distinct columns (-1 if more than SB_CAP
// entries: such a block is served by direct gathers), the sorted distinct
// columns at ucol[row_ptr[b SB_R] ..], and per nonzero the index of its
// column among them
__global__ void __launch_bounds__(SB_T) spmm_blk_prep_kernel(int n_cells, const int64_t *__restrict__ row_ptr,
                                                             const int32_t *__restrict__ col, int *__restrict__ nu,
                                                             int32_t *__restrict__ ucol,
                                                             uint16_t *__restrict__ lidx) {
  __shared__ int keys[SB_CAP];
  __shared__ int uniq[SB_CAP];
  __shared__ int wsum[SB_T / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x;
  const int r0 = b * SB_R, r1 = min(r0 + SB_R, n_cells);
  const int64_t o0 = row_ptr[r0], o1 = row_ptr[r1];
  const int m = (int)(o1 - o0);
  if (m > SB_CAP) {  // uniform over the block
    if (tid == 0) nu[b] = -1;
    return;
  }
  int np2 = 1;
  while (np2 < m) np2 <<= 1;
  for (int i = tid; i < np2; i += SB_T) keys[i] = i < m ? col[o0 + i] : INT_MAX;
  __syncthreads();
  // bitonic sort, ascending
  for (int k = 2; k <= np2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < np2; i += SB_T) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int a = keys[i], c = keys[ixj];
          const bool up = (i & k) == 0;
          if ((a > c) == up) {
            keys[i] = c;
            keys[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  // distinct values: each thread takes a contiguous run of PER entries,
  // counts its first occurrences, and a block scan gives their positions
  const int PER = (np2 + SB_T - 1) / SB_T;
  const int i0 = tid * PER;
  int cnt = 0;
  for (int q = 0; q < PER; ++q) {
    const int i = i0 + q;
    if (i < m && (i == 0 || keys[i] != keys[i - 1])) ++cnt;
  }
  int incl = cnt;
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; ++w) before += wsum[w];
  int pos = before + incl - cnt;
  for (int q = 0; q < PER; ++q) {
    const int i = i0 + q;
    if (i < m && (i == 0 || keys[i] != keys[i - 1])) {
      uniq[pos] = keys[i];
      ucol[o0 + pos] = keys[i];
      ++pos;
    }
  }
  __syncthreads();
  int total = 0;
  for (int w = 0; w < SB_T / 32; ++w) total += wsum[w];
  if (tid == 0) nu[b] = total;
  // column index of every nonzero among the block's distinct columns
  for (int i = tid; i < m; i += SB_T) {
    const int c = col[o0 + i];
    int lo = 0, hi = total - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (uniq[mid] < c)
        lo = mid + 1;
      else
        hi = mid;
    }
    lidx[o0 + i] = (uint16_t)lo;
  }
}

// one CTA per (block of SB_R rows, tile of SB_ET energies); warp w owns row
// b SB_R + w, lane e energy tile * SB_ET + e
template <int NCH>
__global__ void __launch_bounds__(SB_T, 2) spmm_blk_kernel(SpmmParams S, const float *__restrict__ val,
                                                           const int *__restrict__ nu,
                                                           const int32_t *__restrict__ ucol,
                                                           const uint16_t *__restrict__ lidx,
                                                           const float2 *__restrict__ y, float2 *__restrict__ z) {
  constexpr int NPAIR = pair_count(NCH);
  extern __shared__ float2 ys[];  // [SB_UC][NCH][SB_ET]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x;
  const int B = S.B, n_cells = S.n_cells;
  const int e0 = blockIdx.y * SB_ET;
  const int en = e0 + lane;
  const int r = b * SB_R + warp;
  const bool row_in = r < n_cells;
  const int64_t ob = S.row_ptr[b * SB_R];
  int64_t cur = row_in ? S.row_ptr[r] : 0;
  const int64_t oe = row_in ? S.row_ptr[r + 1] : 0;
  AccF acc[NCH][2];
  float part[NCH][2];
#pragma unroll
  for (int l = 0; l < NCH; ++l) {
    acc[l][0].zero();
    acc[l][1].zero();
    part[l][0] = part[l][1] = 0.f;
  }
  int np = 0;  // nonzeros in the open block partial
  auto flush = [&]() {
#pragma unroll
    for (int l = 0; l < NCH; ++l) {
      acc[l][0].add(part[l][0]);
      acc[l][1].add(part[l][1]);
      part[l][0] = part[l][1] = 0.f;
    }
    np = 0;
  };
  const int nub = nu[b];
  if (nub < 0) {
    // a block too wide for the shared-memory sort: direct gathers
    for (; cur < oe; ++cur) {
      const int c = S.col[cur];
      float2 q[NCH];
#pragma unroll
      for (int l = 0; l < NCH; ++l)
        q[l] = en < B ? __ldg(y + ((size_t)l * n_cells + c) * B + en) : make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < NPAIR; ++m) {
        const float v = __ldg(val + (size_t)m * S.nnz + cur);
        const int l = pair_first(NCH, m), lp = pair_second(NCH, m);
        part[l][0] = fmaf(v, q[lp].x, part[l][0]);
        part[l][1] = fmaf(v, q[lp].y, part[l][1]);
      }
      if (++np == SB_FAB) flush();
    }
  } else {
    for (int k0 = 0; k0 < nub; k0 += SB_UC) {  // uniform over the CTA
      const int cnt = min(SB_UC, nub - k0);
      // stage the chunk: consecutive threads take consecutive energies of one
      // (column, channel) row of y
      for (int idx = tid; idx < cnt * NCH * SB_ET; idx += SB_T) {
        const int u = idx / (NCH * SB_ET), l = (idx / SB_ET) % NCH, e = idx % SB_ET;
        const int c = __ldg(ucol + ob + k0 + u);
        ys[idx] = e0 + e < B ? __ldg(y + ((size_t)l * n_cells + c) * B + e0 + e) : make_float2(0.f, 0.f);
      }
      __syncthreads();
      // this chunk's nonzeros of the row: a contiguous run from cur (the
      // columns and their indices rise along the row); warp-uniform loop
      const int lim = k0 + cnt;
      while (cur < oe) {
        int li[SB_U];
        float v[SB_U][NPAIR];
#pragma unroll
        for (int u = 0; u < SB_U; ++u) {
          const int64_t o = cur + u;
          const bool ok = o < oe;
          li[u] = ok ? (int)__ldg(lidx + o) : INT_MAX;
#pragma unroll
          for (int m = 0; m < NPAIR; ++m) v[u][m] = ok ? __ldg(val + (size_t)m * S.nnz + o) : 0.f;
        }
        int used = 0;
#pragma unroll
        for (int u = 0; u < SB_U; ++u) {
          if (li[u] < lim) {
            const float2 *q = ys + (size_t)(li[u] - k0) * NCH * SB_ET + lane;
#pragma unroll
            for (int m = 0; m < NPAIR; ++m) {
              const int l = pair_first(NCH, m), lp = pair_second(NCH, m);
              const float2 w = q[lp * SB_ET];
              part[l][0] = fmaf(v[u][m], w.x, part[l][0]);
              part[l][1] = fmaf(v[u][m], w.y, part[l][1]);
            }
            ++used;
          }
        }
        cur += used;
        np += used;
        if (np >= SB_FAB) flush();
        if (used < SB_U) break;  // the rest of the row lies in later chunks
      }
      __syncthreads();
    }
  }
  flush();
  if (row_in && en < B)
#pragma unroll
    for (int l = 0; l < NCH; ++l)
      z[((size_t)l * n_cells + r) * B + en] = make_float2(acc[l][0].value(), acc[l][1].value());
}

bool attr_done[64] = {};

}  // namespace

// the block structure of P0 (once per matrix)
wpcd_status spmm_blk_prepare(const wpcd_problem *pr, wpcd_P *P, cudaStream_t s) {
  if (P->blk_nu) return WPCD_OK;
  const int n_cells = pr->N * pr->M;
  const int nblk = (n_cells + SB_R - 1) / SB_R;
  WPCD_CUDA_TRY(dev_malloc(&P->blk_nu, sizeof(int) * nblk));
  WPCD_CUDA_TRY(dev_malloc(&P->blk_ucol, sizeof(int32_t) * (size_t)P->nnz + 4));
  WPCD_CUDA_TRY(dev_malloc(&P->blk_lidx, sizeof(uint16_t) * (size_t)P->nnz + 4));
  spmm_blk_prep_kernel<<<nblk, SB_T, 0, s>>>(n_cells, P->row_ptr, P->col, P->blk_nu, P->blk_ucol, P->blk_lidx);
  count_launches(1);
  if (pr->device >= 0 && pr->device < 64 && !attr_done[pr->device]) {
    const int bytes = SB_UC * 5 * SB_ET * (int)sizeof(float2);  // up to five channels
    for (auto f : {spmm_blk_kernel<1>, spmm_blk_kernel<2>, spmm_blk_kernel<3>, spmm_blk_kernel<4>,
                   spmm_blk_kernel<5>})
      WPCD_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    attr_done[pr->device] = true;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "row-block SpMM preparation");
}

// z = P0 y, FP32 values and vectors, the row-block kernel (prepared P)
wpcd_status launch_spmm_blk(const wpcd_problem *pr, const wpcd_P *P, const float *vals, const float *y, float *z,
                            int B, cudaStream_t s) {
  if (!P->blk_nu) return set_error(WPCD_EINVAL, "row-block SpMM not prepared");
  SpmmParams S{};
  S.n_cells = pr->N * pr->M;
  S.B = B;
  S.row_ptr = P->row_ptr;
  S.col = P->col;
  S.nnz = P->nnz;
  const int nblk = (S.n_cells + SB_R - 1) / SB_R;
  dim3 grid(nblk, (B + SB_ET - 1) / SB_ET);
  const size_t smem = (size_t)SB_UC * pr->n_ch * SB_ET * sizeof(float2);
  const float2 *y2 = reinterpret_cast<const float2 *>(y);
  float2 *z2 = reinterpret_cast<float2 *>(z);
  switch (pr->n_ch) {
    case 1:
      spmm_blk_kernel<1><<<grid, SB_T, smem, s>>>(S, vals, P->blk_nu, P->blk_ucol, P->blk_lidx, y2, z2);
      break;
    case 2:
      spmm_blk_kernel<2><<<grid, SB_T, smem, s>>>(S, vals, P->blk_nu, P->blk_ucol, P->blk_lidx, y2, z2);
      break;
    case 3:
      spmm_blk_kernel<3><<<grid, SB_T, smem, s>>>(S, vals, P->blk_nu, P->blk_ucol, P->blk_lidx, y2, z2);
      break;
    case 4:
      spmm_blk_kernel<4><<<grid, SB_T, smem, s>>>(S, vals, P->blk_nu, P->blk_ucol, P->blk_lidx, y2, z2);
      break;
    case 5:
      spmm_blk_kernel<5><<<grid, SB_T, smem, s>>>(S, vals, P->blk_nu, P->blk_ucol, P->blk_lidx, y2, z2);
      break;
    default:
      return set_error(WPCD_EINVAL, "unsupported channel count for the SpMM");
  }
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "row-block spmm launch");
}

}  // namespace wpcd
