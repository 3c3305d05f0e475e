// One-right-hand-side SpMV z = P0 y, the sparse step of the K application
// (Sec. 3.3 Eq. kernel; P0 of Sec. 3.2 Eq. perm) for a single energy, in
// FP32 (the mixed solve's inner cycles) or FP64 (the plain iteration).
//
// With one right-hand side every value of P0 is used for one complex
// multiply-add per channel pair, so the step streams the bytes of P0: a
// 4-byte column and n_pairs values per nonzero (24 bytes in FP32 for three
// channels), against a y of a few hundred KB that stays in L2.
//   - `RPW` rows per warp, LPR = 32 / RPW lanes per row (the autotuner's
//     "rows per warp" for one right-hand side: 2, 4, 8 or 16); a lane takes
//     one or two chunks per step (the shape's "energies per lane" field for
//     one right-hand side), their loads issued together;
//   - chunks are four consecutive nonzeros, aligned to four elements, so the
//     columns come in one 16-byte load and the values of each (l, l') pair
//     in 16-, 8- or 4-byte loads (whatever the alignment of the pair-major
//     value array allows); elements of a chunk outside the row get value 0
//     (only the first and last chunk of a row), and a chunk reaching past the
//     end of the arrays takes element loads;
//   - y is gathered per nonzero and channel (three 8-byte FP32 loads for
//     three channels), from L2.
// Measured on the 3-channel 200 x 200 lattice (FP32, L2 flushed): 34 us, 2.2
// TB/s; the limit is the L1 pipeline (about 10 million sector look-ups, of
// which the gathers are two thirds), not DRAM.
// Sums: FP32 lanes sum at most 16 nonzeros plainly and add each such block
// to a compensated accumulator (TwoSum hi, lo), and the lanes of a row are
// combined with TwoSum as well (the FABsum scheme of the batched SpMM);
// FP64 sums plainly.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "wpcd_internal.h"

namespace wpcd {
namespace {

// widest value load the pair-major layout allows at every pair's offset
// m * nnz + o (o a multiple of 4): 4, 2 or 1 elements
template <typename T>
inline int value_width(int64_t nnz) {
  if (sizeof(T) == 4 && nnz % 4 == 0) return 4;
  return nnz % 2 == 0 ? 2 : 1;
}

// running sum of one output: FP32 compensated (hi, lo), FP64 plain
template <typename T>
struct SvSum;
template <>
struct SvSum<float> {
  float hi = 0.f, lo = 0.f;
  __device__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb)));
    hi = s;
  }
  __device__ void add_lane(int off) {
    const float ohi = __shfl_xor_sync(0xffffffffu, hi, off);
    const float olo = __shfl_xor_sync(0xffffffffu, lo, off);
    add(ohi);
    lo = __fadd_rn(lo, olo);
  }
  __device__ float value() const { return __fadd_rn(hi, lo); }
};
template <>
struct SvSum<double> {
  double v = 0.0;
  __device__ void add(double x) { v += x; }
  __device__ void add_lane(int off) { v += __shfl_xor_sync(0xffffffffu, v, off); }
  __device__ double value() const { return v; }
};

// four consecutive values starting at an element index that is a multiple
// of vw (16-, 8- or 4-byte loads; vw is uniform over a launch)
__device__ __forceinline__ void load4(const float *__restrict__ p, float (&v)[4], int vw) {
  if (vw == 4) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
  } else if (vw == 2) {
    const float2 a = __ldg(reinterpret_cast<const float2 *>(p)), b = __ldg(reinterpret_cast<const float2 *>(p + 2));
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __ldg(p + k);
  }
}
__device__ __forceinline__ void load4(const double *__restrict__ p, double (&v)[4], int vw) {
  if (vw >= 2) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p)), b = __ldg(reinterpret_cast<const double2 *>(p + 2));
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __ldg(p + k);
  }
}

// one chunk of four consecutive nonzeros at element o (a multiple of 4):
// columns and the values of every (l, l') pair; a chunk reaching past the end
// of the arrays takes element loads (column 0, value 0 beyond the end)
template <typename T, int NPAIR>
__device__ __forceinline__ void load_chunk(const int32_t *__restrict__ col, const T *__restrict__ val, int64_t nnz,
                                           int64_t o, int (&t)[4], T (&v)[NPAIR][4], int vw) {
  if (o + 4 <= nnz) {
    const int4 cc = __ldg(reinterpret_cast<const int4 *>(col + o));
    t[0] = cc.x, t[1] = cc.y, t[2] = cc.z, t[3] = cc.w;
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) load4(val + (size_t)m * nnz + o, v[m], vw);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool in = o + k < nnz;
      t[k] = in ? __ldg(col + o + k) : 0;
#pragma unroll
      for (int m = 0; m < NPAIR; ++m) v[m][k] = in ? __ldg(val + (size_t)m * nnz + o + k) : T(0);
    }
  }
}

// y of every channel at cell t (layout y[l][c])
template <typename T, int NCH>
__device__ __forceinline__ void gather_y(const typename Cx<T>::t *__restrict__ y, int n_cells, int t, T (&yr)[NCH],
                                         T (&yim)[NCH]) {
#pragma unroll
  for (int l = 0; l < NCH; ++l) {
    const typename Cx<T>::t q = __ldg(y + (size_t)l * n_cells + t);
    yr[l] = q.x, yim[l] = q.y;
  }
}

// the chunk's products into the row partials.  Elements outside the row
// [b, e) get value 0: their column is still a valid cell (the column array
// holds cell indices everywhere, and 0 past its end), so the gather stays
// in bounds and no lane branches inside a chunk.
template <typename T, int NCH, int NPAIR>
__device__ __forceinline__ void use_chunk(const typename Cx<T>::t *__restrict__ y, int n_cells, int64_t o, int64_t b,
                                          int64_t e, const int (&t)[4], T (&v)[NPAIR][4], T (&part)[NCH][2]) {
  using C2 = typename Cx<T>::t;
  if (o < b || o + 4 > e) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool in = o + k >= b && o + k < e;
#pragma unroll
      for (int m = 0; m < NPAIR; ++m) v[m][k] = in ? v[m][k] : T(0);
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T yr[NCH], yi[NCH];
    gather_y<T, NCH>(y, n_cells, t[k], yr, yi);
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) {
      const int l = pair_first(NCH, m), lp = pair_second(NCH, m);
      part[l][0] = fma(v[m][k], yr[lp], part[l][0]);
      part[l][1] = fma(v[m][k], yi[lp], part[l][1]);
    }
  }
}

// CPS chunks per step: 1 (for up to three channels three FP32 / two FP64
// CTAs of 256 threads per SM) or 2 (their loads in flight together, about
// twice the registers; up to three channels)
template <typename T, int NCH, int RPW, int CPS>
__global__ void __launch_bounds__(256, CPS == 1 && NCH <= 3 ? (sizeof(T) == 4 ? 3 : 2) : 1)
    spmv_kernel(int n_cells, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                const T *__restrict__ val, int64_t nnz, const typename Cx<T>::t *__restrict__ y,
                typename Cx<T>::t *__restrict__ z, int vw) {
  using C2 = typename Cx<T>::t;
  constexpr int NPAIR = pair_count(NCH);
  constexpr int LPR = 32 / RPW;
  // FP32: plain sums over blocks of 16 nonzeros per lane, each block added to
  // the compensated accumulator
  constexpr int BLK = sizeof(T) == 4 ? 4 / CPS : 1 << 30;  // steps per plain block
  const int lane = threadIdx.x & 31, sub = lane % LPR;
  const int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW + lane / LPR;
  const bool active = c < n_cells;
  const int64_t b = active ? __ldg(row_ptr + c) : 0, e = active ? __ldg(row_ptr + c + 1) : 0;
  SvSum<T> acc[NCH][2];
  T part[NCH][2];
#pragma unroll
  for (int l = 0; l < NCH; ++l) part[l][0] = part[l][1] = T(0);
  int nblk = 0;
  // CPS chunks per step (their loads issued together), LPR lanes apart
  constexpr int64_t STEP = 4 * CPS * LPR;
  for (int64_t o = (b & ~(int64_t)3) + 4 * sub; o < e; o += STEP) {
    int t0[4], t1[4];
    T v0[NPAIR][4], v1[NPAIR][4];
    const int64_t o1 = o + 4 * LPR;
    const bool second = CPS == 2 && o1 < e;
    load_chunk<T, NPAIR>(col, val, nnz, o, t0, v0, vw);
    if (second) load_chunk<T, NPAIR>(col, val, nnz, o1, t1, v1, vw);
    use_chunk<T, NCH, NPAIR>(y, n_cells, o, b, e, t0, v0, part);
    if (second) use_chunk<T, NCH, NPAIR>(y, n_cells, o1, b, e, t1, v1, part);
    if (++nblk == BLK) {
      nblk = 0;
#pragma unroll
      for (int l = 0; l < NCH; ++l) {
        acc[l][0].add(part[l][0]);
        acc[l][1].add(part[l][1]);
        part[l][0] = part[l][1] = T(0);
      }
    }
  }
#pragma unroll
  for (int l = 0; l < NCH; ++l) {
    acc[l][0].add(part[l][0]);
    acc[l][1].add(part[l][1]);
  }
  // the LPR lanes of a row are consecutive: xor offsets below LPR stay in it
#pragma unroll
  for (int off = 1; off < LPR; off <<= 1)
#pragma unroll
    for (int l = 0; l < NCH; ++l) {
      acc[l][0].add_lane(off);
      acc[l][1].add_lane(off);
    }
  if (active && sub == 0)
#pragma unroll
    for (int l = 0; l < NCH; ++l) {
      C2 out;
      out.x = acc[l][0].value();
      out.y = acc[l][1].value();
      z[(size_t)l * n_cells + c] = out;
    }
}

template <typename T, int NCH, int RPW, int CPS>
void launch_vw(int n_cells, const int64_t *row_ptr, const int32_t *col, const T *val, int64_t nnz, const void *y,
               void *z, cudaStream_t s) {
  using C2 = typename Cx<T>::t;
  const int rows_per_cta = 8 * RPW;
  const unsigned grid = (unsigned)((n_cells + rows_per_cta - 1) / rows_per_cta);
  spmv_kernel<T, NCH, RPW, CPS><<<grid, 256, 0, s>>>(n_cells, row_ptr, col, val, nnz, static_cast<const C2 *>(y),
                                                    static_cast<C2 *>(z), value_width<T>(nnz));
}

template <typename T, int NCH, int CPS>
void launch_rpw(int rpw, int n_cells, const int64_t *row_ptr, const int32_t *col, const T *val, int64_t nnz,
                const void *y, void *z, cudaStream_t s) {
  switch (rpw) {
    case 2: launch_vw<T, NCH, 2, CPS>(n_cells, row_ptr, col, val, nnz, y, z, s); break;
    case 4: launch_vw<T, NCH, 4, CPS>(n_cells, row_ptr, col, val, nnz, y, z, s); break;
    case 8: launch_vw<T, NCH, 8, CPS>(n_cells, row_ptr, col, val, nnz, y, z, s); break;
    default: launch_vw<T, NCH, 16, CPS>(n_cells, row_ptr, col, val, nnz, y, z, s); break;
  }
}

template <typename T, int NCH>
void launch_cps(int cps, int rpw, int n_cells, const int64_t *row_ptr, const int32_t *col, const T *val,
                int64_t nnz, const void *y, void *z, cudaStream_t s) {
  if constexpr (NCH <= 3) {
    if (cps == 2) {
      launch_rpw<T, NCH, 2>(rpw, n_cells, row_ptr, col, val, nnz, y, z, s);
      return;
    }
  }
  launch_rpw<T, NCH, 1>(rpw, n_cells, row_ptr, col, val, nnz, y, z, s);
}

template <typename T>
wpcd_status launch_spmv_t(int n_ch, int rpw, int cps, int n_cells, const int64_t *row_ptr, const int32_t *col, const T *val,
                          int64_t nnz, const void *y, void *z, cudaStream_t s) {
  switch (n_ch) {
    case 1: launch_cps<T, 1>(cps, rpw, n_cells, row_ptr, col, val, nnz, y, z, s); break;
    case 2: launch_cps<T, 2>(cps, rpw, n_cells, row_ptr, col, val, nnz, y, z, s); break;
    case 3: launch_cps<T, 3>(cps, rpw, n_cells, row_ptr, col, val, nnz, y, z, s); break;
    case 4: launch_cps<T, 4>(cps, rpw, n_cells, row_ptr, col, val, nnz, y, z, s); break;
    case 5: launch_cps<T, 5>(cps, rpw, n_cells, row_ptr, col, val, nnz, y, z, s); break;
    default: return set_error(WPCD_EINVAL, "SpMV: unsupported channel count");
  }
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "spmv launch");
}

}  // namespace

wpcd_status launch_spmv1(const wpcd_problem *pr, const wpcd_P *P, bool fp64, const void *val, const void *y, void *z,
                         const SpmmConfig &cfg, cudaStream_t s) {
  const int n_cells = pr->N * pr->M;
  if (fp64)
    return launch_spmv_t<double>(pr->n_ch, cfg.rpw, cfg.ept, n_cells, P->row_ptr, P->col,
                                 static_cast<const double *>(val), P->nnz, y, z, s);
  return launch_spmv_t<float>(pr->n_ch, cfg.rpw, cfg.ept, n_cells, P->row_ptr, P->col, static_cast<const float *>(val),
                              P->nnz, y, z, s);
}

}  // namespace wpcd
