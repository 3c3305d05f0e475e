// Float-float pieces shared by the single-problem residual (df.cu) and the
// grouped residual (group.cu): hi + lo float arithmetic (TwoProduct by FMA,
// Knuth's TwoSum, Fast2Sum renormalisation), the FP64 -> float-float split
// kernels, the 32 x 128 block-product tile and the SpMM row sums.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace wpcd {
namespace {

// Knuth's TwoSum of (hi, p) with the error folded into lo together with e
__device__ __forceinline__ void df_add(float &hi, float &lo, float p, float e) {
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// (ah + al)(bh + bl) = p + e: p the rounded product, e its exact error
// (TwoProduct by FMA) plus the cross terms; al bl is below the precision
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &p, float &e) {
  p = __fmul_rn(ah, bh);
  e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
}

// renormalise (hi, lo) so that |lo| <= ulp(hi) / 2 (Fast2Sum)
__device__ __forceinline__ void df_norm(float &hi, float &lo) {
  const float s = __fadd_rn(hi, lo);
  lo = __fsub_rn(lo, __fsub_rn(s, hi));
  hi = s;
}

__global__ void df_split_kernel(int64_t n, const double *__restrict__ x, float *__restrict__ hi,
                                float *__restrict__ lo) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[f];
    const float h = f64_to_f32_rn(v);
    hi[f] = h;
    lo[f] = f64_to_f32_rn(v - f32_to_f64(h));
  }
}

// panel = G1 o x (complex, FP64), split into float-float real arrays
__global__ void df_split_scaled_kernel(int64_t nc, const double2 *__restrict__ x, const double2 *__restrict__ g,
                                       float *__restrict__ hi, float *__restrict__ lo) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nc; f += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = x[f];
    double2 v = a;
    if (g) {
      const double2 b = g[f];
      v = make_double2(b.x * a.x - b.y * a.y, b.x * a.y + b.y * a.x);
    }
    const float hr = f64_to_f32_rn(v.x), hm = f64_to_f32_rn(v.y);
    reinterpret_cast<float2 *>(hi)[f] = make_float2(hr, hm);
    reinterpret_cast<float2 *>(lo)[f] =
        make_float2(f64_to_f32_rn(v.x - f32_to_f64(hr)), f64_to_f32_rn(v.y - f32_to_f64(hm)));
  }
}

// C[b] (n x ncol) = A[b] (n x n) B[b] (n x ncol) in float-float: 32 x 128
// outputs per CTA, 2 x 8 per thread (rows ty, ty + 16; columns 4 tx .. 4 tx
// + 3 and 64 + 4 tx .. + 3), so that a k step reads the panel with two
// 16-byte loads per part; 16-deep K tiles in shared memory.
// OUT_DF: C as a float-float pair (Ch, Cl); otherwise FP64 C.
constexpr int DF_N = 128;

struct DfGemmSmem {
  float sAh[GB_K][GB_M + 1], sAl[GB_K][GB_M + 1];
  __align__(16) float sBh[GB_K][DF_N], sBl[GB_K][DF_N];
};

// one 32 x 128 output tile; A, B, C (or Ch, Cl) at the channel block's
// origin (offA = offB = 0 below), rows row0.., columns col0..
template <bool OUT_DF>
__device__ __forceinline__ void gemm_df_tile(int n, int64_t ncol, const float *__restrict__ Ah,
                                             const float *__restrict__ Al, const float *__restrict__ Bh,
                                             const float *__restrict__ Bl, double *__restrict__ C,
                                             float *__restrict__ Ch, float *__restrict__ Cl, int row0, int64_t col0,
                                             DfGemmSmem &sm) {
  auto &sAh = sm.sAh;
  auto &sAl = sm.sAl;
  auto &sBh = sm.sBh;
  auto &sBl = sm.sBl;
  const size_t offA = 0, offB = 0;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  // 16-byte aligned panel rows (the grouped solve's segments may start on 8 bytes)
  const bool vec = ncol % 4 == 0 && ((reinterpret_cast<uintptr_t>(Bh) | reinterpret_cast<uintptr_t>(Bl)) & 15) == 0;
  float hi[2][8], lo[2][8];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) hi[u][v] = lo[u][v] = 0.f;
  for (int k0 = 0; k0 < n; k0 += GB_K) {
    for (int t = threadIdx.x; t < GB_M * GB_K; t += G_THREADS) {
      const int r = t / GB_K, kk = t % GB_K;
      const int gr = row0 + r, gk = k0 + kk;
      const bool in = gr < n && gk < n;
      const size_t o = offA + (size_t)gr * n + gk;
      sAh[kk][r] = in ? Ah[o] : 0.f;
      sAl[kk][r] = in ? Al[o] : 0.f;
    }
    if (vec) {
      for (int t = threadIdx.x; t < GB_K * DF_N / 4; t += G_THREADS) {
        const int kk = t / (DF_N / 4), c4 = (t % (DF_N / 4)) * 4;
        const int gk = k0 + kk;
        const int64_t gc = col0 + c4;
        float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
        if (gk < n && gc < ncol) {  // ncol % 4 == 0: the four columns are all in or all out
          const size_t o = offB + (size_t)gk * ncol + gc;
          h = *reinterpret_cast<const float4 *>(Bh + o);
          l = *reinterpret_cast<const float4 *>(Bl + o);
        }
        *reinterpret_cast<float4 *>(&sBh[kk][c4]) = h;
        *reinterpret_cast<float4 *>(&sBl[kk][c4]) = l;
      }
    } else {
      for (int t = threadIdx.x; t < GB_K * DF_N; t += G_THREADS) {
        const int kk = t / DF_N, cc = t % DF_N;
        const int gk = k0 + kk;
        const int64_t gc = col0 + cc;
        const bool in = gk < n && gc < ncol;
        const size_t o = offB + (size_t)gk * ncol + gc;
        sBh[kk][cc] = in ? Bh[o] : 0.f;
        sBl[kk][cc] = in ? Bl[o] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GB_K; ++kk) {
      float ah[2], al[2], bh[8], bl[8];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        ah[u] = sAh[kk][ty + 16 * u];
        al[u] = sAl[kk][ty + 16 * u];
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 qh = *reinterpret_cast<const float4 *>(&sBh[kk][64 * h + 4 * tx]);
        const float4 ql = *reinterpret_cast<const float4 *>(&sBl[kk][64 * h + 4 * tx]);
        bh[4 * h] = qh.x;
        bh[4 * h + 1] = qh.y;
        bh[4 * h + 2] = qh.z;
        bh[4 * h + 3] = qh.w;
        bl[4 * h] = ql.x;
        bl[4 * h + 1] = ql.y;
        bl[4 * h + 2] = ql.z;
        bl[4 * h + 3] = ql.w;
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          float p, e;
          df_mul(ah[u], al[u], bh[v], bl[v], p, e);
          df_add(hi[u][v], lo[u][v], p, e);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int gr = row0 + ty + 16 * u;
      const int64_t gc = col0 + 64 * (v / 4) + 4 * tx + (v % 4);
      if (gr < n && gc < ncol) {
        const size_t o = offB + (size_t)gr * ncol + gc;
        float h = hi[u][v], l = lo[u][v];
        df_norm(h, l);
        if (OUT_DF) {
          Ch[o] = h;
          Cl[o] = l;
        } else {
          C[o] = (double)h + (double)l;
        }
      }
    }
}

// The float-float sums of one block-CSR row for the SpMM kernels (the lane
// layout of spmm_row: nonzero lanes nl of nl_count, EPT energies per lane
// at en0 + estride t); values pre-split (vl NULL for FP32-valued matrices,
// whose values are exact in hi); y at the problem's own vector block
template <int NCH, int EPT>
__device__ __forceinline__ void spmm_df_row(int64_t b, int64_t e, int nl, int nl_count, const int32_t *__restrict__ col,
                                            const float *__restrict__ vh, const float *__restrict__ vl, int64_t nnz,
                                            const float2 *__restrict__ yh, const float2 *__restrict__ yl, int n_cells,
                                            int B, int en0, int estride, float (&ah)[NCH][EPT][2],
                                            float (&al)[NCH][EPT][2]) {
  constexpr int NPAIR = pair_count(NCH);
  for (int64_t o = b + nl; o < e; o += nl_count) {
    const int tc = __ldg(col + o);
    float wh[NPAIR], wl[NPAIR];
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) {
      wh[m] = __ldg(vh + (size_t)m * nnz + o);
      wl[m] = vl ? __ldg(vl + (size_t)m * nnz + o) : 0.f;
    }
#pragma unroll
    for (int t = 0; t < EPT; ++t) {
      const int en = en0 + estride * t;
      if (en < B) {
        float2 qh[NCH], ql[NCH];
#pragma unroll
        for (int l = 0; l < NCH; ++l) {
          const size_t yo = ((size_t)l * n_cells + tc) * B + en;
          qh[l] = __ldg(yh + yo);
          ql[l] = __ldg(yl + yo);
        }
#pragma unroll
        for (int m = 0; m < NPAIR; ++m) {
          const int l = pair_first(NCH, m), lp = pair_second(NCH, m);
          float p, er;
          df_mul(wh[m], wl[m], qh[lp].x, ql[lp].x, p, er);
          df_add(ah[l][t][0], al[l][t][0], p, er);
          df_mul(wh[m], wl[m], qh[lp].y, ql[lp].y, p, er);
          df_add(ah[l][t][1], al[l][t][1], p, er);
        }
      }
    }
  }
}

// reduce a row's float-float sums over its nonzero lanes (xor offsets el_n
// .. lpr/2) and write them renormalised to (zh, zl)
template <int NCH, int EPT>
__device__ __forceinline__ void spmm_df_finish(int el_n, int lpr, bool write, float (&ah)[NCH][EPT][2],
                                               float (&al)[NCH][EPT][2], float2 *__restrict__ zh,
                                               float2 *__restrict__ zl, int n_cells, int c, int B, int en0,
                                               int estride) {
  for (int off = el_n; off < lpr; off <<= 1)
#pragma unroll
    for (int l = 0; l < NCH; ++l)
#pragma unroll
      for (int t = 0; t < EPT; ++t)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float oh = __shfl_xor_sync(0xffffffffu, ah[l][t][q], off);
          const float ol = __shfl_xor_sync(0xffffffffu, al[l][t][q], off);
          df_add(ah[l][t][q], al[l][t][q], oh, ol);
        }
  if (!write) return;
#pragma unroll
  for (int t = 0; t < EPT; ++t) {
    const int en = en0 + estride * t;
    if (en < B)
#pragma unroll
      for (int l = 0; l < NCH; ++l) {
        float hr = ah[l][t][0], lr = al[l][t][0], hm = ah[l][t][1], lm = al[l][t][1];
        df_norm(hr, lr);
        df_norm(hm, lm);
        const size_t zo = ((size_t)l * n_cells + c) * B + en;
        zh[zo] = make_float2(hr, hm);
        zl[zo] = make_float2(lr, lm);
      }
  }
}

}  // namespace
}  // namespace wpcd
