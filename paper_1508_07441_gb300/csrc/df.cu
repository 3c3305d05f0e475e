// Float-float K application for the refinement residual of the mixed solve
// (Sec. 3.3, Eq. kernel: K = O P0 Vt G1).
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so in the mixed solve the FP64
// K applications (Born term, refinement residuals) cost more than all the
// FP32 inner cycles.  Here they run on the FP32 pipe in float-float
// arithmetic: every FP64 operand x is held as an unevaluated sum hi + lo of
// two floats (hi = fl(x), lo = fl(x - hi); about 48 significant bits), a
// product a b as p + e with p = fl(a_h b_h) and e the exact error of p
// (TwoProduct with an FMA) plus the cross terms a_h b_l + a_l b_h, and sums
// are carried with Knuth's TwoSum.  The result is FP64-class: relative
// error ~1e-14, far below the 1e-10 residual tolerance of the refinement.
//
//   df_split_scaled_kernel  (G1 o x) in FP64 -> float-float panel
//   gemm_df_kernel          C = A B for every channel block, A = Vt or O
//                           pre-split once per problem
//   spmm_df_kernel          z = P0 y, P0 values pre-split once per matrix
// The intermediates stay float-float; the last product writes FP64.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "df_common.cuh"
#include "wpcd_internal.h"

namespace wpcd {
namespace {

template <bool OUT_DF>
__global__ void __launch_bounds__(G_THREADS) gemm_df_kernel(int n, int64_t ncol, const float *__restrict__ Ah,
                                                            const float *__restrict__ Al,
                                                            const float *__restrict__ Bh,
                                                            const float *__restrict__ Bl, double *__restrict__ C,
                                                            float *__restrict__ Ch, float *__restrict__ Cl) {
  __shared__ DfGemmSmem sm;
  const int b = blockIdx.z;
  const size_t offA = (size_t)b * n * n, offB = (size_t)b * n * ncol;
  gemm_df_tile<OUT_DF>(n, ncol, Ah + offA, Al + offA, Bh + offB, Bl + offB, OUT_DF ? nullptr : C + offB,
                       OUT_DF ? Ch + offB : nullptr, OUT_DF ? Cl + offB : nullptr, blockIdx.y * GB_M,
                       (int64_t)blockIdx.x * DF_N, sm);
}

// z = P0 y in float-float: the SpMM lane layout (rows per warp, energy
// lanes, nonzero lanes, EPT strided energies per lane)
template <int NCH, int EPT>
__global__ void __launch_bounds__(256) spmm_df_kernel(SpmmParams S, const float *__restrict__ vh,
                                                      const float *__restrict__ vl, const float2 *__restrict__ yh,
                                                      const float2 *__restrict__ yl, float2 *__restrict__ zh,
                                                      float2 *__restrict__ zl) {
  const int lane = threadIdx.x & 31;
  const int lpr = 32 / S.rpw, nl_count = lpr / S.el;
  const int r_in = lane / lpr, sub = lane % lpr;
  const int el = sub % S.el, nl = sub / S.el;
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int n_warps = gridDim.x * blockDim.x / 32;
  const int e_base = blockIdx.y * S.el * EPT;
  for (int base = warp_global * S.rpw; base < S.n_cells; base += n_warps * S.rpw) {
    const int c = base + r_in;
    const bool active = c < S.n_cells;
    float ah[NCH][EPT][2], al[NCH][EPT][2];
#pragma unroll
    for (int l = 0; l < NCH; ++l)
#pragma unroll
      for (int t = 0; t < EPT; ++t) ah[l][t][0] = ah[l][t][1] = al[l][t][0] = al[l][t][1] = 0.f;
    const int64_t b = active ? S.row_ptr[c] : 0, e = active ? S.row_ptr[c + 1] : 0;
    spmm_df_row<NCH, EPT>(b, e, nl, nl_count, S.col, vh, vl, S.nnz, yh, yl, S.n_cells, S.B, e_base + el, S.el, ah,
                          al);
    spmm_df_finish<NCH, EPT>(S.el, lpr, active && nl == 0, ah, al, zh, zl, S.n_cells, c, S.B, e_base + el, S.el);
  }
}

// Vt e0 per energy in float-float: column 0 of Vt_0 at (channel 0, q-bin j0)
__global__ void df_born_vt_kernel(int64_t n, int B, int N, int M, const float *Vh, const float *Vl, const int *r0,
                                  float2 *yh, float2 *yl) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(f % B);
    const int64_t r = f / B;
    float h = 0.f, l = 0.f;
    if (r < (int64_t)N * M && (int)(r % M) == r0[e]) {
      h = Vh[(r / M) * N];
      l = Vl[(r / M) * N];
    }
    yh[f] = make_float2(h, 0.f);
    yl[f] = make_float2(l, 0.f);
  }
}

__global__ void df_join_kernel(int64_t n, const float *__restrict__ hi, const float *__restrict__ lo,
                               double *__restrict__ x) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x)
    x[f] = (double)hi[f] + (double)lo[f];
}

template <bool OUT_DF>
wpcd_status gemm_df_simt(const wpcd_problem *pr, bool use_O, const float *Bh, const float *Bl, double *C, float *Ch,
                         float *Cl, int64_t ncol, cudaStream_t s) {
  const int N = pr->N;
  dim3 grid((unsigned)((ncol + DF_N - 1) / DF_N), (N + GB_M - 1) / GB_M, pr->n_ch);
  gemm_df_kernel<OUT_DF><<<grid, G_THREADS, 0, s>>>(N, ncol, use_O ? pr->d.O_h : pr->d.Vt_h,
                                                    use_O ? pr->d.O_l : pr->d.Vt_l, Bh, Bl, C, Ch, Cl);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "float-float gemm launch");
}

// the channel-block products of the float-float K application: from bf16
// digit planes on the tensor cores where prepared (oz_gemm.cu, N <= 256),
// else float-float on the FP32 pipe
template <bool OUT_DF>
wpcd_status gemm_df(const wpcd_problem *pr, bool use_O, const float *Bh, const float *Bl, double *C, float *Ch,
                    float *Cl, int64_t ncol, cudaStream_t s) {
  if (pr->d.O_oz && oz_enabled()) return oz_gemm(pr, use_O, Bh, Bl, C, Ch, Cl, ncol, s);
  return gemm_df_simt<OUT_DF>(pr, use_O, Bh, Bl, C, Ch, Cl, ncol, s);
}

}  // namespace

// the float-float SpMM with a given launch shape
wpcd_status launch_spmm_df_cfg(const wpcd_problem *pr, const wpcd_P *P, const float *yh, const float *yl,
                               float *zh, float *zl, int B, const SpmmConfig &cfg, cudaStream_t s) {
  SpmmParams S{};
  S.n_cells = pr->N * pr->M;
  S.B = B;
  S.rpw = cfg.rpw;
  S.el = cfg.el;
  S.row_ptr = P->row_ptr;
  S.col = P->col;
  S.nnz = P->nnz;
  const float *vh = P->prec == WPCD_FP64 ? P->val_h : P->val32;
  const float *vl = P->prec == WPCD_FP64 ? P->val_l : nullptr;
  const float2 *y2h = reinterpret_cast<const float2 *>(yh), *y2l = reinterpret_cast<const float2 *>(yl);
  float2 *z2h = reinterpret_cast<float2 *>(zh), *z2l = reinterpret_cast<float2 *>(zl);
  dim3 grid(grid_for((int64_t)S.n_cells, 8 * cfg.rpw, 152 * 16), (B + cfg.el * cfg.ept - 1) / (cfg.el * cfg.ept));
#define WPCD_DF_EPT(NCH, EPT) spmm_df_kernel<NCH, EPT><<<grid, 256, 0, s>>>(S, vh, vl, y2h, y2l, z2h, z2l)
#define WPCD_DF_CASE(NCH)  \
  case NCH:                \
    if (cfg.ept == 1)      \
      WPCD_DF_EPT(NCH, 1); \
    else if (cfg.ept == 2) \
      WPCD_DF_EPT(NCH, 2); \
    else                   \
      WPCD_DF_EPT(NCH, 4); \
    break;
  switch (pr->n_ch) {
    WPCD_DF_CASE(1)
    WPCD_DF_CASE(2)
    WPCD_DF_CASE(3)
    WPCD_DF_CASE(4)
    WPCD_DF_CASE(5)
    default:
      return set_error(WPCD_EINVAL, "unsupported channel count for the SpMM");
  }
#undef WPCD_DF_CASE
#undef WPCD_DF_EPT
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "float-float spmm launch");
}

namespace {

// the float-float SpMM with the autotuner's shape for this batch
wpcd_status spmm_df(const wpcd_problem *pr, const wpcd_P *P, const float *yh, const float *yl, float *zh, float *zl,
                    int B, cudaStream_t s) {
  SpmmConfig cfg;
  wpcd_status st = tune_spmm(pr, const_cast<wpcd_P *>(P), B, 2, s, &cfg);
  if (st != WPCD_OK) return st;
  return launch_spmm_df_cfg(pr, P, yh, yl, zh, zl, B, cfg, s);
}

}  // namespace

DfWork::~DfWork() {
  pool_free(xh, st);
  pool_free(xl, st);
  pool_free(yh, st);
  pool_free(yl, st);
}

cudaError_t DfWork::alloc(size_t dim, int B, cudaStream_t s) {
  const size_t bytes = 2 * sizeof(float) * dim * (size_t)B;
  st = s;
  cudaError_t e;
  if ((e = pool_malloc(&xh, bytes, s)) != cudaSuccess) return e;
  if ((e = pool_malloc(&xl, bytes, s)) != cudaSuccess) return e;
  if ((e = pool_malloc(&yh, bytes, s)) != cudaSuccess) return e;
  return pool_malloc(&yl, bytes, s);
}

// split O, Vt (once per problem) and FP64 P0 values (once per matrix)
wpcd_status df_prepare(wpcd_problem *pr, wpcd_P *P, cudaStream_t s, bool digits) {
  const int64_t nmat = (int64_t)pr->n_ch * pr->N * pr->N;
  if (!pr->d.O_h) {
    WPCD_CUDA_TRY(dev_malloc(&pr->d.O_h, sizeof(float) * nmat));
    WPCD_CUDA_TRY(dev_malloc(&pr->d.O_l, sizeof(float) * nmat));
    WPCD_CUDA_TRY(dev_malloc(&pr->d.Vt_h, sizeof(float) * nmat));
    WPCD_CUDA_TRY(dev_malloc(&pr->d.Vt_l, sizeof(float) * nmat));
    df_split_kernel<<<grid_for(nmat, 256), 256, 0, s>>>(nmat, pr->d.O, pr->d.O_h, pr->d.O_l);
    df_split_kernel<<<grid_for(nmat, 256), 256, 0, s>>>(nmat, pr->d.Vt, pr->d.Vt_h, pr->d.Vt_l);
    count_launches(2);
  }
  // digit planes of O and Vt for the tensor-core products
  if (digits && oz_supported(pr) && oz_enabled()) {
    wpcd_status st = oz_prepare(pr, s);
    if (st != WPCD_OK) return st;
  }
  if (P && P->prec == WPCD_FP64 && !P->val_h) {
    const int64_t nv = (int64_t)P->nnz * P->n_pairs;
    WPCD_CUDA_TRY(dev_malloc(&P->val_h, sizeof(float) * nv + 4));
    WPCD_CUDA_TRY(dev_malloc(&P->val_l, sizeof(float) * nv + 4));
    df_split_kernel<<<grid_for(nv, 256), 256, 0, s>>>(nv, P->val64, P->val_h, P->val_l);
    count_launches(1);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "float-float split");
}

// out = K x = O P0 Vt (g o x) for a batch of B energies, FP64 in and out,
// float-float inside
wpcd_status df_kapply(const wpcd_problem *pr, const wpcd_P *P, const double *g, const double *x, double *out, int B,
                      DfWork &w, cudaStream_t s) {
  const int64_t nc = (int64_t)pr->n_ch * pr->N * pr->M * B;  // complex elements
  const int64_t ncol = 2LL * pr->M * B;
  df_split_scaled_kernel<<<grid_for(nc, 256), 256, 0, s>>>(nc, reinterpret_cast<const double2 *>(x),
                                                          reinterpret_cast<const double2 *>(g), w.xh, w.xl);
  count_launches(1);
  wpcd_status st = gemm_df<true>(pr, false, w.xh, w.xl, nullptr, w.yh, w.yl, ncol, s);
  if (st != WPCD_OK) return st;
  st = spmm_df(pr, P, w.yh, w.yl, w.xh, w.xl, B, s);
  if (st != WPCD_OK) return st;
  st = gemm_df<false>(pr, true, w.xh, w.xl, out, nullptr, nullptr, ncol, s);
  if (st != WPCD_OK) return st;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "float-float kapply launch");
}

// y = A (g o x) per channel block in float-float, FP64 in and out
wpcd_status df_gemm_op(wpcd_problem *pr, bool use_O, bool digits, const double *g, const double *x, double *y, int B,
                       float *ms, cudaStream_t s) {
  wpcd_status st = df_prepare(pr, nullptr, s);
  if (st != WPCD_OK) return st;
  if (digits) {
    if (!oz_supported(pr)) return set_error(WPCD_EINVAL, "the digit-plane tensor-core GEMM needs N <= 256");
    st = oz_prepare(pr, s);
    if (st == WPCD_OK) st = tc_clear(pr, s);
    if (st != WPCD_OK) return st;
  }
  const size_t dim = (size_t)pr->n_ch * pr->N * pr->M;
  DfWork w;
  WPCD_CUDA_TRY(w.alloc(dim, B, s));
  const int64_t nc = (int64_t)dim * B;
  df_split_scaled_kernel<<<grid_for(nc, 256), 256, 0, s>>>(nc, reinterpret_cast<const double2 *>(x),
                                                          reinterpret_cast<const double2 *>(g), w.xh, w.xl);
  count_launches(1);
  {
    LaunchTimer t(ms, s);
    t.start();
    st = digits ? oz_gemm(pr, use_O, w.xh, w.xl, y, nullptr, nullptr, 2LL * pr->M * B, s)
                : gemm_df_simt<false>(pr, use_O, w.xh, w.xl, y, nullptr, nullptr, 2LL * pr->M * B, s);
    t.stop();
  }
  if (st != WPCD_OK) return st;
  if (digits) {
    st = tc_check(pr, s);
    if (st != WPCD_OK) return st;
  }
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));  // the work space is freed on return
  return WPCD_OK;
}

// z = P0 y in float-float, FP64 in and out
wpcd_status df_spmm_op(wpcd_problem *pr, wpcd_P *P, const double *y, double *z, int B, float *ms, cudaStream_t s) {
  wpcd_status st = df_prepare(pr, P, s);
  if (st != WPCD_OK) return st;
  const size_t dim = (size_t)pr->n_ch * pr->N * pr->M;
  const int64_t nr = 2LL * (int64_t)dim * B;  // reals
  DfWork w;
  WPCD_CUDA_TRY(w.alloc(dim, B, s));
  df_split_kernel<<<grid_for(nr, 256), 256, 0, s>>>(nr, y, w.yh, w.yl);
  count_launches(1);
  {
    SpmmConfig cfg;  // tune outside the timed launch
    st = tune_spmm(pr, P, B, 2, s, &cfg);
    if (st != WPCD_OK) return st;
    LaunchTimer t(ms, s);
    t.start();
    st = spmm_df(pr, P, w.yh, w.yl, w.xh, w.xl, B, s);
    t.stop();
  }
  if (st != WPCD_OK) return st;
  df_join_kernel<<<grid_for(nr, 256), 256, 0, s>>>(nr, w.xh, w.xl, z);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "float-float spmm launch");
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  return WPCD_OK;
}

// Born terms b = O P0 Vt e0 for a batch (r0: device on-shell indices)
wpcd_status df_born(const wpcd_problem *pr, const wpcd_P *P, const int *r0, int B, double *b, DfWork &w,
                    cudaStream_t s) {
  const int64_t nc = (int64_t)pr->n_ch * pr->N * pr->M * B;
  df_born_vt_kernel<<<grid_for(nc, 256), 256, 0, s>>>(nc, B, pr->N, pr->M, pr->d.Vt_h, pr->d.Vt_l, r0,
                                                     reinterpret_cast<float2 *>(w.yh),
                                                     reinterpret_cast<float2 *>(w.yl));
  count_launches(1);
  wpcd_status st = spmm_df(pr, P, w.yh, w.yl, w.xh, w.xl, B, s);
  if (st != WPCD_OK) return st;
  st = gemm_df<false>(pr, true, w.xh, w.xl, b, nullptr, nullptr, 2LL * pr->M * B, s);
  if (st != WPCD_OK) return st;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "float-float born launch");
}

}  // namespace wpcd

using namespace wpcd;

extern "C" {

wpcd_status wpcd_split_f64(const double *x, int64_t n, float *hi, float *lo, void *stream) {
  clear_error();
  if (!x || !hi || !lo || n < 0) return set_error(WPCD_EINVAL, "bad split arguments");
  if (n == 0) return WPCD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  df_split_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, x, hi, lo);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "split");
}

}  // extern "C"
