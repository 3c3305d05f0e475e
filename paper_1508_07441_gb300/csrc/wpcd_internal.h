// Internal declarations of the WPCD library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "wpcd.h"

namespace wpcd {

constexpr int kMaxCh = 8;
// Krylov steps per FP32 inner cycle of the mixed solve when the caller
// leaves it open.  A cycle's gain is bounded by the FP32 arithmetic (about
// 5e-6 in residual per cycle on the 200 x 200, 3-channel workload) and ten
// steps already reach that bound: measured there at 128 energies, 8 steps
// need 3 cycles, 10-32 steps 2 cycles, so 10 gives the fewest K
// applications (20 against 32 at 16 steps).
constexpr int kDefaultInner = 10;
constexpr int kMaxPairs = kMaxCh * kMaxCh;

// (l, l') channel pairs with l + l' even, ordered by l then l' (compile-time
// versions, so that unrolled loops index register arrays statically)
__host__ __device__ constexpr int pair_count(int nch) {
  int n = 0;
  for (int l = 0; l < nch; ++l)
    for (int lp = 0; lp < nch; ++lp)
      if (((l + lp) & 1) == 0) ++n;
  return n;
}
__host__ __device__ constexpr int pair_first(int nch, int m) {
  int n = 0;
  for (int l = 0; l < nch; ++l)
    for (int lp = 0; lp < nch; ++lp)
      if (((l + lp) & 1) == 0) {
        if (n == m) return l;
        ++n;
      }
  return 0;
}
__host__ __device__ constexpr int pair_second(int nch, int m) {
  int n = 0;
  for (int l = 0; l < nch; ++l)
    for (int lp = 0; lp < nch; ++lp)
      if (((l + lp) & 1) == 0) {
        if (n == m) return lp;
        ++n;
      }
  return 0;
}

// Kernel launch counter (wpcd_launch_count); every launch site bumps it.
void count_launches(int n);

// Status plumbing: every entry point funnels errors through set_error.
wpcd_status set_error(wpcd_status st, const std::string &msg);
wpcd_status cuda_error(cudaError_t e, const char *what);
void clear_error();

#define WPCD_CUDA_TRY(expr)                                  \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return ::wpcd::cuda_error(_e, #expr); \
  } while (0)

// Body of every extern "C" entry point: no C++ exception crosses the ABI
#define WPCD_GUARD_BEGIN try {
#define WPCD_GUARD_END                                                              \
  }                                                                                 \
  catch (const std::bad_alloc &) {                                                  \
    return ::wpcd::set_error(WPCD_ENOMEM, "host allocation failed");                \
  }                                                                                 \
  catch (...) {                                                                     \
    return ::wpcd::set_error(WPCD_EINVAL, "internal error (unexpected exception)"); \
  }

// ---- host mathematics of step 1 (setup.cpp) -------------------------------
void gauss_legendre(int n, double *t, double *w);
// symmetric eigensolver: A (n x n, row-major) -> eigenvalues ascending,
// vectors as rows with the largest-magnitude component positive.
bool sym_eig(int n, std::vector<double> A, std::vector<double> &evals, std::vector<double> &rows);
void pair_nodes(int N, const double *edges, int n_nodes, std::vector<double> &pn, std::vector<double> &pw,
                std::vector<double> &rsB);
void pair_h(int N, const double *edges, int n_ch, const std::vector<std::vector<double>> &v,
            std::vector<std::vector<double>> &h);
// the potential matrices v_l of every channel on the device (pair.cu), read
// back to the host; synchronous
wpcd_status pair_matrices_gpu(int device, int N, const double *edges, int n_nodes, int n_ch, int n_terms,
                              const double *V, const double *a, std::vector<std::vector<double>> &v);
void pair_eig(int N, const std::vector<double> &h, std::vector<double> &eps, std::vector<double> &O);
inline double shell_volume(double lo, double hi) {
  // int_lo^hi p^2 dp, written to avoid cancellation for narrow bins
  return (hi - lo) * (hi * hi + hi * lo + lo * lo) / 3.0;
}

// ---- handles -----------------------------------------------------------------
struct DeviceTables {
  double *pe2 = nullptr, *qe2 = nullptr;        // squared edges [N+1], [M+1]
  double *pn = nullptr, *wp = nullptr;          // p nodes / weights*p^2 [N*n_p]
  double *qn = nullptr, *wq = nullptr;          // q nodes / weights*q^2 [M*n_q]
  double *yn = nullptr, *wy = nullptr;          // y nodes / weights [n_x]
  double *rsb = nullptr;                        // 1/sqrt(B_i Bq_j) per cell [N*M]
  double *qe = nullptr;                         // q edges [M+1]
  double *eps = nullptr;                        // [n_ch][N]
  double *O = nullptr, *Vt = nullptr;           // [n_ch][N][N]
  float *O32 = nullptr, *Vt32 = nullptr;        // FP32 copies for the inner solve
  float *O_tc = nullptr, *Vt_tc = nullptr;      // TF32 hi/lo operand blocks (tc_gemm.cu)
  float *O_h = nullptr, *O_l = nullptr;         // float-float split of O (df.cu)
  float *Vt_h = nullptr, *Vt_l = nullptr;       // float-float split of Vt
  uint16_t *O_oz = nullptr, *Vt_oz = nullptr;   // bf16 digit planes (oz_gemm.cu)
  int *O_ozE = nullptr, *Vt_ozE = nullptr;      // their row exponents
  int *tc_err = nullptr;                        // tensor-core wait-limit flag
};

}  // namespace wpcd

// The packet lattice (Sec. 2.4 Eq. xij) and its quadrature tables: what P0
// depends on.  Reference-counted: problems built on it and P0 matrices
// assembled on it keep it alive after wpcd_grid_destroy.
struct wpcd_grid {
  int device = 0;
  int N = 0, M = 0, n_p = 0, n_q = 0, n_x = 0;
  std::vector<double> pe, qe;                   // host edges
  double *pe2 = nullptr, *qe2 = nullptr;        // squared edges [N+1], [M+1]
  double *pn = nullptr, *wp = nullptr;          // p nodes / weights*p^2 [N*n_p]
  double *qn = nullptr, *wq = nullptr;          // q nodes / weights*q^2 [M*n_q]
  double *yn = nullptr, *wy = nullptr;          // y nodes / weights [n_x]
  double *rsb = nullptr;                        // 1/sqrt(B_i Bq_j) per cell [N*M]
  double *qe_d = nullptr;                       // q edges [M+1]
  bool y_ascending = false;                     // the y nodes strictly increase
  std::atomic<int> refs{1};
};

struct wpcd_problem {
  wpcd_grid *grid = nullptr;  // the lattice (one reference held)
  int device = 0;
  int N = 0, M = 0, n_p = 0, n_q = 0, n_x = 0, n_ch = 0, n_pairs = 0;
  int pair_l[wpcd::kMaxPairs], pair_lp[wpcd::kMaxPairs];
  std::vector<double> pe, qe;                   // host edges
  std::vector<double> eps, O, v, Vt;            // host [n_ch][N](*N)
  double eps_b = 0.0;
  wpcd::DeviceTables d;
};

// SpMM launch shape chosen by the autotuner: rows per warp, energy lanes per
// row, energies per lane (RHS tile = el * ept); tile > 0: the row-tiled FP32
// SpMM (spmm_tile.cu) with tiles of `tile` cells and ept energies per lane
struct SpmmConfig {
  int rpw = 1, el = 1, ept = 1, tile = 0;
};

namespace wpcd {
// Key of an autotuner choice: the problem shape, the batch B and the
// arithmetic mode (0 FP64 vectors, 1 FP32, 2 float-float), so that one cache
// file can serve several problems
inline int64_t spmm_tune_key(int n_ch, int N, int M, int B, int mode) {
  return ((((int64_t)n_ch * 4096 + N) * 4096 + M) * 4096 + B) * 4 + mode;
}
}  // namespace wpcd

struct wpcd_P {
  wpcd_grid *grid = nullptr;  // the lattice P0 was assembled on (one reference held)
  int device = 0, n_ch = 0;
  int prec = WPCD_FP64;
  int n_pairs = 0;
  int64_t nnz = 0;
  int64_t *row_ptr = nullptr;   // device [N*M+1]
  int32_t *col = nullptr;       // device [nnz]
  double *val64 = nullptr;      // device [n_pairs][nnz] (FP64 assembly)
  float *val32 = nullptr;       // device [n_pairs][nnz] (FP32C assembly)
  float ms = 0.f;
  float ms_phase[3] = {0.f, 0.f, 0.f};  // count, scan, fill
  int64_t work = 0;                     // quadrature points evaluated by the assembly
  float *val32_copy = nullptr;          // FP32 values made from FP64 ones (mixed solve)
  float *val_h = nullptr, *val_l = nullptr;  // float-float split of FP64 values (df.cu)
  int64_t *tile_ptr[2] = {nullptr, nullptr};  // row tiles of 2 / 4 cells (spmm_tile.cu): offsets,
  int32_t *tile_col[2] = {nullptr, nullptr};  // merged columns,
  float *tile_val[2] = {nullptr, nullptr};    // per-column value blocks (FP32)
  int64_t tile_n[2] = {0, 0};
  std::map<int64_t, SpmmConfig> tuned;  // autotuner choices keyed by (B, precision)
};

namespace wpcd {
// a P0 serves every problem on its lattice with its channel count (P0
// depends on neither the potential nor the energy, Sec. 3.3)
inline bool P_fits(const wpcd_P *P, const wpcd_problem *pr) { return P->grid == pr->grid && P->n_ch == pr->n_ch; }
// capi.cpp: grid references
void grid_retain(wpcd_grid *g);
void grid_release(wpcd_grid *g);
// assemble.cu
wpcd_status assemble(wpcd_grid *g, int n_ch, int prec, cudaStream_t s, wpcd_P **out);
// assemble_vl.cu: P0 with variable limits (FP64 values)
wpcd_status assemble_vl(wpcd_grid *g, int n_ch, cudaStream_t s, wpcd_P **out);
// solve.cu
wpcd_status resolvent(const wpcd_problem *pr, const double *E, int n_E, double *g, int *j0,
                      double *D, cudaStream_t s);
wpcd_status onshell(const wpcd_problem *pr, double E, int *j0, double *Elo, double *Ehi, double *q0);
wpcd_status kapply(const wpcd_problem *pr, const wpcd_P *P, const double *g, const double *x,
                   double *y, cudaStream_t s);
wpcd_status solve(wpcd_problem *pr, const wpcd_P *P, const double *E, int n_E,
                  const wpcd_solve_opts *o, double *U00, wpcd_solve_stats *st, cudaStream_t s);
wpcd_status tune_spmm(const wpcd_problem *pr, wpcd_P *P, int B, int mode, cudaStream_t s,
                      SpmmConfig *out);
wpcd_status kapply_scratch(const wpcd_problem *pr, const wpcd_P *P, const double *g, const double *x,
                           double *y, double *scratch_y, double *scratch_z, cudaStream_t s);
wpcd_status born_vectors(wpcd_problem *pr, const wpcd_P *P, const double *E, int n_E, double *b_major,
                         cudaStream_t s);
wpcd_status spmm_apply(wpcd_problem *pr, wpcd_P *P, int mode, const void *y, void *z, int n_rhs, float *ms,
                       cudaStream_t s);
wpcd_status channel_gemm(wpcd_problem *pr, int which, int mode, const void *g, const void *x, void *y, int n_rhs,
                         float *ms, cudaStream_t s);
// G1 of n_E energies in the batched layout (element (r, e) at r * n_E + e)
wpcd_status resolvent_minor(const wpcd_problem *pr, const double *E, int n_E, double *g, cudaStream_t s);
// tc_gemm.cu: tensor-core (TF32 x 3) channel-block products for FP32 vectors
bool tc_supported(const wpcd_problem *pr);
bool tc_enabled();
wpcd_status tc_prepare(wpcd_problem *pr, cudaStream_t s);
// spmv.cu: one-right-hand-side SpMV in the vectors' precision (FP32 values
// and vectors, or FP64 both): cfg.rpw rows per warp, cfg.ept chunks of four
// nonzeros per lane and step
wpcd_status launch_spmv1(const wpcd_problem *pr, const wpcd_P *P, bool fp64, const void *val, const void *y, void *z,
                         const SpmmConfig &cfg, cudaStream_t s);
// spmm_tile.cu: the row-tiled FP32 SpMM (tiles of 2 or 4 cells; the tile
// structure built on first use, which synchronises the stream)
bool tile_supported(const wpcd_problem *pr, int B);
wpcd_status tile_prepare(const wpcd_problem *pr, wpcd_P *P, const float *v32, int tile, cudaStream_t s);
wpcd_status launch_spmm_tile(const wpcd_problem *pr, wpcd_P *P, const float *v32, const float *y, float *z, int B,
                             const SpmmConfig &cfg, cudaStream_t s);
// one problem of a grouped tensor-core product: its vectors are the segment
// at float offset off of the group vectors, [n_ch][N][ncol] floats
struct TcGroupProb {
  const wpcd_problem *pr;
  int64_t off, ncol;
};
wpcd_status tc_gemm_group(const TcGroupProb *gp, int n_prob, bool use_O, const float *G, const float *X,
                          const float *S, float *C, cudaStream_t s);
wpcd_status tc_gemm(const wpcd_problem *pr, bool use_O, const float *G, const float *X, const float *S, float *C,
                    int64_t ncol, cudaStream_t s);
wpcd_status tc_check(const wpcd_problem *pr, cudaStream_t s);
wpcd_status tc_clear(const wpcd_problem *pr, cudaStream_t s);
// test knobs of the abort path: the role of the warp-specialised GEMM (0
// producer, 1 MMA issuer, 2 converters, 3 epilogue; -1 none) whose first
// wait runs out at once, and whether the digit-plane GEMM's first copy wait
// does
extern std::atomic<int> g_ws_expire_role;
extern std::atomic<int> g_oz_expire_first;
// oz_gemm.cu: FP64-class channel-block products from bf16 digit planes on
// the tensor cores (float-float panel in, FP64 or float-float out), N <= 256
bool oz_supported(const wpcd_problem *pr);
bool oz_enabled();
wpcd_status oz_prepare(wpcd_problem *pr, cudaStream_t s);
wpcd_status oz_gemm(const wpcd_problem *pr, bool use_O, const float *Bh, const float *Bl, double *C, float *Ch,
                    float *Cl, int64_t ncol, cudaStream_t s);
// df.cu: float-float ("FP64-class", about 48 significant bits) K application
// on the FP32 pipe, for the refinement residual of the mixed solve
// Work space of the solves: a stream-ordered pool per device that keeps
// freed memory for the next solve (allocation from it takes microseconds
// instead of a cudaMalloc's page mapping, and a free does not synchronise
// the device).  The pool lives as long as the process.
cudaError_t pool_malloc(void **p, size_t bytes, cudaStream_t s);
void pool_free(void *p, cudaStream_t s);
template <typename T>
cudaError_t pool_malloc(T **p, size_t bytes, cudaStream_t s) {
  return pool_malloc(reinterpret_cast<void **>(p), bytes, s);
}
// Persistent device memory (problem tables, P0, packed operands, the MLP):
// cudaMalloc / cudaFree, or the caller's allocator (wpcd_set_allocator)
cudaError_t dev_malloc(void **p, size_t bytes);
void dev_free(void *p);
template <typename T>
cudaError_t dev_malloc(T **p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void **>(p), bytes);
}

struct DfWork {
  float *xh = nullptr, *xl = nullptr, *yh = nullptr, *yl = nullptr;  // [2 dim B] each
  cudaStream_t st = nullptr;                                         // stream of the pool frees
  ~DfWork();
  cudaError_t alloc(size_t dim, int B, cudaStream_t s);
};
// the float-float splits of O, Vt (and P's values), and with digits the bf16
// digit planes of O and Vt for the tensor-core products (N <= 256)
wpcd_status df_prepare(wpcd_problem *pr, wpcd_P *P, cudaStream_t s, bool digits = true);
wpcd_status df_kapply(const wpcd_problem *pr, const wpcd_P *P, const double *g, const double *x, double *out, int B,
                      DfWork &w, cudaStream_t s);
wpcd_status launch_spmm_df_cfg(const wpcd_problem *pr, const wpcd_P *P, const float *yh, const float *yl,
                               float *zh, float *zl, int B, const SpmmConfig &cfg, cudaStream_t s);
// digits: the digit-plane tensor-core product (oz_gemm.cu) instead of the
// float-float SIMT kernel
wpcd_status df_gemm_op(wpcd_problem *pr, bool use_O, bool digits, const double *g, const double *x, double *y, int B,
                       float *ms, cudaStream_t s);
wpcd_status df_spmm_op(wpcd_problem *pr, wpcd_P *P, const double *y, double *z, int B, float *ms, cudaStream_t s);
wpcd_status df_born(const wpcd_problem *pr, const wpcd_P *P, const int *r0, int B, double *b, DfWork &w,
                    cudaStream_t s);
// group.cu
wpcd_status solve_group(int n_prob, wpcd_problem *const *prs, const wpcd_P *const *Ps, const double *const *E,
                        const int *n_E, const wpcd_solve_opts *o, double *const *U00, wpcd_solve_stats *const *st,
                        cudaStream_t s);
}  // namespace wpcd
