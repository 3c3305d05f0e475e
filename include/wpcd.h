/*
 * wpcd.h -- C ABI of the GB300 (sm_103a) library for the hot path of the
 * wave-packet continuum-discretisation (WPCD) Faddeev method of
 * Pomerantsev, Kukulin, Rubtsova and Sakhiev, "Fast GPU-based calculations
 * in few-body quantum scattering" (arXiv:1508.07441).
 *
 * The calls follow the paper's statement of the problem (Sec. 3.3, the four
 * steps of the numerical scheme): build the packet grids and the pair
 * quantities (step 1), assemble the lattice permutation matrix P0 (step 2),
 * build the channel resolvent G1 (step 3) and solve the matrix Faddeev
 * equation by iterating K = O P0 Vt G1 and summing the iterates (step 4).
 *
 * System: three identical spinless bosons, hbar = m = 1, pair potential
 * V(r) = sum_k V_k exp(-r^2 / a_k), total orbital momentum L = 0, channels
 * alpha = (l, lambda = l) for l = 0 .. n_ch-1.  Momenta are Jacobi momenta p
 * (pair) and q (spectator); the free energy is p^2 + 3 q^2 / 4.
 *
 * Conventions used by every call:
 *   - cell index c = i*M + j for p-bin i in [0, N) and q-bin j in [0, M);
 *   - channel-basis vector index r = ch*N*M + k*M + j (k: pair eigenstate,
 *     ascending energy, k = 0 the dimer); complex vectors are interleaved
 *     (re, im) doubles (or floats where stated);
 *   - (l, l') channel pairs with l + l' even, ordered by l then l'
 *     (n_pairs of them: 1, 5, 13 for n_ch = 1, 3, 5);
 *   - P0 is block-CSR over cells: row_ptr[N*M + 1] (int64), col[nnz]
 *     (int32, ascending within a row), val[n_pairs][nnz] (pair-major), one
 *     value per (l, l') pair of each nonzero cell pair.
 *
 * Ownership: the library allocates and owns everything behind a handle
 * (device memory via cudaMalloc on the problem's device) until the matching
 * *_destroy.  The solves take their work space from a stream-ordered memory
 * pool per device, owned by the library: freed blocks stay in the pool for
 * the next solve (no cudaFree, no device synchronisation) until the process
 * exits.  Caller arrays are never retained.  Pointers documented as
 * "device" must be device (or managed) memory on the problem's device;
 * "host" pointers are ordinary host memory.  `stream` is a cudaStream_t
 * (NULL: the legacy default stream); calls that return results to host
 * memory synchronise that stream before returning.
 *
 * Errors: every call returns a wpcd_status (0 on success, < 0 on failure) and
 * leaves a message for wpcd_last_error() (thread-local).  No call aborts or
 * lets a C++ exception escape.  Invalid sizes, non-monotone edges, NaN
 * inputs, energies without an open elastic channel and out-of-range
 * channels are rejected with WPCD_EINVAL / WPCD_ENOBOUND before any launch.
 */
#ifndef WPCD_H
#define WPCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int wpcd_status;

#define WPCD_OK 0
#define WPCD_EINVAL -1      /* invalid argument */
#define WPCD_ENOMEM -2      /* allocation failed */
#define WPCD_ECUDA -3       /* CUDA runtime error (message has the detail) */
#define WPCD_ENOCONV -4     /* summation did not reach the tolerance */
#define WPCD_EBREAKDOWN -5  /* zero divisor in the Pade table / Krylov basis */
#define WPCD_ETIMEOUT -6    /* a device-side wait ran out of its budget */
#define WPCD_ENOBOUND -7    /* no bound pair state / energy below threshold */

/* arithmetic of the assembled values and of the solve */
#define WPCD_FP64 0   /* all node values and sums in FP64 */
#define WPCD_FP32C 1  /* FP64 binning, FP32 node values, compensated sums */
#define WPCD_FP64_VL 2 /* assembly only: FP64 with variable limits instead of
                          node binning (the y-interval of every (p, q) node and
                          target cell from the theta limits of Eq. perm,
                          integrated by the n_x-point GL rule; Sec. 3.2) */

/* summation of the iterates */
#define WPCD_SUM_KRYLOV 0 /* vector form: minimal-residual extrapolation of
                             the iterates through an orthonormal basis */
#define WPCD_SUM_WYNN 1   /* scalar Pade approximants of sum_n c_n by
                             Wynn's epsilon algorithm (the paper's route) */

/* Thread-local text of the last error on this thread ("" if none). */
const char *wpcd_last_error(void);

/* ABI version (major * 10000 + minor * 100 + patch). */
int wpcd_version(void);

/* Caller-supplied device allocator.  alloc returns `bytes` of device memory
 * on device `device`, to be used on `stream` (a cudaStream_t; NULL: the
 * legacy default stream), or NULL on failure (the call then returns
 * WPCD_ECUDA); free releases such a block, ordered after the work already
 * queued on `stream` (persistent tables are freed with stream NULL after a
 * device synchronisation).  `user` is passed through.  The callbacks may be
 * called from any library call that allocates (problem creation, assembly,
 * the solves' work space, the MLP). */
typedef void *(*wpcd_alloc_fn)(size_t bytes, int device, void *stream, void *user);
typedef void (*wpcd_free_fn)(void *ptr, void *stream, void *user);

/* Route every device allocation of the library through (alloc, free), or
 * back to the library's own (cudaMalloc for tables, a stream-ordered pool
 * for work space) with both NULL.  Process-wide; EINVAL if only one is NULL
 * or while allocations of the other allocator are live (set it before
 * creating handles, or after destroying them all). */
wpcd_status wpcd_set_allocator(wpcd_alloc_fn alloc, wpcd_free_fn free_fn, void *user);

/* Number of CUDA kernel launches this library has issued in this process
 * (all devices, all threads); lets a caller count the device work of a
 * region by differencing. */
int64_t wpcd_launch_count(void);

/* Test knob of the wait-limit path of the tensor-core GEMMs, on valid input
 * and without a fault.  kernel 1: the warp-specialised TF32x3 GEMM of the
 * FP32 inner cycles, role 0 producer, 1 MMA issuer, 2 converters, 3
 * epilogue; kernel 2: the digit-plane GEMM of the refinement residual, role
 * 0 (the first operand-copy wait).  Until the knob is cleared (kernel 0),
 * every launch of that kernel gives the first wait of that role a limit of
 * zero spins: the wait runs out, the CTA aborts, every copy and MMA already
 * issued is still waited for (with the full limit) before the tensor memory
 * is freed, and the operation returns WPCD_ETIMEOUT.  Process-wide, for tests
 * only; EINVAL for another kernel or role. */
wpcd_status wpcd_debug_expire_first_wait(int kernel, int role);

/* Step 1, packet grid (Sec. 2.2 Eq. ip, Sec. 2.4 Eq. xij): n_bins + 1 edges
 * of the tangent map k_n = s tan(pi n / (2 (n_bins + 1))), s chosen so that
 * the last edge is k_max; edges[0] = 0.  edges: host, n_bins + 1 doubles.
 * EINVAL if n_bins < 1 or k_max is not positive and finite. */
wpcd_status wpcd_tangent_edges(int n_bins, double k_max, double *edges);

/* Description of one three-body problem (all pointers host, read during
 * wpcd_problem_create only). */
typedef struct {
  int N, M;               /* number of p-bins and q-bins */
  const double *p_edges;  /* N + 1 strictly increasing, p_edges[0] = 0 */
  const double *q_edges;  /* M + 1 strictly increasing, q_edges[0] = 0 */
  int n_p, n_q, n_x;      /* GL nodes per p-bin, per q-bin, and in y on [-1, 1] */
  int n_ch;               /* channels l = 0 .. n_ch - 1 (1 <= n_ch <= 5) */
  int n_terms;            /* Gaussian terms of V(r) */
  const double *V;        /* strengths V_k */
  const double *a;        /* ranges a_k > 0 (V_k exp(-r^2 / a_k)) */
  int n_pair_nodes;       /* GL nodes per bin for the pair double integrals */
  int device;             /* CUDA device ordinal */
} wpcd_problem_desc;

typedef struct wpcd_problem wpcd_problem;
typedef struct wpcd_P wpcd_P;
typedef struct wpcd_grid wpcd_grid;

/* The packet lattice alone (all pointers host, read during
 * wpcd_grid_create only). */
typedef struct {
  int N, M;               /* number of p-bins and q-bins */
  const double *p_edges;  /* N + 1 strictly increasing, p_edges[0] = 0 */
  const double *q_edges;  /* M + 1 strictly increasing, q_edges[0] = 0 */
  int n_p, n_q, n_x;      /* GL nodes per p-bin, per q-bin, and in y on [-1, 1] */
  int device;             /* CUDA device ordinal */
} wpcd_grid_desc;

/* The pair interaction on a grid (pointers host, read during
 * wpcd_pair_create only). */
typedef struct {
  int n_ch;               /* channels l = 0 .. n_ch - 1 (1 <= n_ch <= 5) */
  int n_terms;            /* Gaussian terms of V(r) */
  const double *V;        /* strengths V_k */
  const double *a;        /* ranges a_k > 0 (V_k exp(-r^2 / a_k)) */
  int n_pair_nodes;       /* GL nodes per bin for the pair double integrals */
} wpcd_pair_desc;

/* Step 1, the lattice (Sec. 2.2 Eq. ip, Sec. 2.4 Eq. xij): the p and q
 * packet bins with their GL node and weight tables, squared edges and cell
 * norms, uploaded to the device.  This is all that P0 depends on: P0 is
 * computed once per lattice and serves every potential and every energy
 * (Sec. 3.3).  EINVAL for sizes or edges as in wpcd_problem_create. */
wpcd_status wpcd_grid_create(const wpcd_grid_desc *desc, wpcd_grid **out);
/* Releases the caller's reference: problems and P0 matrices made on the grid
 * keep it alive until they are destroyed. */
void wpcd_grid_destroy(wpcd_grid *g);

/* Step 1, the pair part (Sec. 3.3 "processing of the input data"; Sec. 2.2
 * Eq. vpot and Eq. exp_z) on a grid: potential matrices v_l on the grid's p
 * bins, diagonalisation of h1 in every channel (O, eps), Vt = v O^T.  The
 * result is a problem (grid + pair) usable with every call that takes one;
 * it holds a reference to the grid.  ENOBOUND if channel 0 has no bound pair
 * state. */
wpcd_status wpcd_pair_create(wpcd_grid *g, const wpcd_pair_desc *desc, wpcd_problem **out);

/* The grid of a problem (a new reference: release it with wpcd_grid_destroy). */
wpcd_status wpcd_problem_grid(const wpcd_problem *pr, wpcd_grid **out);

/* Step 1 (Sec. 3.3, "processing of the input data"; Sec. 2.2 Eq. vpot and
 * Eq. exp_z) in one call: a grid of its own (wpcd_grid_create) and the pair
 * setup on it (wpcd_pair_create): free-packet potential matrices v_l,
 * diagonalisation of h1 = h0 + v in every channel (rotation matrices O,
 * energies eps), Vt = O^T V1 = v O^T, node and edge tables, all uploaded to
 * the device.  Runs on the host in FP64 (the paper calls this step
 * negligible).  ENOBOUND if channel 0 has no bound pair state. */
wpcd_status wpcd_problem_create(const wpcd_problem_desc *desc, wpcd_problem **out);
void wpcd_problem_destroy(wpcd_problem *pr);

/* dim = n_ch*N*M, n_pairs, eps_bound = lowest eigenvalue of channel 0. */
wpcd_status wpcd_problem_info(const wpcd_problem *pr, int *dim, int *n_pairs, double *eps_bound);

/* Host copies of channel l's eps[N], O[N][N] (row k = eigenvector k in the
 * free-packet basis, largest component positive) and v[N][N]; any output
 * may be NULL. */
wpcd_status wpcd_problem_pair(const wpcd_problem *pr, int l, double *eps, double *O, double *v);

/* Step 2 (Sec. 3.2 Eqs. perm_z, perm, gal; Sec. 4.2 pre-selection and
 * nonzero elements): assemble P0 on the device by quadrature-node binning.
 * Every source cell's (p, q, y) GL nodes are mapped through the recoupled
 * momenta p' = -(p/2 + 3q/4), q' = p - q/2, binned against the squared
 * edges in FP64 (bin k holds [e_k^2, e_{k+1}^2), the last bin also e_N^2;
 * larger values leave the grid), and summed per target cell:
 *   P0[(l,c),(l',c')] = sqrt((2l+1)(2l'+1)) / sqrt(B_i Bq_j B_i' Bq_j')
 *                       * sum_nodes w p^2 q^2 P_l(y) P_l'(y') [node -> c'].
 * prec = WPCD_FP64 or WPCD_FP32C.  Two passes (count, then fill) with no
 * atomics: the result is bit-reproducible for a given device.
 * prec = WPCD_FP64_VL assembles the same elements with variable limits (the
 * paper's "double integral with variable limits", Sec. 3.2): for every GL
 * node (p, q) of the source cell and every target cell, the y-interval on
 * which p' and q' lie in the target's bins (p'^2, q'^2 are linear in y, so
 * the limits are (e^2 - Bp) / A for the edges e) is integrated with the
 * n_x-point GL rule mapped onto it; the theta functions are then exact in y.
 * FP64 values (the P0 reports WPCD_FP64), one thread per nonzero element,
 * bit-reproducible; EINVAL if a row (source cell) has more than
 * 3 (N + M) target cells (rounded up to 3/4 of a power of two, 6144 at
 * most).
 * Runs on `stream` and returns when the assembly has completed (the stream
 * is synchronised twice: for the nonzero count, and at the end).  The P0
 * belongs to the problem's grid and channel count (see wpcd_assemble_P_grid):
 * every problem on that grid with that many channels can use it. */
wpcd_status wpcd_assemble_P(wpcd_problem *pr, int prec, void *stream, wpcd_P **out);

/* Step 2 on a grid alone: P0 for channels l = 0 .. n_ch - 1 (1 <= n_ch <= 5)
 * as in wpcd_assemble_P.  P0 depends on the lattice only, not on the
 * potential or the energy (Sec. 3.3: computed once, then used for many
 * energies); the calls that take (problem, P) accept it for every problem
 * made on this grid (wpcd_pair_create) with n_ch channels, EINVAL for
 * another grid or channel count.  The P0 holds a reference to the grid. */
wpcd_status wpcd_assemble_P_grid(wpcd_grid *g, int n_ch, int prec, void *stream, wpcd_P **out);
void wpcd_P_destroy(wpcd_P *P);

/* nnz (cell pairs), n_pairs, prec, and the timing of the last assembly in
 * milliseconds (count pass + scan + fill; CUDA events); any may be NULL. */
wpcd_status wpcd_P_info(const wpcd_P *P, int64_t *nnz, int *n_pairs, int *prec, float *ms);

/* Device time of each assembly phase of P, in milliseconds, from CUDA events
 * recorded on the assembly stream: ms[0] count pass (map, bin, sort, count),
 * ms[1] scan, ms[2] fill pass (values and segmented reduction). */
wpcd_status wpcd_P_timing(const wpcd_P *P, float ms[3]);

/* Quadrature points the assembly of P evaluated: N M n_p n_q n_x for node
 * binning (every node mapped once), the (node, target) y-intervals times n_x
 * for WPCD_FP64_VL. */
wpcd_status wpcd_P_work(const wpcd_P *P, int64_t *points);

/* Copy P0 out: row_ptr[N*M + 1], col[nnz], val[n_pairs][nnz] as FP64 (FP32C
 * values are widened).  Destinations may be host or device memory; any may
 * be NULL.  Synchronises `stream`. */
wpcd_status wpcd_P_export(const wpcd_P *P, int64_t *row_ptr, int32_t *col, double *val,
                          void *stream);

/* Step 3 (Sec. 2.1 Eq. g_tot, Sec. 2.3 energy averaging, Sec. 2.4): the
 * channel resolvent G1 at n_E energies, each averaged over its on-shell
 * bin [E_lo, E_hi] = eps_b + 3/4 [q_j0^2, q_j0+1^2]:
 *   g_kj = [Phi_j(E_hi - eps_k) - Phi_j(E_lo - eps_k)] / (D Bq_j)
 *          - i pi / (D Bq_j) int_{bin j} q^2 dq theta(E_lo < eps_k + 3q^2/4 < E_hi),
 *   Phi_j(a) = int_{bin j} q^2 ln|a - 3q^2/4| dq,  D = E_hi - E_lo.
 * E: host [n_E].  g: device [n_E][dim] interleaved complex FP64.
 * j0, D: host [n_E] (may be NULL).  ENOBOUND if some E <= eps_b; EINVAL if
 * its on-shell momentum lies beyond the q grid. */
wpcd_status wpcd_resolvent(const wpcd_problem *pr, const double *E, int n_E, double *g, int *j0,
                           double *D, void *stream);

/* One application of the Faddeev kernel (Sec. 3.3 Eq. kernel):
 * y = O P0 Vt (g o x), FP64.  g: device [dim] complex or NULL (G1 = 1).
 * x, y: device [dim] complex, distinct. */
wpcd_status wpcd_kapply(const wpcd_problem *pr, const wpcd_P *P, const double *g, const double *x,
                        double *y, void *stream);

/* precision of the solve */
#define WPCD_SOLVE_FP64 0  /* plain FP64 iteration (the comparison baseline) */
#define WPCD_SOLVE_MIXED 1 /* FP32 inner Krylov cycles (FP32 P0 values,
                              tensor-core TF32x3 block products, compensated
                              FP32 SpMM sums) inside an iterative-refinement
                              loop whose Born term and residual
                              b - (I - K) u are formed in float-float
                              arithmetic on the FP32 pipe (FP64-class, about
                              48 significant bits; the single-problem solve) */
#define WPCD_SOLVE_MIXED_FP64 2 /* the same with the Born term and residual
                              in native FP64 */

typedef struct {
  int method;      /* WPCD_SUM_KRYLOV or WPCD_SUM_WYNN (Wynn: FP64, one energy at a time) */
  int max_iter;    /* FP64 Krylov / Wynn: cap on K applications (<= 512) */
  int min_iter;    /* Wynn: minimum number of terms before stopping */
  double tol;      /* Krylov, mixed: relative residual; Wynn: relative change */
  int check_every; /* FP64 Krylov: read the residual estimates back every n
                      steps (1 gives exact per-energy step counts) */
  int precision;   /* WPCD_SOLVE_FP64, WPCD_SOLVE_MIXED (float-float residual
                      and Born term) or WPCD_SOLVE_MIXED_FP64 (native FP64
                      residual), in wpcd_solve and wpcd_solve_batch alike */
  int batch;       /* energies solved together in one batched iteration
                      (block K applications, SpMM over the batch); 0: all */
  int inner_iter;  /* mixed: Krylov steps of the first refinement cycle and the
                      most of any later one (0: 10); a later cycle takes the
                      steps that the previous cycle's per-step reduction of the
                      worst residual says reach a tenth of tol, at least 2 */
  int max_outer;   /* mixed: cap on refinement cycles (0: 12) */
  int use_graph;   /* mixed: replay each inner cycle from a CUDA graph (1) or
                      launch its kernels one by one (0) */
  const double *u_init; /* device [n_E][dim] complex warm start, or NULL (0) */
  double *u_out;   /* device [n_E][dim] complex solutions u = (I - K)^-1 u0,
                      or NULL */
} wpcd_solve_opts;

typedef struct {
  int status;        /* per-energy status */
  int n_kapply;      /* K applications used */
  int j0;            /* on-shell q-bin */
  double D;          /* on-shell energy width */
  double relres;     /* Krylov: final relative residual estimate */
  double U00[2];     /* on-shell element <Z_{0,0,j0}|U|Z_{0,0,j0}> */
  double S[2];       /* S = 1 - 2 pi i U00 / D */
  double A[2];       /* paper's amplitude (2/(3 q0)) U00 / (q_j0+1 - q_j0) */
  float ms;          /* device time of the batch holding this energy
                        (CUDA events), divided by the batch size */
  int n_kapply32;    /* mixed: FP32 K applications (n_kapply counts FP64 ones) */
  int n_outer;       /* mixed: refinement cycles */
  int warm_fallback; /* FP64 Krylov: 1 if this energy's warm start was not
                        better than the zero start and was replaced by it */
} wpcd_solve_stats;

/* Step 4 (Sec. 3.3: iterations of the matrix equation and Pade
 * summation): for every energy, the on-shell element U00 of
 * U = P V1 + P V1 G1 U, from the iterates of K = O P0 Vt G1 started at the
 * Born term u0 = O P0 Vt e0 (column e0 of U solves u = u0 + K u).
 * Energies are processed in batches of opts->batch: one batched iteration
 * applies K to all of them at once (the energy index innermost in device
 * memory, so P0 is read once per batch), each energy keeping its own G1 and
 * its own Krylov basis.  WPCD_SOLVE_FP64 runs the plain FP64 iteration;
 * WPCD_SOLVE_MIXED runs FP32 inner cycles under an FP64 refinement loop and
 * reaches the same FP64 tolerance.  E: host [n_E]; U00: host [n_E] complex
 * (interleaved); stats: host [n_E] or NULL.  Returns the worst per-energy
 * status (ENOCONV / EBREAKDOWN still deliver the best estimate). */
wpcd_status wpcd_solve(wpcd_problem *pr, const wpcd_P *P, const double *E, int n_E,
                       const wpcd_solve_opts *opts, double *U00, wpcd_solve_stats *stats,
                       void *stream);

/* Largest number of problems in one grouped solve, and of energies per
 * problem there. */
#define WPCD_GROUP_MAX 64
#define WPCD_GROUP_MAX_E 32

/* Batching across grids (Sec. 3.3 iterations of the matrix equation, the
 * same summation as wpcd_solve with WPCD_SUM_KRYLOV): n_prob problems whose
 * packet grids differ in size, each with its own energies, solved together.
 * Every operation of the iteration is ONE launch over all problems: the
 * Vt / O block products walk one tile list over (problem, channel, tile),
 * the P0 SpMM walks the concatenated rows of all P0 matrices, and the
 * Krylov vector kernels work on the concatenated per-problem batches (the
 * wpcd_solve layout, energy index innermost, one segment per problem).
 * Each (problem, energy) system keeps its own G1 and Krylov basis; with
 * WPCD_SOLVE_MIXED the FP32 inner cycle of all problems is one CUDA graph
 * and the refinement residual is one float-float launch per operation.
 * problems[g], P[g]: problem g and its assembled P0 (all on one device, the
 * same channel count and the same P0 precision); E[g]: host [n_E[g]]
 * energies, 1 <= n_E[g] <= WPCD_GROUP_MAX_E; U00[g]: host [n_E[g]] complex
 * (interleaved) results; stats: NULL, or host array of n_prob pointers each
 * NULL or to [n_E[g]] stats.  opts as for wpcd_solve, with method
 * WPCD_SUM_KRYLOV, batch 0 and no vectors (EINVAL otherwise); 1 <= n_prob
 * <= WPCD_GROUP_MAX.  Work space from the library's pool (returned to it
 * before this call returns).  Returns the worst per-energy status (ENOCONV and
 * EBREAKDOWN still deliver the best estimate). */
wpcd_status wpcd_solve_batch(int n_prob, wpcd_problem *const *problems, const wpcd_P *const *P,
                             const double *const *E, const int *n_E, const wpcd_solve_opts *opts,
                             double *const *U00, wpcd_solve_stats *const *stats, void *stream);

/* arithmetic of wpcd_spmm */
#define WPCD_SPMM_FP64 0 /* FP64 vectors, the P's own value precision */
#define WPCD_SPMM_FP32 1 /* FP32 vectors and values (FP32 values made from FP64
                            ones on first use), blocked compensated sums */
#define WPCD_SPMM_FF 2   /* FP64 vectors in and out, float-float arithmetic on
                            the FP32 pipe (about 48 significant bits), as in
                            the refinement residual of WPCD_SOLVE_MIXED */
#define WPCD_SPMM_FP32_BLOCKED 3 /* as WPCD_SPMM_FP32 with the row-tiled kernel
                            on tiles of 2 x 2 cells (every column of a tile
                            gathered once for its four rows; n_rhs even, at
                            most three channels); the autotuner also weighs
                            the row-tiled shapes for WPCD_SPMM_FP32 */

/* The sparse step of the K application (Sec. 3.3, Eq. kernel; P0 of
 * Eq. perm): z = P0 y for n_rhs vectors in the batched layout (device
 * [n_ch][N][M][n_rhs] complex, energy index innermost, y and z distinct;
 * FP32 for WPCD_SPMM_FP32, FP64 otherwise).  The launch shape is the
 * autotuner's choice for the batch, tuned on first use (which synchronises
 * the stream).  kernel_ms: NULL, or receives the device time of the SpMM
 * kernel alone (CUDA events on the stream; the call then synchronises). */
wpcd_status wpcd_spmm(wpcd_problem *pr, wpcd_P *P, int mode, const void *y, void *z, int n_rhs, float *kernel_ms,
                      void *stream);

/* arithmetic of wpcd_channel_gemm */
#define WPCD_GEMM_FP64 0   /* FP64 vectors, FP64 SIMT kernel */
#define WPCD_GEMM_FP32 1   /* FP32 vectors, FP32 SIMT kernel */
#define WPCD_GEMM_TF32X3 2 /* FP32 vectors, tensor cores (tcgen05): each FP32
                              operand split into TF32 hi + lo, products
                              hi*hi + hi*lo + lo*hi accumulated in FP32 */
#define WPCD_GEMM_FF 3     /* FP64 vectors in and out, float-float arithmetic on
                              the FP32 pipe (about 48 significant bits) */
#define WPCD_GEMM_DIGITS 4 /* FP64 vectors in and out: the FP64 A and the
                              float-float split of (G1 o X) cut into eight
                              7-bit bf16 digit planes over per-row / per-column
                              power-of-two scales; the 36 digit-plane products
                              of weight above 2^-56 on the tensor cores
                              (tcgen05 kind::f16), each diagonal summed exactly
                              in FP32, combined in FP64; N <= 256 */

/* One dense step of the K application (Sec. 3.3, Eq. kernel): for every
 * channel block ch, Y_ch = A_ch (G1 o X)_ch with A = Vt (which = 0) or O
 * (which = 1), N x N, applied to the [N][M][n_rhs] complex block of the
 * channel (energy index innermost, as in wpcd_solve).  g: device resolvent
 * in the same layout and precision as x, or NULL for no scaling; x, y:
 * device [n_ch][N][M][n_rhs] complex, FP32 for WPCD_GEMM_FP32 and
 * WPCD_GEMM_TF32X3, FP64 otherwise, distinct.  The mixed solve runs its FP32
 * inner cycles with WPCD_GEMM_TF32X3 when N <= 512 (the environment
 * variable WPCD_GEMM=simt selects WPCD_GEMM_FP32 instead) and its residual
 * and Born-term products with WPCD_GEMM_DIGITS when N <= 256, else
 * WPCD_GEMM_FF (WPCD_RESIDUAL_GEMM=ff selects WPCD_GEMM_FF always).  kernel_ms: NULL, or receives the device time of the
 * product kernel alone (the call then synchronises).  EINVAL for a bad
 * mode, bad vectors, WPCD_GEMM_TF32X3 with N > 512 or WPCD_GEMM_DIGITS with
 * N > 256; ETIMEOUT if a
 * tensor-core wait ran out. */
wpcd_status wpcd_channel_gemm(wpcd_problem *pr, int which, int mode, const void *g, const void *x, void *y,
                              int n_rhs, float *kernel_ms, void *stream);

/* Autotuner (batching): time the candidate SpMM launch shapes (rows per
 * warp, energy lanes per row, energies per lane = RHS tile width) for a
 * batch of n_rhs energies in the arithmetic of mode (WPCD_SPMM_FP64,
 * WPCD_SPMM_FP32 or WPCD_SPMM_FF) and keep the fastest for later solves
 * (for every P0 of the same shape in the process); returns the choice.
 * For WPCD_SPMM_FP32 with an even batch of at least 16 the candidates
 * include the row-tiled kernel (WPCD_SPMM_FP32_BLOCKED's), reported as
 * rows_per_warp = 2 or 4 (the cells of a tile) with 32 energy lanes, a pair
 * the warp-per-row shapes never use.  For one right-hand side the shapes are
 * those of the one-vector SpMV: rows per warp 2-16, energy lanes 1 and
 * energies per lane = nonzero chunks per step (1 or 2).
 * Solves tune on first use of a (batch, arithmetic) pair.  With
 * WPCD_TUNE_CACHE set to a file path, choices are also read from /
 * appended to that file (text lines "key rows_per_warp energy_lanes
 * energies_per_lane [cells_per_tile]"). */
wpcd_status wpcd_tune_spmm(wpcd_problem *pr, wpcd_P *P, int n_rhs, int mode, void *stream,
                           int *rows_per_warp, int *energy_lanes, int *energies_per_lane);

/* Largest problem dimension n_ch*N*M that wpcd_kapply_noalloc accepts. */
#define WPCD_NOALLOC_MAX_DIM 131072

/* The same K application as wpcd_kapply, for callers that cannot allocate
 * device memory: code running while a stream is captured into a CUDA graph,
 * applications whose device memory belongs to a fixed pool or a foreign
 * allocator, loops that must not touch the allocator once running.  The
 * paper has no counterpart.  It calls no cudaMalloc or cudaFree: its two
 * intermediate vectors live in a 4 MiB array of device memory
 * (WPCD_NOALLOC_MAX_DIM x 2 complex doubles) that every GPU loading the
 * library holds until the process exits.  The caller still passes g (device
 * [dim] complex or NULL), x and y (device [dim] complex, distinct), as for
 * wpcd_kapply.  The first call on a device looks up the array's device
 * address (with that device current); make it before any stream capture.
 * EINVAL if dim exceeds WPCD_NOALLOC_MAX_DIM.  All calls share the array:
 * calls that overlap on the GPU (other streams, other host threads on the
 * same device) race.  The SpMM uses the shape the autotuner chose for one
 * FP64 right-hand side (the one wpcd_kapply tunes on its first call) if P
 * has one, else a fixed shape.  Enqueued on `stream`; does not synchronise. */
wpcd_status wpcd_kapply_noalloc(const wpcd_problem *pr, const wpcd_P *P, const double *g, const double *x,
                                double *y, void *stream);

/* Born terms u0 = O P0 Vt e0 (the first iterate, Eq. kernel with G1
 * removed) for n_E energies: b device [n_E][dim] complex FP64. */
wpcd_status wpcd_born(wpcd_problem *pr, const wpcd_P *P, const double *E, int n_E, double *b, void *stream);

/* ---------------------------------------------------------------------------
 * Learned warm start.  The paper has no learned component: this is a growth
 * line around its iteration, which stays the fallback and decides
 * convergence.  A 3-layer MLP (n_in -> width -> width -> n_out, tanh hidden layers) is
 * trained on the GPU by the library's own FP32 forward, backward and Adam
 * kernels and inferred with BF16 weights (FP32 arithmetic); its outputs are
 * coefficients of the solution in a projected basis Phi built from the
 * method's own solutions.  All arrays named device are device memory.
 * ------------------------------------------------------------------------- */
typedef struct wpcd_mlp wpcd_mlp;

/* Glorot-uniform weights (counter-based splitmix64 stream from `seed`),
 * zero biases, identity input/output affine maps. */
wpcd_status wpcd_mlp_create(int n_in, int width, int n_out, uint64_t seed, int device, wpcd_mlp **out);
void wpcd_mlp_destroy(wpcd_mlp *m);
wpcd_status wpcd_mlp_info(const wpcd_mlp *m, int64_t *n_params, int *n_in, int *width, int *n_out);

/* Flat FP32 parameters [W1 (width x n_in), b1, W2 (width x width), b2,
 * W3 (n_out x width), b3], weights row-major (output x input); `get` and
 * `set` (either may be NULL) are host or device arrays of n_params. */
wpcd_status wpcd_mlp_params(wpcd_mlp *m, float *get, const float *set);

/* Input map x -> x * in_scale + in_shift before layer 1 and output map
 * z -> z * out_scale + out_shift after layer 3 (training fits z to the
 * targets mapped back by the inverse of the output map).  Host or device
 * arrays; NULL leaves a map unchanged. */
wpcd_status wpcd_mlp_set_affine(wpcd_mlp *m, const float *in_scale, const float *in_shift,
                                const float *out_scale, const float *out_shift);

/* Y [n][n_out] = MLP(X [n][n_in]) (device FP32); bf16 != 0 uses BF16 weights. */
wpcd_status wpcd_mlp_forward(wpcd_mlp *m, const float *X, int n, float *Y, int bf16, void *stream);

/* Mean squared error of the normalised outputs against targets T [n][n_out]
 * (host *loss) and its gradient (device grad [n_params], may be NULL). */
wpcd_status wpcd_mlp_loss_grad(wpcd_mlp *m, const float *X, const float *T, int n, float *loss, float *grad,
                               void *stream);

/* Minibatch Adam (lr, beta 0.9 / 0.999, eps 1e-8) over `epochs` shuffles of
 * the n rows (X, T), batches of `batch` (a trailing partial batch is
 * skipped); loss_hist: host [epochs] mean batch loss per epoch, or NULL. */
wpcd_status wpcd_mlp_train(wpcd_mlp *m, const float *X, const float *T, int n, int epochs, int batch, float lr,
                           uint64_t seed, float *loss_hist, void *stream);

/* Projected basis: C [n][k] = <Phi_j, U_e> (complex FP64, device) for
 * Phi [k][dim] and U [n][dim]. */
wpcd_status wpcd_basis_project(const double *Phi, int k, int dim, const double *U, int n, double *C,
                               void *stream);
/* U [n][dim] = sum_j C[e][j] Phi_j with C as FP32 (re, im) pairs [n][k][2]. */
wpcd_status wpcd_basis_expand(const double *Phi, int k, int dim, const float *C, int n, double *U,
                              void *stream);
/* Orthonormalise the k rows of Phi [k][dim] in place (two-pass modified
 * Gram-Schmidt). */
wpcd_status wpcd_basis_orthonormalize(double *Phi, int k, int dim, void *stream);
/* X [n][1 + 2 kf] = [(Ebin - e_lo)/(e_hi - e_lo), Re/Im Cb[e][0..kf)]
 * (FP32, device), Ebin the centre of E's on-shell energy bin (G1 depends on E
 * through that bin only), E host [n], Cb [n][k] complex FP64 device (the Born
 * term's coefficients in the basis). */
wpcd_status wpcd_warm_features(const wpcd_problem *pr, const double *E, int n, double e_lo, double e_hi,
                               const double *Cb, int k, int kf, float *X, void *stream);
/* y += alpha x over n reals (device FP64). */
wpcd_status wpcd_vec_axpy(double alpha, const double *x, double *y, int64_t n, void *stream);
/* dst [2n] FP32 (re, im) pairs from src [n] complex FP64 (device). */
wpcd_status wpcd_complex_to_f32(const double *src, int64_t n, float *dst, void *stream);
/* The float-float split of the mixed solve's FP64-class residual (Sec. 4.1
 * precision): for n FP64 values x (device), hi = x rounded to the nearest
 * float (ties to even) and lo = (x - hi) rounded likewise, so hi + lo carries
 * x to about 2^-48; values whose part lies below the float normal range
 * (2^-126) give zero there instead of a subnormal.  hi, lo device [n] FP32,
 * caller-owned.  EINVAL for null pointers or n < 0.  Enqueued on stream. */
wpcd_status wpcd_split_f64(const double *x, int64_t n, float *hi, float *lo, void *stream);
/* Mixture weights of the warm start: for each of n rows of k logits (FP32,
 * device [n][k]) the softmax w_j = exp(z_j - max z) / sum_i exp(z_i - max z),
 * written as real coefficients C [n][k][2] = (w_j, 0) for wpcd_basis_expand.
 * EINVAL for n < 1 or k < 1 or k > 1024. */
wpcd_status wpcd_warm_softmax(const float *logits, int n, int k, float *C, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* WPCD_H */
