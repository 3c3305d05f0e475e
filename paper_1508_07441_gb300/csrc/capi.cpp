// extern "C" entry points of include/wpcd.h: argument validation, handle
// lifetime, uploads, and error reporting.  No C++ exception crosses the ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "wpcd_internal.h"

namespace wpcd {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

wpcd_status set_error(wpcd_status st, const std::string &msg) {
  g_last_error = msg;
  return st;
}

wpcd_status cuda_error(cudaError_t e, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return WPCD_ECUDA;
}

// Called on entry to the ABI calls that launch work: clears this thread's
// message and any CUDA error another component left pending in the runtime
// (cudaGetLastError is per host thread), so that the launch checks below
// report this library's own failures only.
void clear_error() {
  g_last_error.clear();
  (void)cudaGetLastError();
}

// WPCD_POOL=0 takes the work space with cudaMalloc / cudaFree instead (for
// tools that save and restore device allocations around a kernel, which
// know plain allocations)
static bool pool_enabled() {
  static const bool on = [] {
    const char *v = std::getenv("WPCD_POOL");
    return !(v && std::strcmp(v, "0") == 0);
  }();
  return on;
}

// the caller's allocator (wpcd_set_allocator), and the number of live
// blocks of whichever allocator is current
struct AllocHook {
  wpcd_alloc_fn alloc = nullptr;
  wpcd_free_fn free = nullptr;
  void *user = nullptr;
};
static std::mutex g_hook_mu;
static AllocHook g_hook;
static std::atomic<long long> g_live{0};

static AllocHook current_hook() {
  std::lock_guard<std::mutex> lock(g_hook_mu);
  return g_hook;
}

static cudaError_t hook_alloc(const AllocHook &h, void **p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  void *q = h.alloc(bytes ? bytes : 16, dev, static_cast<void *>(s), h.user);
  if (!q) return cudaErrorMemoryAllocation;
  *p = q;
  ++g_live;
  return cudaSuccess;
}

cudaError_t dev_malloc(void **p, size_t bytes) {
  const AllocHook h = current_hook();
  if (h.alloc) return hook_alloc(h, p, bytes, nullptr);
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e == cudaSuccess) ++g_live;
  return e;
}

void dev_free(void *p) {
  if (!p) return;
  --g_live;
  const AllocHook h = current_hook();
  if (h.free) {
    cudaDeviceSynchronize();  // as cudaFree: no queued work still uses the block
    h.free(p, nullptr, h.user);
  } else {
    cudaFree(p);
  }
}

cudaError_t pool_malloc(void **p, size_t bytes, cudaStream_t s) {
  const AllocHook h = current_hook();
  if (h.alloc) return hook_alloc(h, p, bytes, s);
  cudaError_t e;
  if (!pool_enabled()) {
    e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) ++g_live;
    return e;
  }
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
      cudaMemPoolProps props{};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      if ((e = cudaMemPoolCreate(&pools[dev], &props)) != cudaSuccess) return e;
      // keep freed blocks for reuse rather than returning them at each sync
      uint64_t keep = UINT64_MAX;
      if ((e = cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) return e;
    }
    pool = pools[dev];
  }
  e = cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, s);
  if (e == cudaSuccess) ++g_live;
  return e;
}

void pool_free(void *p, cudaStream_t s) {
  if (!p) return;
  --g_live;
  const AllocHook h = current_hook();
  if (h.free)
    h.free(p, static_cast<void *>(s), h.user);
  else if (pool_enabled())
    cudaFreeAsync(p, s);
  else
    cudaFree(p);
}

static void free_tables(DeviceTables &d) {
  // the lattice tables (pe2 ... qe) belong to the grid: not freed here
  double **all[] = {&d.eps, &d.O, &d.Vt};
  for (double **p : all) {
    dev_free(*p);
    *p = nullptr;
  }
  dev_free(d.O32);
  dev_free(d.Vt32);
  d.O32 = d.Vt32 = nullptr;
  dev_free(d.O_tc);
  dev_free(d.Vt_tc);
  dev_free(d.O_h);
  dev_free(d.O_l);
  dev_free(d.Vt_h);
  dev_free(d.Vt_l);
  d.O_h = d.O_l = d.Vt_h = d.Vt_l = nullptr;
  dev_free(d.O_oz);
  dev_free(d.Vt_oz);
  dev_free(d.O_ozE);
  dev_free(d.Vt_ozE);
  d.O_oz = d.Vt_oz = nullptr;
  d.O_ozE = d.Vt_ozE = nullptr;
  dev_free(d.tc_err);
  d.O_tc = d.Vt_tc = nullptr;
  d.tc_err = nullptr;
}

static wpcd_status upload32(float **dst, const std::vector<double> &src) {
  std::vector<float> f(src.begin(), src.end());
  cudaError_t e = dev_malloc(dst, sizeof(float) * (f.empty() ? 1 : f.size()));
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc (problem tables)");
  if (!f.empty()) {
    e = cudaMemcpy(*dst, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy (problem tables)");
  }
  return WPCD_OK;
}

static wpcd_status upload(double **dst, const std::vector<double> &src) {
  cudaError_t e = dev_malloc(dst, sizeof(double) * (src.empty() ? 1 : src.size()));
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc (problem tables)");
  if (!src.empty()) {
    e = cudaMemcpy(*dst, src.data(), sizeof(double) * src.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy (problem tables)");
  }
  return WPCD_OK;
}

static bool valid_edges(const double *e, int n) {
  if (!e || !(e[0] == 0.0)) return false;
  for (int k = 0; k < n; ++k)
    if (!(e[k + 1] > e[k]) || !std::isfinite(e[k + 1])) return false;
  return true;
}

static void free_grid_tables(wpcd_grid &g) {
  double **all[] = {&g.pe2, &g.qe2, &g.pn, &g.wp, &g.qn, &g.wq, &g.yn, &g.wy, &g.rsb, &g.qe_d};
  for (double **p : all) {
    dev_free(*p);
    *p = nullptr;
  }
}

void grid_retain(wpcd_grid *g) { g->refs.fetch_add(1, std::memory_order_relaxed); }

void grid_release(wpcd_grid *g) {
  if (!g || g->refs.fetch_sub(1, std::memory_order_acq_rel) != 1) return;
  cudaSetDevice(g->device);
  free_grid_tables(*g);
  delete g;
}

// Step 1, the lattice part (Sec. 2.2 Eq. ip, Sec. 2.4 Eq. xij): edges, the
// GL node and weight tables of every bin, squared edges and the cell norms
// 1/sqrt(B_i Bq_j), uploaded once; everything P0 needs
static wpcd_status grid_create(const wpcd_grid_desc *d, wpcd_grid **out) {
  if (!d || !out) return set_error(WPCD_EINVAL, "null argument");
  *out = nullptr;
  if (d->N < 1 || d->M < 1) return set_error(WPCD_EINVAL, "N and M must be >= 1");
  if ((int64_t)d->N * d->M > (1 << 24)) return set_error(WPCD_EINVAL, "lattice too large (N*M > 2^24)");
  if (d->n_p < 1 || d->n_q < 1 || d->n_x < 1 || d->n_p > 64 || d->n_q > 64 || d->n_x > 256)
    return set_error(WPCD_EINVAL, "node counts must be in [1, 64] (p, q) and [1, 256] (x)");
  if (!valid_edges(d->p_edges, d->N) || !valid_edges(d->q_edges, d->M))
    return set_error(WPCD_EINVAL, "edges must start at 0 and increase strictly");
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess) return cuda_error(ce, "cudaGetDeviceCount");
  if (d->device < 0 || d->device >= ndev) return set_error(WPCD_EINVAL, "no such CUDA device");
  ce = cudaSetDevice(d->device);
  if (ce != cudaSuccess) return cuda_error(ce, "cudaSetDevice");
  wpcd_grid *g = new (std::nothrow) wpcd_grid();
  if (!g) return set_error(WPCD_ENOMEM, "host allocation");
  g->device = d->device;
  g->N = d->N;
  g->M = d->M;
  g->n_p = d->n_p;
  g->n_q = d->n_q;
  g->n_x = d->n_x;
  g->pe.assign(d->p_edges, d->p_edges + d->N + 1);
  g->qe.assign(d->q_edges, d->q_edges + d->M + 1);
  const int N = d->N, M = d->M;
  // node and edge tables (canonical node placement: mid + half * t)
  std::vector<double> tp(d->n_p), wp(d->n_p), tq(d->n_q), wq(d->n_q), ty(d->n_x), wy(d->n_x);
  gauss_legendre(d->n_p, tp.data(), wp.data());
  gauss_legendre(d->n_q, tq.data(), wq.data());
  gauss_legendre(d->n_x, ty.data(), wy.data());
  g->y_ascending = true;
  for (int x = 1; x < d->n_x; ++x) g->y_ascending = g->y_ascending && ty[x] > ty[x - 1];
  std::vector<double> pn((size_t)N * d->n_p), pw((size_t)N * d->n_p), qn((size_t)M * d->n_q),
      qw((size_t)M * d->n_q), pe2(N + 1), qe2(M + 1), rsb((size_t)N * M);
  for (int i = 0; i < N; ++i) {
    double lo = g->pe[i], hi = g->pe[i + 1], half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
    for (int a = 0; a < d->n_p; ++a) {
      double p = mid + half * tp[a];
      pn[(size_t)i * d->n_p + a] = p;
      pw[(size_t)i * d->n_p + a] = half * wp[a] * p * p;
    }
  }
  for (int j = 0; j < M; ++j) {
    double lo = g->qe[j], hi = g->qe[j + 1], half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
    for (int b = 0; b < d->n_q; ++b) {
      double q = mid + half * tq[b];
      qn[(size_t)j * d->n_q + b] = q;
      qw[(size_t)j * d->n_q + b] = half * wq[b] * q * q;
    }
  }
  for (int k = 0; k <= N; ++k) pe2[k] = g->pe[k] * g->pe[k];
  for (int k = 0; k <= M; ++k) qe2[k] = g->qe[k] * g->qe[k];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < M; ++j)
      rsb[(size_t)i * M + j] = 1.0 / std::sqrt(shell_volume(g->pe[i], g->pe[i + 1]) *
                                               shell_volume(g->qe[j], g->qe[j + 1]));
  wpcd_status st = WPCD_OK;
  if ((st = upload(&g->pe2, pe2)) || (st = upload(&g->qe2, qe2)) || (st = upload(&g->pn, pn)) ||
      (st = upload(&g->wp, pw)) || (st = upload(&g->qn, qn)) || (st = upload(&g->wq, qw)) ||
      (st = upload(&g->yn, ty)) || (st = upload(&g->wy, wy)) || (st = upload(&g->rsb, rsb)) ||
      (st = upload(&g->qe_d, g->qe))) {
    free_grid_tables(*g);
    delete g;
    return st;
  }
  *out = g;
  return WPCD_OK;
}

// Step 1, the pair part (Sec. 3.3 "processing of the input data"; Sec. 2.2
// Eq. vpot, Eq. exp_z): free-packet potential matrices v_l on the grid's p
// bins, diagonalisation of h1 = h0 + v in every channel (O, eps), Vt = v O^T,
// uploaded; the lattice tables are the grid's (the problem holds a reference)
static wpcd_status check_pair_desc(const wpcd_pair_desc *d) {
  if (d->n_ch < 1 || d->n_ch > 5) return set_error(WPCD_EINVAL, "n_ch must be in [1, 5]");
  if (d->n_terms < 1 || !d->V || !d->a) return set_error(WPCD_EINVAL, "potential needs >= 1 term");
  for (int k = 0; k < d->n_terms; ++k)
    if (!std::isfinite(d->V[k]) || !(d->a[k] > 0.0) || !std::isfinite(d->a[k]))
      return set_error(WPCD_EINVAL, "potential terms must be finite with a_k > 0");
  if (d->n_pair_nodes < 1 || d->n_pair_nodes > 64) return set_error(WPCD_EINVAL, "n_pair_nodes in [1, 64]");
  return WPCD_OK;
}

static wpcd_status pair_create(wpcd_grid *g, const wpcd_pair_desc *d, wpcd_problem **out) {
  if (!g || !d || !out) return set_error(WPCD_EINVAL, "null argument");
  *out = nullptr;
  wpcd_status vst = check_pair_desc(d);
  if (vst != WPCD_OK) return vst;
  cudaError_t ce = cudaSetDevice(g->device);
  if (ce != cudaSuccess) return cuda_error(ce, "cudaSetDevice");
  wpcd_problem *pr = new (std::nothrow) wpcd_problem();
  if (!pr) return set_error(WPCD_ENOMEM, "host allocation");
  pr->device = g->device;
  pr->N = g->N;
  pr->M = g->M;
  pr->n_p = g->n_p;
  pr->n_q = g->n_q;
  pr->n_x = g->n_x;
  pr->n_ch = d->n_ch;
  int np = 0;
  for (int l = 0; l < d->n_ch; ++l)
    for (int lp = 0; lp < d->n_ch; ++lp)
      if (((l + lp) & 1) == 0) {
        pr->pair_l[np] = l;
        pr->pair_lp[np] = lp;
        ++np;
      }
  pr->n_pairs = np;
  pr->pe = g->pe;
  pr->qe = g->qe;
  const int N = g->N;
  // pair quantities per channel
  pr->eps.assign((size_t)d->n_ch * N, 0.0);
  pr->O.assign((size_t)d->n_ch * N * N, 0.0);
  pr->v.assign((size_t)d->n_ch * N * N, 0.0);
  pr->Vt.assign((size_t)d->n_ch * N * N, 0.0);
  // the potential matrices of every channel on the device, then the
  // channels' eigenproblems side by side on the host cores
  std::vector<std::vector<double>> vs(d->n_ch), hs(d->n_ch), epss(d->n_ch), Os(d->n_ch);
  wpcd_status pst = pair_matrices_gpu(g->device, N, g->pe.data(), d->n_pair_nodes, d->n_ch, d->n_terms, d->V, d->a, vs);
  if (pst != WPCD_OK) {
    delete pr;
    return pst;
  }
  pair_h(N, g->pe.data(), d->n_ch, vs, hs);
#pragma omp parallel for schedule(dynamic, 1)
  for (int l = 0; l < d->n_ch; ++l) pair_eig(N, hs[l], epss[l], Os[l]);
  for (int l = 0; l < d->n_ch; ++l) {
    const std::vector<double> &v = vs[l], &eps = epss[l], &O = Os[l];
    if ((int)eps.size() != N) {
      delete pr;
      return set_error(WPCD_EINVAL, "pair Hamiltonian eigensolver did not converge");
    }
    std::copy(eps.begin(), eps.end(), pr->eps.begin() + (size_t)l * N);
    std::copy(O.begin(), O.end(), pr->O.begin() + (size_t)l * N * N);
    std::copy(v.begin(), v.end(), pr->v.begin() + (size_t)l * N * N);
    // Vt = O^T V1 in the channel basis = v O^T:  Vt[i][k] = sum_m v[i][m] O[k][m],
    // sixteen outputs of a row at a time held in registers, each summed over
    // m ascending (the order of the plain dot product) from a row of O^T:
    // independent lanes instead of one dependent sum per element (4 ms -> 1
    // ms for three 200 x 200 channels on eight cores, the same bits)
    double *Vt = pr->Vt.data() + (size_t)l * N * N;
    std::vector<double> OT((size_t)N * N);
    for (int k = 0; k < N; ++k)
      for (int m = 0; m < N; ++m) OT[(size_t)m * N + k] = O[(size_t)k * N + m];
    constexpr int KB = 16;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
      const double *vi = v.data() + (size_t)i * N;
      for (int k0 = 0; k0 < N; k0 += KB) {
        const int kn = std::min(KB, N - k0);
        double acc[KB] = {};
        if (kn == KB) {
          for (int m = 0; m < N; ++m) {
            const double a = vi[m], *om = OT.data() + (size_t)m * N + k0;
            for (int j = 0; j < KB; ++j) acc[j] += a * om[j];
          }
        } else {
          for (int m = 0; m < N; ++m) {
            const double a = vi[m], *om = OT.data() + (size_t)m * N + k0;
            for (int j = 0; j < kn; ++j) acc[j] += a * om[j];
          }
        }
        for (int j = 0; j < kn; ++j) Vt[(size_t)i * N + k0 + j] = acc[j];
      }
    }
  }
  pr->eps_b = pr->eps[0];
  if (!(pr->eps_b < 0.0)) {
    delete pr;
    return set_error(WPCD_ENOBOUND, "channel 0 has no bound pair state on this grid");
  }
  wpcd_status st = WPCD_OK;
  DeviceTables &t = pr->d;
  if ((st = upload(&t.eps, pr->eps)) || (st = upload(&t.O, pr->O)) || (st = upload(&t.Vt, pr->Vt)) ||
      (st = upload32(&t.O32, pr->O)) || (st = upload32(&t.Vt32, pr->Vt))) {
    free_tables(t);
    delete pr;
    return st;
  }
  // the lattice tables: the grid's
  t.pe2 = g->pe2;
  t.qe2 = g->qe2;
  t.pn = g->pn;
  t.wp = g->wp;
  t.qn = g->qn;
  t.wq = g->wq;
  t.yn = g->yn;
  t.wy = g->wy;
  t.rsb = g->rsb;
  t.qe = g->qe_d;
  pr->grid = g;
  grid_retain(g);
  *out = pr;
  return WPCD_OK;
}

// wpcd_problem_create: a grid of its own and the pair setup on it
static wpcd_status create(const wpcd_problem_desc *d, wpcd_problem **out) {
  if (!d || !out) return set_error(WPCD_EINVAL, "null argument");
  *out = nullptr;
  const wpcd_pair_desc pd{d->n_ch, d->n_terms, d->V, d->a, d->n_pair_nodes};
  wpcd_status st = check_pair_desc(&pd);  // every input checked before any device call
  if (st != WPCD_OK) return st;
  const wpcd_grid_desc gd{d->N, d->M, d->p_edges, d->q_edges, d->n_p, d->n_q, d->n_x, d->device};
  wpcd_grid *g = nullptr;
  st = grid_create(&gd, &g);
  if (st != WPCD_OK) return st;
  st = pair_create(g, &pd, out);
  grid_release(g);  // the problem holds the remaining reference
  return st;
}
}  // namespace wpcd

using namespace wpcd;

extern "C" {

const char *wpcd_last_error(void) { return g_last_error.c_str(); }

int wpcd_version(void) { return 100; }

int64_t wpcd_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

wpcd_status wpcd_debug_expire_first_wait(int kernel, int role) {
  clear_error();
  if (kernel == 0) {
    g_ws_expire_role.store(-1);
    g_oz_expire_first.store(0);
  } else if (kernel == 1 && role >= 0 && role <= 3) {
    g_ws_expire_role.store(role);
  } else if (kernel == 2 && role == 0) {
    g_oz_expire_first.store(1);
  } else {
    return set_error(WPCD_EINVAL, "kernel 1 takes roles 0-3, kernel 2 role 0, kernel 0 clears");
  }
  return WPCD_OK;
}

wpcd_status wpcd_set_allocator(wpcd_alloc_fn alloc, wpcd_free_fn free_fn, void *user) {
  clear_error();
  if ((alloc == nullptr) != (free_fn == nullptr)) return set_error(WPCD_EINVAL, "give both allocator callbacks or neither");
  std::lock_guard<std::mutex> lock(g_hook_mu);
  const long long live = g_live.load();
  if (live != 0)
    return set_error(WPCD_EINVAL, "device blocks of the current allocator are live (" + std::to_string(live) +
                                      "); set the allocator before creating handles or after destroying them");
  g_hook.alloc = alloc;
  g_hook.free = free_fn;
  g_hook.user = user;
  return WPCD_OK;
}

wpcd_status wpcd_tangent_edges(int n_bins, double k_max, double *edges) {
  if (n_bins < 1 || !(k_max > 0.0) || !std::isfinite(k_max) || !edges)
    return set_error(WPCD_EINVAL, "tangent edges need n_bins >= 1, finite k_max > 0");
  const double half_pi = 1.5707963267948966192;
  double span = half_pi / (n_bins + 1.0);
  double scale = k_max / std::tan(span * n_bins);
  edges[0] = 0.0;
  for (int n = 1; n < n_bins; ++n) edges[n] = scale * std::tan(span * n);
  edges[n_bins] = k_max;
  return WPCD_OK;
}

wpcd_status wpcd_problem_create(const wpcd_problem_desc *desc, wpcd_problem **out) {
  WPCD_GUARD_BEGIN
  clear_error();
  return create(desc, out);
  WPCD_GUARD_END
}

void wpcd_problem_destroy(wpcd_problem *pr) {
  if (!pr) return;
  cudaSetDevice(pr->device);
  free_tables(pr->d);
  grid_release(pr->grid);
  delete pr;
}

wpcd_status wpcd_problem_info(const wpcd_problem *pr, int *dim, int *n_pairs, double *eps_bound) {
  if (!pr) return set_error(WPCD_EINVAL, "null problem");
  if (dim) *dim = pr->n_ch * pr->N * pr->M;
  if (n_pairs) *n_pairs = pr->n_pairs;
  if (eps_bound) *eps_bound = pr->eps_b;
  return WPCD_OK;
}

wpcd_status wpcd_problem_pair(const wpcd_problem *pr, int l, double *eps, double *O, double *v) {
  if (!pr || l < 0 || l >= pr->n_ch) return set_error(WPCD_EINVAL, "bad problem or channel");
  const size_t N = pr->N;
  if (eps) std::memcpy(eps, pr->eps.data() + l * N, sizeof(double) * N);
  if (O) std::memcpy(O, pr->O.data() + l * N * N, sizeof(double) * N * N);
  if (v) std::memcpy(v, pr->v.data() + l * N * N, sizeof(double) * N * N);
  return WPCD_OK;
}

wpcd_status wpcd_assemble_P(wpcd_problem *pr, int prec, void *stream, wpcd_P **out) {
  WPCD_GUARD_BEGIN
  clear_error();
  if (!pr || !out) return set_error(WPCD_EINVAL, "null argument");
  *out = nullptr;
  if (prec == WPCD_FP64_VL) return assemble_vl(pr->grid, pr->n_ch, static_cast<cudaStream_t>(stream), out);
  return assemble(pr->grid, pr->n_ch, prec, static_cast<cudaStream_t>(stream), out);
  WPCD_GUARD_END
}

wpcd_status wpcd_grid_create(const wpcd_grid_desc *desc, wpcd_grid **out) {
  WPCD_GUARD_BEGIN
  clear_error();
  return grid_create(desc, out);
  WPCD_GUARD_END
}

void wpcd_grid_destroy(wpcd_grid *g) { grid_release(g); }

wpcd_status wpcd_pair_create(wpcd_grid *g, const wpcd_pair_desc *desc, wpcd_problem **out) {
  WPCD_GUARD_BEGIN
  clear_error();
  return pair_create(g, desc, out);
  WPCD_GUARD_END
}

wpcd_status wpcd_assemble_P_grid(wpcd_grid *g, int n_ch, int prec, void *stream, wpcd_P **out) {
  WPCD_GUARD_BEGIN
  clear_error();
  if (!g || !out) return set_error(WPCD_EINVAL, "null argument");
  *out = nullptr;
  if (prec == WPCD_FP64_VL) return assemble_vl(g, n_ch, static_cast<cudaStream_t>(stream), out);
  return assemble(g, n_ch, prec, static_cast<cudaStream_t>(stream), out);
  WPCD_GUARD_END
}

wpcd_status wpcd_problem_grid(const wpcd_problem *pr, wpcd_grid **out) {
  if (!pr || !out) return set_error(WPCD_EINVAL, "null argument");
  grid_retain(pr->grid);
  *out = pr->grid;
  return WPCD_OK;
}

void wpcd_P_destroy(wpcd_P *P) {
  if (!P) return;
  cudaSetDevice(P->device);
  dev_free(P->row_ptr);
  dev_free(P->col);
  dev_free(P->val64);
  dev_free(P->val32);
  dev_free(P->val32_copy);
  dev_free(P->val_h);
  dev_free(P->val_l);
  for (int i = 0; i < 2; ++i) {
    dev_free(P->tile_ptr[i]);
    dev_free(P->tile_col[i]);
    dev_free(P->tile_val[i]);
  }
  grid_release(P->grid);
  delete P;
}

wpcd_status wpcd_P_info(const wpcd_P *P, int64_t *nnz, int *n_pairs, int *prec, float *ms) {
  if (!P) return set_error(WPCD_EINVAL, "null P");
  if (nnz) *nnz = P->nnz;
  if (n_pairs) *n_pairs = P->n_pairs;
  if (prec) *prec = P->prec;
  if (ms) *ms = P->ms;
  return WPCD_OK;
}

wpcd_status wpcd_P_work(const wpcd_P *P, int64_t *points) {
  if (!P || !points) return set_error(WPCD_EINVAL, "null argument");
  *points = P->work;
  return WPCD_OK;
}

wpcd_status wpcd_P_timing(const wpcd_P *P, float ms[3]) {
  if (!P || !ms) return set_error(WPCD_EINVAL, "null argument");
  for (int i = 0; i < 3; ++i) ms[i] = P->ms_phase[i];
  return WPCD_OK;
}

wpcd_status wpcd_P_export(const wpcd_P *P, int64_t *row_ptr, int32_t *col, double *val, void *stream) {
  WPCD_GUARD_BEGIN
  clear_error();
  if (!P) return set_error(WPCD_EINVAL, "null P");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  WPCD_CUDA_TRY(cudaSetDevice(P->device));
  const size_t ncell = (size_t)P->grid->N * P->grid->M;
  if (row_ptr) WPCD_CUDA_TRY(cudaMemcpyAsync(row_ptr, P->row_ptr, sizeof(int64_t) * (ncell + 1), cudaMemcpyDefault, s));
  if (col && P->nnz) WPCD_CUDA_TRY(cudaMemcpyAsync(col, P->col, sizeof(int32_t) * P->nnz, cudaMemcpyDefault, s));
  if (val && P->nnz) {
    const size_t n = (size_t)P->nnz * P->n_pairs;
    if (P->prec == WPCD_FP64) {
      WPCD_CUDA_TRY(cudaMemcpyAsync(val, P->val64, sizeof(double) * n, cudaMemcpyDefault, s));
    } else {
      std::vector<float> tmp(n);
      WPCD_CUDA_TRY(cudaMemcpyAsync(tmp.data(), P->val32, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
      WPCD_CUDA_TRY(cudaStreamSynchronize(s));
      std::vector<double> wide(tmp.begin(), tmp.end());
      WPCD_CUDA_TRY(cudaMemcpy(val, wide.data(), sizeof(double) * n, cudaMemcpyDefault));
    }
  }
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  return WPCD_OK;
  WPCD_GUARD_END
}

wpcd_status wpcd_resolvent(const wpcd_problem *pr, const double *E, int n_E, double *g, int *j0,
                           double *D, void *stream) {
  WPCD_GUARD_BEGIN
  clear_error();
  if (!pr) return set_error(WPCD_EINVAL, "null problem");
  return resolvent(pr, E, n_E, g, j0, D, static_cast<cudaStream_t>(stream));
  WPCD_GUARD_END
}

wpcd_status wpcd_kapply(const wpcd_problem *pr, const wpcd_P *P, const double *g, const double *x,
                        double *y, void *stream) {
  WPCD_GUARD_BEGIN
  clear_error();
  if (!pr || !P || !x || !y || x == y) return set_error(WPCD_EINVAL, "bad kapply arguments");
  if (!P_fits(P, pr)) return set_error(WPCD_EINVAL, "P was assembled on another lattice or for another channel count");
  return kapply(pr, P, g, x, y, static_cast<cudaStream_t>(stream));
  WPCD_GUARD_END
}

wpcd_status wpcd_solve(wpcd_problem *pr, const wpcd_P *P, const double *E, int n_E,
                       const wpcd_solve_opts *opts, double *U00, wpcd_solve_stats *stats, void *stream) {
  WPCD_GUARD_BEGIN
  clear_error();
  if (!pr || !P) return set_error(WPCD_EINVAL, "null problem or P");
  if (!P_fits(P, pr)) return set_error(WPCD_EINVAL, "P was assembled on another lattice or for another channel count");
  return solve(pr, P, E, n_E, opts, U00, stats, static_cast<cudaStream_t>(stream));
  WPCD_GUARD_END
}

wpcd_status wpcd_solve_batch(int n_prob, wpcd_problem *const *problems, const wpcd_P *const *P,
                             const double *const *E, const int *n_E, const wpcd_solve_opts *opts,
                             double *const *U00, wpcd_solve_stats *const *stats, void *stream) {
  WPCD_GUARD_BEGIN
  clear_error();
  return solve_group(n_prob, problems, P, E, n_E, opts, U00, stats, static_cast<cudaStream_t>(stream));
  WPCD_GUARD_END
}

wpcd_status wpcd_spmm(wpcd_problem *pr, wpcd_P *P, int mode, const void *y, void *z, int n_rhs, float *kernel_ms,
                      void *stream) {
  WPCD_GUARD_BEGIN
  clear_error();
  if (!pr || !P) return set_error(WPCD_EINVAL, "null problem or P");
  if (!P_fits(P, pr)) return set_error(WPCD_EINVAL, "P was assembled on another lattice or for another channel count");
  return spmm_apply(pr, P, mode, y, z, n_rhs, kernel_ms, static_cast<cudaStream_t>(stream));
  WPCD_GUARD_END
}

wpcd_status wpcd_channel_gemm(wpcd_problem *pr, int which, int mode, const void *g, const void *x, void *y,
                              int n_rhs, float *kernel_ms, void *stream) {
  WPCD_GUARD_BEGIN
  clear_error();
  if (!pr) return set_error(WPCD_EINVAL, "null problem");
  return channel_gemm(pr, which, mode, g, x, y, n_rhs, kernel_ms, static_cast<cudaStream_t>(stream));
  WPCD_GUARD_END
}

wpcd_status wpcd_born(wpcd_problem *pr, const wpcd_P *P, const double *E, int n_E, double *b, void *stream) {
  WPCD_GUARD_BEGIN
  clear_error();
  if (!pr || !P || !P_fits(P, pr)) return set_error(WPCD_EINVAL, "bad problem or P");
  return born_vectors(pr, P, E, n_E, b, static_cast<cudaStream_t>(stream));
  WPCD_GUARD_END
}

wpcd_status wpcd_tune_spmm(wpcd_problem *pr, wpcd_P *P, int n_rhs, int mode, void *stream,
                           int *rows_per_warp, int *energy_lanes, int *energies_per_lane) {
  WPCD_GUARD_BEGIN
  clear_error();
  if (!pr || !P || !P_fits(P, pr)) return set_error(WPCD_EINVAL, "bad problem or P");
  if (n_rhs < 1 || n_rhs > 1024) return set_error(WPCD_EINVAL, "n_rhs must be in [1, 1024]");
  if (mode < WPCD_SPMM_FP64 || mode > WPCD_SPMM_FF) return set_error(WPCD_EINVAL, "unknown SpMM mode");
  if (mode == WPCD_SPMM_FP32 && !P->val32 && !P->val32_copy)
    return set_error(WPCD_EINVAL, "FP32 tuning needs an FP32C P (or a mixed solve first)");
  WPCD_CUDA_TRY(cudaSetDevice(pr->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (mode == WPCD_SPMM_FF) {
    wpcd_status st = df_prepare(pr, P, s);
    if (st != WPCD_OK) return st;
  }
  SpmmConfig c;
  wpcd_status st = tune_spmm(pr, P, n_rhs, mode, s, &c);
  if (st != WPCD_OK) return st;
  if (rows_per_warp) *rows_per_warp = c.tile ? c.tile : c.rpw;  // a tile's rows per warp
  if (energy_lanes) *energy_lanes = c.el;
  if (energies_per_lane) *energies_per_lane = c.ept;
  return WPCD_OK;
  WPCD_GUARD_END
}

}  // extern "C"
