// Learned warm start for the Faddeev iteration: a 3-layer MLP (tanh hidden
// layers) trained on the GPU by hand-written forward, backward and Adam
// kernels (FP32), inferred with BF16 weights (FP32 arithmetic), plus the
// projected-basis helpers (Born terms, orthonormalisation, projection and
// expansion) that turn its outputs into a starting vector for the solve.
// The paper has no learned component; this is a growth line around its
// iteration, which stays the fallback and decides convergence.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <vector>

#include "wpcd_internal.h"

struct wpcd_mlp {
  int device = 0, n_in = 0, width = 0, n_out = 0;
  int64_t n_params = 0;
  float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  __nv_bfloat16 *params_bf16 = nullptr;
  bool bf16_stale = true;
  float *in_scale = nullptr, *in_shift = nullptr, *out_scale = nullptr, *out_shift = nullptr;
  int cap = 0;  // rows of the scratch buffers
  float *xn = nullptr, *h1 = nullptr, *h2 = nullptr, *z = nullptr, *dz = nullptr, *d1 = nullptr,
        *d2 = nullptr, *loss = nullptr, *tn = nullptr;
  int *idx = nullptr;
  int64_t adam_t = 0;
  // parameter offsets: W1 [width][n_in], b1, W2 [width][width], b2,
  // W3 [n_out][width], b3
  int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
};

namespace wpcd {
namespace {

// splitmix64: counter-based generator (Steele, Lea, Flood 2014)
uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
double uniform01(uint64_t seed, uint64_t i) { return (splitmix64(seed * 0x100000001B3ull + i) >> 11) * 0x1.0p-53; }

// ---------------------------------------------------------------------------
// generic small GEMM:  C[m][n] = act(sum_k A(m,k) B(k,n) + bias[n]) (+ C)
// A(m,k) = A[m * sam + k * sak], B(k,n) = B[k * sbk + n * sbn]; B may be BF16
// ---------------------------------------------------------------------------
constexpr int MT = 32, NT = 32, KT = 16;

template <typename TB>
__device__ __forceinline__ float ldb(const TB *B, int64_t i);
template <>
__device__ __forceinline__ float ldb<float>(const float *B, int64_t i) { return B[i]; }
template <>
__device__ __forceinline__ float ldb<__nv_bfloat16>(const __nv_bfloat16 *B, int64_t i) {
  return __bfloat162float(B[i]);
}

template <typename TB>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, const float *A, int64_t sam,
                                                    int64_t sak, const TB *B, int64_t sbk, int64_t sbn,
                                                    const float *bias, int act, int accumulate, float *C,
                                                    int64_t ldc) {
  __shared__ float As[KT][MT + 1];
  __shared__ float Bs[KT][NT + 1];
  const int m0 = blockIdx.y * MT, n0 = blockIdx.x * NT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 2 x 2 outputs each
  float acc[2][2] = {};
  for (int k0 = 0; k0 < K; k0 += KT) {
    for (int t = threadIdx.x; t < MT * KT; t += 256) {
      int r = t / KT, kk = t % KT;
      As[kk][r] = (m0 + r < M && k0 + kk < K) ? A[(int64_t)(m0 + r) * sam + (int64_t)(k0 + kk) * sak] : 0.f;
    }
    for (int t = threadIdx.x; t < NT * KT; t += 256) {
      int kk = t / NT, cc = t % NT;
      Bs[kk][cc] = (n0 + cc < N && k0 + kk < K) ? ldb<TB>(B, (int64_t)(k0 + kk) * sbk + (int64_t)(n0 + cc) * sbn) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
      float a0 = As[kk][ty], a1 = As[kk][ty + 16], b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      int m = m0 + ty + 16 * u, n = n0 + tx + 16 * v;
      if (m < M && n < N) {
        float r = acc[u][v] + (bias ? bias[n] : 0.f);
        if (act == 1) r = tanhf(r);
        float *c = C + (int64_t)m * ldc + n;
        *c = accumulate ? *c + r : r;
      }
    }
}

template <typename TB>
void sgemm(int M, int N, int K, const float *A, int64_t sam, int64_t sak, const TB *B, int64_t sbk, int64_t sbn,
           const float *bias, int act, int accumulate, float *C, int64_t ldc, cudaStream_t s) {
  dim3 grid((N + NT - 1) / NT, (M + MT - 1) / MT);
  sgemm_kernel<TB><<<grid, 256, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, bias, act, accumulate, C, ldc);
  count_launches(1);
}

// Y[n][c] = X[n][c] * scale[c] + shift[c]
__global__ void affine_kernel(int n, int cols, const float *X, const float *scale, const float *shift, float *Y) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < (int64_t)n * cols;
       f += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(f % cols);
    Y[f] = X[f] * scale[c] + shift[c];
  }
}

// gather rows: dst[r] = src[idx[r]]
__global__ void gather_rows_kernel(int n, int cols, const int *idx, const float *src, float *dst) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < (int64_t)n * cols;
       f += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(f / cols), c = (int)(f % cols);
    dst[f] = src[(int64_t)idx[r] * cols + c];
  }
}

// mean-squared error against normalised targets: dz = 2 (z - t) / (n * cols),
// loss += sum (z - t)^2 / (n * cols)
__global__ void mse_kernel(int n, int cols, const float *z, const float *t, float *dz, float *loss) {
  __shared__ float red[256];
  float s = 0.f;
  const float inv = 1.f / ((float)n * cols);
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < (int64_t)n * cols;
       f += (int64_t)gridDim.x * blockDim.x) {
    float d = z[f] - t[f];
    dz[f] = 2.f * d * inv;
    s += d * d * inv;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// d[n][c] *= 1 - h[n][c]^2  (tanh derivative through its output)
__global__ void tanh_back_kernel(int64_t n, const float *h, float *d) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x)
    d[f] *= 1.f - h[f] * h[f];
}

// db[c] = sum_n d[n][c]   (one thread per column, fixed order)
__global__ void colsum_kernel(int n, int cols, const float *d, float *db) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < n; ++r) s += d[(int64_t)r * cols + c];
  db[c] = s;
}

// Adam (Kingma & Ba 2015) with bias correction
__global__ void adam_kernel(int64_t n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void to_bf16_kernel(int64_t n, const float *src, __nv_bfloat16 *dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

int gridn(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8));
}

wpcd_status ensure_cap(wpcd_mlp *m, int n) {
  if (n <= m->cap) return WPCD_OK;
  float **bufs[] = {&m->xn, &m->h1, &m->h2, &m->z, &m->dz, &m->d1, &m->d2, &m->tn};
  for (float **b : bufs) {
    dev_free(*b);
    *b = nullptr;
  }
  dev_free(m->idx);
  m->idx = nullptr;
  const int W = m->width;
  WPCD_CUDA_TRY(dev_malloc(&m->xn, sizeof(float) * (size_t)n * m->n_in));
  WPCD_CUDA_TRY(dev_malloc(&m->h1, sizeof(float) * (size_t)n * W));
  WPCD_CUDA_TRY(dev_malloc(&m->h2, sizeof(float) * (size_t)n * W));
  WPCD_CUDA_TRY(dev_malloc(&m->z, sizeof(float) * (size_t)n * m->n_out));
  WPCD_CUDA_TRY(dev_malloc(&m->dz, sizeof(float) * (size_t)n * m->n_out));
  WPCD_CUDA_TRY(dev_malloc(&m->d1, sizeof(float) * (size_t)n * W));
  WPCD_CUDA_TRY(dev_malloc(&m->d2, sizeof(float) * (size_t)n * W));
  WPCD_CUDA_TRY(dev_malloc(&m->tn, sizeof(float) * (size_t)n * m->n_out));
  WPCD_CUDA_TRY(dev_malloc(&m->idx, sizeof(int) * (size_t)n));
  m->cap = n;
  return WPCD_OK;
}

// forward of n rows already normalised in m->xn; output z (normalised)
template <typename TB>
void forward_norm(wpcd_mlp *m, const TB *P, int n, float *z, cudaStream_t s) {
  const int W = m->width;
  sgemm<TB>(n, W, m->n_in, m->xn, m->n_in, 1, P + m->oW1, 1, m->n_in, m->params + m->ob1, 1, 0, m->h1, W, s);
  sgemm<TB>(n, W, W, m->h1, W, 1, P + m->oW2, 1, W, m->params + m->ob2, 1, 0, m->h2, W, s);
  sgemm<TB>(n, m->n_out, W, m->h2, W, 1, P + m->oW3, 1, W, m->params + m->ob3, 0, 0, z, m->n_out, s);
}

// gradients of the loss on (xn, tn) for n rows into m->grads; loss summed into m->loss
void backward(wpcd_mlp *m, int n, cudaStream_t s) {
  const int W = m->width, ni = m->n_in, no = m->n_out;
  float *g = m->grads;
  mse_kernel<<<gridn((int64_t)n * no), 256, 0, s>>>(n, no, m->z, m->tn, m->dz, m->loss);
  count_launches(1);
  // layer 3: dW3[o][i] = sum_n dz[n][o] h2[n][i]; db3; d2 = dz W3
  sgemm<float>(no, W, n, m->dz, 1, no, m->h2, W, 1, nullptr, 0, 0, g + m->oW3, W, s);
  colsum_kernel<<<(no + 127) / 128, 128, 0, s>>>(n, no, m->dz, g + m->ob3);
  sgemm<float>(n, W, no, m->dz, no, 1, m->params + m->oW3, W, 1, nullptr, 0, 0, m->d2, W, s);
  tanh_back_kernel<<<gridn((int64_t)n * W), 256, 0, s>>>((int64_t)n * W, m->h2, m->d2);
  // layer 2
  sgemm<float>(W, W, n, m->d2, 1, W, m->h1, W, 1, nullptr, 0, 0, g + m->oW2, W, s);
  colsum_kernel<<<(W + 127) / 128, 128, 0, s>>>(n, W, m->d2, g + m->ob2);
  sgemm<float>(n, W, W, m->d2, W, 1, m->params + m->oW2, W, 1, nullptr, 0, 0, m->d1, W, s);
  tanh_back_kernel<<<gridn((int64_t)n * W), 256, 0, s>>>((int64_t)n * W, m->h1, m->d1);
  // layer 1
  sgemm<float>(W, ni, n, m->d1, 1, W, m->xn, ni, 1, nullptr, 0, 0, g + m->oW1, ni, s);
  colsum_kernel<<<(W + 127) / 128, 128, 0, s>>>(n, W, m->d1, g + m->ob1);
  count_launches(5);
}

}  // namespace

// ---------------------------------------------------------------------------
// projected-basis helpers (complex FP64 vectors, energy-major [n][dim])
// ---------------------------------------------------------------------------
namespace {

// C[e][j] = <Phi_j, U_e> (conjugate-linear in Phi); one block per (e, j)
__global__ void project_kernel(int dim, int k, const double2 *Phi, const double2 *U, double2 *C) {
  const int e = blockIdx.y, j = blockIdx.x;
  __shared__ double2 red[256];
  double sx = 0.0, sy = 0.0;
  for (int r = threadIdx.x; r < dim; r += 256) {
    double2 a = Phi[(size_t)j * dim + r], b = U[(size_t)e * dim + r];
    sx += a.x * b.x + a.y * b.y;
    sy += a.x * b.y - a.y * b.x;
  }
  red[threadIdx.x] = make_double2(sx, sy);
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x].x += red[threadIdx.x + o].x;
      red[threadIdx.x].y += red[threadIdx.x + o].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) C[(size_t)e * k + j] = red[0];
}

// U[e] = sum_j C[e][j] Phi_j   (C as FP32 (re, im) pairs or FP64 complex)
template <typename TC>
__global__ void expand_kernel(int64_t dim, int k, int n, const double2 *Phi, const TC *C, double2 *U) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < dim * n;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(f / dim);
    const int64_t r = f % dim;
    double ax = 0.0, ay = 0.0;
    for (int j = 0; j < k; ++j) {
      double cr = (double)C[((size_t)e * k + j) * 2], ci = (double)C[((size_t)e * k + j) * 2 + 1];
      double2 p = Phi[(size_t)j * dim + r];
      ax += cr * p.x - ci * p.y;
      ay += cr * p.y + ci * p.x;
    }
    U[f] = make_double2(ax, ay);
  }
}

// v_j -= c v_i   (c device scalar), then norms
__global__ void axpy_one_kernel(int dim, const double2 *c, const double2 *vi, double2 *vj) {
  double2 cc = *c;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < dim; r += gridDim.x * blockDim.x) {
    double2 a = vi[r];
    vj[r].x -= cc.x * a.x - cc.y * a.y;
    vj[r].y -= cc.x * a.y + cc.y * a.x;
  }
}

__global__ void normalize_one_kernel(int dim, const double2 *nrm2, double2 *v) {
  double s = nrm2->x > 0.0 ? 1.0 / sqrt(nrm2->x) : 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < dim; r += gridDim.x * blockDim.x) {
    v[r].x *= s;
    v[r].y *= s;
  }
}

// X[e] = [Ebin_s, Re/Im of Cb[e][0..kf)] as floats (Ebin: centre of the
// on-shell energy bin, the only way E enters G1)
__global__ void features_kernel(int n, int k, int kf, const double *Ebin, double e_lo, double e_hi,
                                const double2 *Cb, float *X) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int cols = 1 + 2 * kf;
  float *x = X + (size_t)e * cols;
  x[0] = (float)((Ebin[e] - e_lo) / (e_hi - e_lo));
  for (int j = 0; j < kf; ++j) {
    double2 c = Cb[(size_t)e * k + j];
    x[1 + 2 * j] = (float)c.x;
    x[2 + 2 * j] = (float)c.y;
  }
}

// y += alpha x  (n reals)
__global__ void axpy_real_kernel(int64_t n, double alpha, const double *x, double *y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(alpha, x[i], y[i]);
}

__global__ void c2f_kernel(int64_t n, const double2 *src, float *dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    dst[2 * i] = (float)src[i].x;
    dst[2 * i + 1] = (float)src[i].y;
  }
}

}  // namespace
}  // namespace wpcd

using namespace wpcd;

extern "C" {

wpcd_status wpcd_mlp_create(int n_in, int width, int n_out, uint64_t seed, int device, wpcd_mlp **out) {
  clear_error();
  if (!out || n_in < 1 || width < 1 || n_out < 1 || n_in > 4096 || width > 4096 || n_out > 4096)
    return set_error(WPCD_EINVAL, "bad MLP sizes");
  *out = nullptr;
  WPCD_CUDA_TRY(cudaSetDevice(device));
  wpcd_mlp *m = new wpcd_mlp();
  m->device = device;
  m->n_in = n_in;
  m->width = width;
  m->n_out = n_out;
  m->oW1 = 0;
  m->ob1 = m->oW1 + (int64_t)width * n_in;
  m->oW2 = m->ob1 + width;
  m->ob2 = m->oW2 + (int64_t)width * width;
  m->oW3 = m->ob2 + width;
  m->ob3 = m->oW3 + (int64_t)n_out * width;
  m->n_params = m->ob3 + n_out;
  // Glorot-uniform weights, zero biases, from a counter-based generator
  std::vector<float> p(m->n_params, 0.f);
  auto fill = [&](int64_t off, int fo, int fi, uint64_t stream_id) {
    double a = std::sqrt(6.0 / (fi + fo));
    for (int64_t i = 0; i < (int64_t)fo * fi; ++i)
      p[off + i] = (float)((2.0 * uniform01(seed + stream_id, (uint64_t)i) - 1.0) * a);
  };
  fill(m->oW1, width, n_in, 1);
  fill(m->oW2, width, width, 2);
  fill(m->oW3, n_out, width, 3);
  const size_t nb = sizeof(float) * m->n_params;
  cudaError_t e;
  if ((e = dev_malloc(&m->params, nb)) != cudaSuccess || (e = dev_malloc(&m->grads, nb)) != cudaSuccess ||
      (e = dev_malloc(&m->adam_m, nb)) != cudaSuccess || (e = dev_malloc(&m->adam_v, nb)) != cudaSuccess ||
      (e = dev_malloc(&m->params_bf16, sizeof(__nv_bfloat16) * m->n_params)) != cudaSuccess ||
      (e = dev_malloc(&m->in_scale, sizeof(float) * n_in)) != cudaSuccess ||
      (e = dev_malloc(&m->in_shift, sizeof(float) * n_in)) != cudaSuccess ||
      (e = dev_malloc(&m->out_scale, sizeof(float) * n_out)) != cudaSuccess ||
      (e = dev_malloc(&m->out_shift, sizeof(float) * n_out)) != cudaSuccess ||
      (e = dev_malloc(&m->loss, sizeof(float))) != cudaSuccess) {
    wpcd_mlp_destroy(m);
    return cuda_error(e, "cudaMalloc (MLP)");
  }
  cudaMemcpy(m->params, p.data(), nb, cudaMemcpyHostToDevice);
  cudaMemset(m->adam_m, 0, nb);
  cudaMemset(m->adam_v, 0, nb);
  std::vector<float> ones(std::max(n_in, n_out), 1.f), zeros(std::max(n_in, n_out), 0.f);
  cudaMemcpy(m->in_scale, ones.data(), sizeof(float) * n_in, cudaMemcpyHostToDevice);
  cudaMemcpy(m->in_shift, zeros.data(), sizeof(float) * n_in, cudaMemcpyHostToDevice);
  cudaMemcpy(m->out_scale, ones.data(), sizeof(float) * n_out, cudaMemcpyHostToDevice);
  cudaMemcpy(m->out_shift, zeros.data(), sizeof(float) * n_out, cudaMemcpyHostToDevice);
  *out = m;
  return WPCD_OK;
}

void wpcd_mlp_destroy(wpcd_mlp *m) {
  if (!m) return;
  cudaSetDevice(m->device);
  void *bufs[] = {m->params, m->grads, m->adam_m, m->adam_v, m->params_bf16, m->in_scale, m->in_shift,
                  m->out_scale, m->out_shift, m->xn, m->h1, m->h2, m->z, m->dz, m->d1, m->d2,
                  m->loss, m->tn, m->idx};
  for (void *b : bufs) dev_free(b);
  delete m;
}

wpcd_status wpcd_mlp_info(const wpcd_mlp *m, int64_t *n_params, int *n_in, int *width, int *n_out) {
  if (!m) return set_error(WPCD_EINVAL, "null MLP");
  if (n_params) *n_params = m->n_params;
  if (n_in) *n_in = m->n_in;
  if (width) *width = m->width;
  if (n_out) *n_out = m->n_out;
  return WPCD_OK;
}

wpcd_status wpcd_mlp_params(wpcd_mlp *m, float *get, const float *set) {
  clear_error();
  if (!m) return set_error(WPCD_EINVAL, "null MLP");
  WPCD_CUDA_TRY(cudaSetDevice(m->device));
  const size_t nb = sizeof(float) * m->n_params;
  if (get) WPCD_CUDA_TRY(cudaMemcpy(get, m->params, nb, cudaMemcpyDefault));
  if (set) {
    WPCD_CUDA_TRY(cudaMemcpy(m->params, set, nb, cudaMemcpyDefault));
    m->bf16_stale = true;
  }
  return WPCD_OK;
}

wpcd_status wpcd_mlp_set_affine(wpcd_mlp *m, const float *in_scale, const float *in_shift, const float *out_scale,
                                const float *out_shift) {
  clear_error();
  if (!m) return set_error(WPCD_EINVAL, "null MLP");
  WPCD_CUDA_TRY(cudaSetDevice(m->device));
  if (in_scale) WPCD_CUDA_TRY(cudaMemcpy(m->in_scale, in_scale, sizeof(float) * m->n_in, cudaMemcpyDefault));
  if (in_shift) WPCD_CUDA_TRY(cudaMemcpy(m->in_shift, in_shift, sizeof(float) * m->n_in, cudaMemcpyDefault));
  if (out_scale) WPCD_CUDA_TRY(cudaMemcpy(m->out_scale, out_scale, sizeof(float) * m->n_out, cudaMemcpyDefault));
  if (out_shift) WPCD_CUDA_TRY(cudaMemcpy(m->out_shift, out_shift, sizeof(float) * m->n_out, cudaMemcpyDefault));
  return WPCD_OK;
}

wpcd_status wpcd_mlp_forward(wpcd_mlp *m, const float *X, int n, float *Y, int bf16, void *stream) {
  clear_error();
  if (!m || !X || !Y || n < 1) return set_error(WPCD_EINVAL, "bad MLP forward arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  WPCD_CUDA_TRY(cudaSetDevice(m->device));
  wpcd_status st = ensure_cap(m, n);
  if (st != WPCD_OK) return st;
  affine_kernel<<<gridn((int64_t)n * m->n_in), 256, 0, s>>>(n, m->n_in, X, m->in_scale, m->in_shift, m->xn);
  count_launches(1);
  if (bf16) {
    if (m->bf16_stale) {
      to_bf16_kernel<<<gridn(m->n_params), 256, 0, s>>>(m->n_params, m->params, m->params_bf16);
      count_launches(1);
      m->bf16_stale = false;
    }
    forward_norm<__nv_bfloat16>(m, m->params_bf16, n, m->z, s);
  } else {
    forward_norm<float>(m, m->params, n, m->z, s);
  }
  // Y = z * out_scale + out_shift
  affine_kernel<<<gridn((int64_t)n * m->n_out), 256, 0, s>>>(n, m->n_out, m->z, m->out_scale, m->out_shift, Y);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "MLP forward");
}

// loss (host, mean squared error of the normalised outputs) and gradient
// (device [n_params], may be NULL) on n rows of (X, T)
wpcd_status wpcd_mlp_loss_grad(wpcd_mlp *m, const float *X, const float *T, int n, float *loss, float *grad,
                               void *stream) {
  clear_error();
  if (!m || !X || !T || n < 1) return set_error(WPCD_EINVAL, "bad MLP arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  WPCD_CUDA_TRY(cudaSetDevice(m->device));
  wpcd_status st = ensure_cap(m, n);
  if (st != WPCD_OK) return st;
  affine_kernel<<<gridn((int64_t)n * m->n_in), 256, 0, s>>>(n, m->n_in, X, m->in_scale, m->in_shift, m->xn);
  // normalised targets: (T - out_shift) / out_scale
  std::vector<float> sc(m->n_out), sh(m->n_out);
  WPCD_CUDA_TRY(cudaMemcpy(sc.data(), m->out_scale, sizeof(float) * m->n_out, cudaMemcpyDeviceToHost));
  WPCD_CUDA_TRY(cudaMemcpy(sh.data(), m->out_shift, sizeof(float) * m->n_out, cudaMemcpyDeviceToHost));
  std::vector<float> isc(m->n_out), ish(m->n_out);
  for (int c = 0; c < m->n_out; ++c) {
    isc[c] = 1.f / sc[c];
    ish[c] = -sh[c] / sc[c];
  }
  float *d_isc = nullptr;
  WPCD_CUDA_TRY(dev_malloc(&d_isc, sizeof(float) * 2 * m->n_out));
  cudaMemcpy(d_isc, isc.data(), sizeof(float) * m->n_out, cudaMemcpyHostToDevice);
  cudaMemcpy(d_isc + m->n_out, ish.data(), sizeof(float) * m->n_out, cudaMemcpyHostToDevice);
  affine_kernel<<<gridn((int64_t)n * m->n_out), 256, 0, s>>>(n, m->n_out, T, d_isc, d_isc + m->n_out, m->tn);
  count_launches(2);
  forward_norm<float>(m, m->params, n, m->z, s);
  cudaMemsetAsync(m->loss, 0, sizeof(float), s);
  backward(m, n, s);
  float l = 0.f;
  cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
  if (grad) cudaMemcpyAsync(grad, m->grads, sizeof(float) * m->n_params, cudaMemcpyDefault, s);
  cudaError_t e = cudaStreamSynchronize(s);
  dev_free(d_isc);
  if (e != cudaSuccess) return cuda_error(e, "MLP loss/grad");
  if (loss) *loss = l;
  return WPCD_OK;
}

// Minibatch Adam on n rows of (X, T) (device FP32; T in output units, the
// MLP's output affine map defines the normalisation).  Epoch shuffles come
// from a counter-based generator seeded by `seed`.  loss_hist: host [epochs]
// mean loss per epoch (may be NULL).
wpcd_status wpcd_mlp_train(wpcd_mlp *m, const float *X, const float *T, int n, int epochs, int batch, float lr,
                           uint64_t seed, float *loss_hist, void *stream) {
  clear_error();
  if (!m || !X || !T || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.f))
    return set_error(WPCD_EINVAL, "bad MLP training arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  WPCD_CUDA_TRY(cudaSetDevice(m->device));
  batch = std::min(batch, n);
  wpcd_status st = ensure_cap(m, batch);
  if (st != WPCD_OK) return st;
  float *Xb = nullptr, *Tb = nullptr, *d_isc = nullptr;
  int *d_order = nullptr;
  WPCD_CUDA_TRY(dev_malloc(&d_order, sizeof(int) * (size_t)n));
  WPCD_CUDA_TRY(dev_malloc(&Xb, sizeof(float) * (size_t)batch * m->n_in));
  WPCD_CUDA_TRY(dev_malloc(&Tb, sizeof(float) * (size_t)batch * m->n_out));
  WPCD_CUDA_TRY(dev_malloc(&d_isc, sizeof(float) * 2 * m->n_out));
  std::vector<float> sc(m->n_out), sh(m->n_out), isc(2 * m->n_out);
  cudaMemcpy(sc.data(), m->out_scale, sizeof(float) * m->n_out, cudaMemcpyDeviceToHost);
  cudaMemcpy(sh.data(), m->out_shift, sizeof(float) * m->n_out, cudaMemcpyDeviceToHost);
  for (int c = 0; c < m->n_out; ++c) {
    isc[c] = 1.f / sc[c];
    isc[m->n_out + c] = -sh[c] / sc[c];
  }
  cudaMemcpy(d_isc, isc.data(), sizeof(float) * 2 * m->n_out, cudaMemcpyHostToDevice);
  std::vector<int> order(n);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int ep = 0; ep < epochs; ++ep) {
    std::iota(order.begin(), order.end(), 0);
    for (int i = n - 1; i > 0; --i) {  // Fisher-Yates with the counter-based generator
      int j = (int)(uniform01(seed, (uint64_t)ep * n + i) * (i + 1));
      std::swap(order[i], order[std::min(j, i)]);
    }
    // the epoch's order goes up once (synchronously: the host vector is reused)
    WPCD_CUDA_TRY(cudaMemcpy(d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    cudaMemsetAsync(m->loss, 0, sizeof(float), s);
    int nb = 0;
    for (int b0 = 0; b0 + batch <= n; b0 += batch, ++nb) {
      gather_rows_kernel<<<gridn((int64_t)batch * m->n_in), 256, 0, s>>>(batch, m->n_in, d_order + b0, X, Xb);
      gather_rows_kernel<<<gridn((int64_t)batch * m->n_out), 256, 0, s>>>(batch, m->n_out, d_order + b0, T, Tb);
      affine_kernel<<<gridn((int64_t)batch * m->n_in), 256, 0, s>>>(batch, m->n_in, Xb, m->in_scale, m->in_shift, m->xn);
      affine_kernel<<<gridn((int64_t)batch * m->n_out), 256, 0, s>>>(batch, m->n_out, Tb, d_isc, d_isc + m->n_out, m->tn);
      count_launches(4);
      forward_norm<float>(m, m->params, batch, m->z, s);
      backward(m, batch, s);
      ++m->adam_t;
      float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
      adam_kernel<<<gridn(m->n_params), 256, 0, s>>>(m->n_params, m->params, m->grads, m->adam_m, m->adam_v, lr, b1,
                                                   b2, eps, c1, c2);
      count_launches(1);
    }
    if (loss_hist) {
      float l = 0.f;
      cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      loss_hist[ep] = nb > 0 ? l / nb : 0.f;
    }
  }
  m->bf16_stale = true;
  cudaError_t e = cudaStreamSynchronize(s);
  dev_free(Xb);
  dev_free(Tb);
  dev_free(d_isc);
  dev_free(d_order);
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "MLP training");
}

// C[e][j] = <Phi_j, U_e> for e < n, j < k (device FP64 complex)
wpcd_status wpcd_basis_project(const double *Phi, int k, int dim, const double *U, int n, double *C, void *stream) {
  clear_error();
  if (!Phi || !U || !C || k < 1 || dim < 1 || n < 1) return set_error(WPCD_EINVAL, "bad projection arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  project_kernel<<<dim3(k, n), 256, 0, s>>>(dim, k, (const double2 *)Phi, (const double2 *)U, (double2 *)C);
  count_launches(1);
  cudaError_t e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "basis projection");
}

// U[e] = sum_j C[e][j] Phi_j ; C given as FP32 (re, im) pairs [n][k][2]
wpcd_status wpcd_basis_expand(const double *Phi, int k, int dim, const float *C, int n, double *U, void *stream) {
  clear_error();
  if (!Phi || !U || !C || k < 1 || dim < 1 || n < 1) return set_error(WPCD_EINVAL, "bad expansion arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  expand_kernel<float><<<gridn((int64_t)dim * n), 256, 0, s>>>(dim, k, n, (const double2 *)Phi, C, (double2 *)U);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "basis expansion");
}

// Orthonormalise k vectors in place (two passes of modified Gram-Schmidt)
wpcd_status wpcd_basis_orthonormalize(double *Phi, int k, int dim, void *stream) {
  clear_error();
  if (!Phi || k < 1 || dim < 1) return set_error(WPCD_EINVAL, "bad basis arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double2 *c = nullptr;
  WPCD_CUDA_TRY(dev_malloc(&c, sizeof(double2)));
  double2 *V = (double2 *)Phi;
  for (int j = 0; j < k; ++j) {
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i < j; ++i) {
        project_kernel<<<dim3(1, 1), 256, 0, s>>>(dim, 1, V + (size_t)i * dim, V + (size_t)j * dim, c);
        axpy_one_kernel<<<gridn(dim), 256, 0, s>>>(dim, c, V + (size_t)i * dim, V + (size_t)j * dim);
        count_launches(2);
      }
    project_kernel<<<dim3(1, 1), 256, 0, s>>>(dim, 1, V + (size_t)j * dim, V + (size_t)j * dim, c);
    normalize_one_kernel<<<gridn(dim), 256, 0, s>>>(dim, c, V + (size_t)j * dim);
    count_launches(2);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  dev_free(c);
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "orthonormalisation");
}

// Features of the warm-start network: X[e] = [(Ebin - e_lo) / (e_hi - e_lo),
// Re/Im of the first kf coefficients Cb[e][0..kf) of the Born term in the
// basis] as FP32 (device); Ebin = centre of E's on-shell energy bin.
wpcd_status wpcd_warm_features(const wpcd_problem *pr, const double *E, int n, double e_lo, double e_hi,
                               const double *Cb, int k, int kf, float *X, void *stream) {
  clear_error();
  if (!pr || !E || !Cb || !X || n < 1 || kf < 0 || kf > k || !(e_hi > e_lo))
    return set_error(WPCD_EINVAL, "bad feature arguments");
  std::vector<double> eb(n);
  for (int i = 0; i < n; ++i) {
    int j0;
    double lo, hi;
    wpcd_status st = onshell(pr, E[i], &j0, &lo, &hi, nullptr);
    if (st != WPCD_OK) return st;
    eb[i] = 0.5 * (lo + hi);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *d_eb = nullptr;
  WPCD_CUDA_TRY(dev_malloc(&d_eb, sizeof(double) * n));
  WPCD_CUDA_TRY(cudaMemcpy(d_eb, eb.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
  features_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, k, kf, d_eb, e_lo, e_hi, (const double2 *)Cb, X);
  count_launches(1);
  cudaError_t e = cudaStreamSynchronize(s);
  dev_free(d_eb);
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "features");
}

// y += alpha x over n reals (device FP64), e.g. u - u0 or u0 + Phi c
wpcd_status wpcd_vec_axpy(double alpha, const double *x, double *y, int64_t n, void *stream) {
  clear_error();
  if (!x || !y || n < 0) return set_error(WPCD_EINVAL, "bad axpy arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n > 0) {
    axpy_real_kernel<<<gridn(n), 256, 0, s>>>(n, alpha, x, y);
    count_launches(1);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "axpy");
}

// softmax of each row of k logits (one warp per row; k <= 1024), written as
// (w, 0) complex pairs
__global__ void softmax_rows_kernel(int n, int k, const float *__restrict__ z, float2 *__restrict__ C) {
  const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;  // uniform over the warp
  const float *zr = z + (int64_t)row * k;
  float mx = -INFINITY;
  for (int j = lane; j < k; j += 32) mx = fmaxf(mx, zr[j]);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float sum = 0.f;
  for (int j = lane; j < k; j += 32) sum += expf(zr[j] - mx);
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  const float inv = 1.f / sum;
  for (int j = lane; j < k; j += 32) C[(int64_t)row * k + j] = make_float2(expf(zr[j] - mx) * inv, 0.f);
}

// FP64 complex -> FP32 (re, im) pairs (device), e.g. projection
// coefficients as training targets
wpcd_status wpcd_complex_to_f32(const double *src, int64_t n, float *dst, void *stream) {
  clear_error();
  if (!src || !dst || n < 0) return set_error(WPCD_EINVAL, "bad conversion arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n > 0) {
    c2f_kernel<<<gridn(n), 256, 0, s>>>(n, (const double2 *)src, dst);
    count_launches(1);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "conversion");
}

wpcd_status wpcd_warm_softmax(const float *logits, int n, int k, float *C, void *stream) {
  clear_error();
  if (!logits || !C || n < 1 || k < 1 || k > 1024) return set_error(WPCD_EINVAL, "bad softmax arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  softmax_rows_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(n, k, logits, reinterpret_cast<float2 *>(C));
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "softmax");
}

}  // extern "C"
