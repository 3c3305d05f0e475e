// FP64-class channel-block products on the tensor cores, for the float-float
// refinement residual and Born term of the mixed solve (Sec. 3.3, Eq.
// kernel):  C = A B for every channel block, A = Vt_ch or O_ch (N x N, FP64),
// B the float-float panel (hi + lo floats, [n_ch][N][ncol]), C in FP64 or
// float-float.
//
// Error-free splitting into digit planes (the scheme of Ozaki, Ogita, Oishi
// and Rump, Numer. Algorithms 59, 2012, with low-precision digits on tensor
// cores as in Mukunoki, Ozaki, Ogita and Imamura, ICCS 2020):
//   a_ik = 2^E_i  sum_s alpha_s(i,k) 2^(-7 (s + 1))     row exponent E_i
//   b_kj = 2^F_j  sum_t beta_t(k,j)  2^(-7 (t + 1))     column exponent F_j
// with integer digits, |alpha_0|, |beta_0| <= 128 and the later digits
// <= 64 (round-to-nearest extraction), OZ_L = 8 planes (56 bits, beyond the
// 48 of a float-float operand).  Every digit is exact in bf16, every digit
// product exact in FP32, and the products of one diagonal d = s + t summed
// over K stay integers below 2^24 for K <= 409 (diagonal d holds at most
// two products of bound 2^13 and d - 1 of bound 2^12), so the FP32 tensor
// accumulation of a diagonal is exact.  The 36 pairs with s + t < OZ_L run
// as kind::f16 (bf16) MMAs into OZ_L diagonal accumulators in TMEM (one
// MMA per A plane s, its N spanning the B planes 0 .. OZ_L - 1 - s); the
// epilogue forms C = 2^(E_i + F_j - 14) sum_d 2^(-7 d) acc_d in float-float
// on the FP32 pipe (GB300 runs FP64 at 1/64 of that rate).  The
// pairs left out (s + t >= OZ_L) and the digits beyond plane 7 weigh below
// 2^-56 of 2^(E_i + F_j) per term.
//
// One CTA per SM walks the (channel, 32-column) output tiles.  Per K chunk
// of 16: the packed A digits of all row tiles (RT x OZ_L blocks of 128 x 16
// bf16, packed once per problem) arrive by a bulk async copy; the threads
// turn the chunk's B values into OZ_L digit blocks of 32 x 16 bf16; one
// thread issues the 8 RT MMAs and commits them to the stage's mbarrier.
// Shared-memory operands use the no-swizzle K-major layout: 8-row groups of
// 256 B, each two 8 x 16 B core matrices along K (K-core stride 128 B,
// row-group stride 256 B).  Every wait is bounded; a wait that runs out sets
// the error word, and the kernel waits (bounded) for its copies and MMAs
// before it frees TMEM and returns.  N <= 256 (two row tiles): larger
// problems keep the float-float SIMT products.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tc_ptx.cuh"
#include "wpcd_internal.h"

namespace wpcd {
namespace {

constexpr int OZ_L = 8;          // digit planes
constexpr int OZ_M = 128;        // rows per MMA (TMEM lanes)
constexpr int OZ_KC = 16;        // K per stage: one kind::f16 MMA step
constexpr int OZ_BN = 32;        // output columns per tile
constexpr int OZ_THREADS = 256;
constexpr int OZ_STAGES = 3;
constexpr int OZ_MAX_RT = 2;
constexpr uint32_t OZ_A_PLANE = OZ_M * OZ_KC * 2;   // 4 KB: one digit plane of one row tile
constexpr uint32_t OZ_B_PLANE = OZ_BN * OZ_KC * 2;  // 1 KB
constexpr uint32_t OZ_TMEM_COLS = 512;              // OZ_MAX_RT * OZ_L * OZ_BN

struct OzParams {
  int n, RT, nK, n_cb, n_tiles;
  int64_t ncol;
  uint32_t stage_bytes;
  const uint16_t *A;      // digit blocks [n_ch][nK][RT][OZ_L][128 x 16 bf16]
  const int *EA;          // row exponents [n_ch][RT * 128]
  const int *FB;          // column exponents [n_ch][ncol]
  const float *Bh, *Bl;   // panel [n_ch][n][ncol]
  double *C;              // FP64 output, or
  float *Ch, *Cl;         // float-float output
  int *err;
  int expire_first;       // nonzero: thread 0's first copy wait runs out at once
};

// byte offset of element (row r, k) in a [rows / 8][2][8][8] bf16 block
__host__ __device__ __forceinline__ uint32_t oz_off(int r, int k) {
  return (uint32_t)((r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor of that layout: start, K-core stride 128 B
// (leading byte offset), row-group stride 256 B (stride byte offset),
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t oz_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: D F32, A and B bf16, both K-major,
// N columns (a multiple of 16, at most 256), M = 128
__host__ __device__ constexpr uint32_t oz_idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(OZ_M >> 4) << 24);
}

__device__ __forceinline__ void oz_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// bf16 bits of an integer-valued float of at most 8 significant bits (exact)
__host__ __device__ __forceinline__ uint16_t oz_bf16_bits(float d) {
#ifdef __CUDA_ARCH__
  return (uint16_t)(__float_as_uint(d) >> 16);
#else
  uint32_t u;
  std::memcpy(&u, &d, 4);
  return (uint16_t)(u >> 16);
#endif
}

// the OZ_L digits of the float-float value (h + l) 2^-F: v <- 128 v, digit =
// nearest integer of the high part, the high part keeps the (exact)
// remainder and (high, low) are renormalised by TwoSum, so the value is
// carried without error from plane to plane
__device__ __forceinline__ void oz_digits(float h, float l, int F, float (&d)[OZ_L]) {
  float vh = ldexpf(h, -F), vl = ldexpf(l, -F);
#pragma unroll
  for (int t = 0; t < OZ_L; ++t) {
    vh *= 128.f;
    vl *= 128.f;
    const float q = rintf(vh);
    vh -= q;
    const float s = __fadd_rn(vh, vl);
    const float bb = __fsub_rn(s, vh);
    const float e = __fadd_rn(__fsub_rn(vh, __fsub_rn(s, bb)), __fsub_rn(vl, bb));
    vh = s;
    vl = e;
    d[t] = q;
  }
}

// F_j with max_k |B_h(k, j)| < 2^F_j (0 for a zero column), per channel and
// column of the panel
__global__ void oz_colexp_kernel(int n_ch, int n, int64_t ncol, const float *__restrict__ Bh, int *__restrict__ F) {
  const int64_t total = (int64_t)n_ch * ncol;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total; f += (int64_t)gridDim.x * blockDim.x) {
    const int ch = (int)(f / ncol);
    const int64_t j = f % ncol;
    const float *col = Bh + (size_t)ch * n * ncol + j;
    float m = 0.f;
#pragma unroll 4
    for (int k = 0; k < n; ++k) m = fmaxf(m, fabsf(col[(size_t)k * ncol]));
    int e = 0;
    if (m > 0.f) frexpf(m, &e);
    F[f] = e;
  }
}

// C = A B (FP64 or float-float out) for the (channel, 32-column) tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...
template <bool OUT_DF>
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_gemm_kernel(OzParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_a[OZ_STAGES], bar_mma[OZ_STAGES], bar_done;
  __shared__ uint32_t tmem_holder;
  __shared__ int s_F[OZ_BN];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = p.n, RT = p.RT, nK = p.nK;
  const int64_t ncol = p.ncol;
  if (tid == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(&bar_a[s], 1);
      mbar_init(&bar_mma[s], 1);
    }
    mbar_init(&bar_done, 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_holder;
  const uint32_t a_bytes = (uint32_t)RT * OZ_L * OZ_A_PLANE;
  bool ok = true, bail = false;
  uint32_t g = 0;                      // chunks begun by this CTA (stage ring position)
  uint32_t g_issued = 0, g_seen = 0;   // thread 0: A copies issued / seen complete
  uint32_t tl = 0;                     // tiles finished (bar_done phase)
  WaitLimit lim(tid == 0 && p.expire_first != 0);
  // chunk c of a tile: thread (j, kp) converts rows 2 kp, 2 kp + 1 of column j
  const int j = tid & 31, kp = tid >> 5;
  // the CTA's chunks in order: chunk q is K chunk q % nK of its tile q / nK;
  // thread 0 copies the A digits two chunks ahead of the MMAs
  const int my_tiles = blockIdx.x < p.n_tiles ? (p.n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const uint32_t G = (uint32_t)my_tiles * nK;
  auto issue_a = [&](uint32_t q) {
    const int tq = blockIdx.x + (int)(q / nK) * gridDim.x;
    const int sq = (int)(q % OZ_STAGES);
    const uint16_t *src = p.A + ((size_t)(tq / p.n_cb) * nK + q % nK) * (a_bytes / 2);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar_a[sq])), "r"(a_bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(smem + (size_t)sq * p.stage_bytes)),
                 "l"(src), "r"(a_bytes), "r"(smem_u32(&bar_a[sq]))
                 : "memory");
    ++g_issued;
  };
  if (tid == 0)
    for (uint32_t q = 0; q < 2 && q < G; ++q) issue_a(q);
  for (int t = blockIdx.x; t < p.n_tiles; t += gridDim.x, ++tl) {
    const int ch = t / p.n_cb;
    const int64_t col0 = (int64_t)(t % p.n_cb) * OZ_BN;
    const int64_t col = col0 + j;
    const bool col_in = col < ncol;
    const float *Bh = p.Bh + (size_t)ch * n * ncol + (col_in ? col : 0);
    const float *Bl = p.Bl + (size_t)ch * n * ncol + (col_in ? col : 0);
    if (tid < OZ_BN) s_F[tid] = col_in ? p.FB[(size_t)ch * ncol + col] : 0;
    // also orders this tile's MMAs after the previous tile's TMEM reads
    __syncthreads();
    const int F = s_F[j];
    float hv[2], lv[2];  // the raw values of the chunk being converted
    auto load = [&](int c, float (&h)[2], float (&l)[2]) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int k = c * OZ_KC + 2 * kp + q;
        const bool in = col_in && k < n;
        h[q] = in ? Bh[(size_t)k * ncol] : 0.f;
        l[q] = in ? Bl[(size_t)k * ncol] : 0.f;
      }
    };
    load(0, hv, lv);
    for (int c = 0; c < nK; ++c, ++g) {
      const int s = (int)(g % OZ_STAGES);
      const uint32_t use = g / OZ_STAGES;
      unsigned char *st = smem + (size_t)s * p.stage_bytes;
      // the MMAs of chunk g - OZ_STAGES read this stage
      if (g >= OZ_STAGES && ok) ok = mbar_wait(&bar_mma[s], (use - 1) & 1);
      float hn[2], ln[2];
      if (c + 1 < nK) load(c + 1, hn, ln);
      // B digits: plane t of (j, 2 kp .. 2 kp + 1) as one 32-bit store
      unsigned char *bst = st + a_bytes;
      float d0[OZ_L], d1[OZ_L];
      oz_digits(hv[0], lv[0], F, d0);
      oz_digits(hv[1], lv[1], F, d1);
#pragma unroll
      for (int q = 0; q < OZ_L; ++q)
        *reinterpret_cast<uint32_t *>(bst + q * OZ_B_PLANE + oz_off(j, 2 * kp)) =
            (uint32_t)oz_bf16_bits(d0[q]) | ((uint32_t)oz_bf16_bits(d1[q]) << 16);
      if (c + 1 < nK)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          hv[q] = hn[q];
          lv[q] = ln[q];
        }
      // the A copy of chunk g + 2 into the stage that chunk g - 1 frees
      if (tid == 0 && ok && g + 2 < G) {
        if (g >= 1) ok = mbar_wait(&bar_mma[(g - 1) % OZ_STAGES], ((g - 1) / OZ_STAGES) & 1);
        if (ok) issue_a(g + 2);
      }
      // generic-proxy stores -> visible to the tensor core (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      bail = __syncthreads_or(!ok) != 0;
      if (bail) break;
      if (tid == 0) {
        tc_fence_after();
        ok = mbar_wait(&bar_a[s], use & 1, lim.next());
        if (ok) {
          g_seen = g + 1;
          // descriptors of the plane blocks: the start address field is
          // addr / 16, so a block offset adds offset / 16 (smem < 256 KB)
          const uint64_t da = oz_desc(smem_u32(st)), db = oz_desc(smem_u32(bst));
          // A plane sa against B planes 0 .. OZ_L - 1 - sa in one MMA: the B
          // planes are consecutive 32-row groups of one K-major operand and
          // the diagonal accumulators sa .. OZ_L - 1 consecutive 32-column
          // groups of TMEM, so N = 32 (OZ_L - sa) and the A block is read
          // once per plane
#pragma unroll 1
          for (int rt = 0; rt < RT; ++rt)
#pragma unroll
            for (int sa = 0; sa < OZ_L; ++sa)
              oz_mma(tmem + (uint32_t)((rt * OZ_L + sa) * OZ_BN), da + (uint64_t)((rt * OZ_L + sa) * (OZ_A_PLANE >> 4)),
                     db, oz_idesc(OZ_BN * (OZ_L - sa)), (c > 0 || sa > 0) ? 1u : 0u);
        }
        tc_commit(&bar_mma[s]);
      }
    }
    if (bail) break;
    if (tid == 0) tc_commit(&bar_done);
    const bool done = mbar_wait(&bar_done, tl & 1);
    ok = ok && done;
    tc_fence_after();
    bail = __syncthreads_or(!ok) != 0;
    if (bail) break;
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, columns 16 (w / 4) .. + 15
    const int lg = warp & 3, half = warp >> 2;
    for (int rt = 0; rt < RT; ++rt) {
      const int row = rt * OZ_M + lg * 32 + lane;
      // sum_d 2^(-7 d) acc_d in float-float (TwoSum; the acc_d are exact
      // integers below 2^24 and their power-of-two scaling is exact), on the
      // FP32 pipe: GB300's FP64 rate is 1/64 of it
      float xh[16], xl[16];
#pragma unroll
      for (int d = 0; d < OZ_L; ++d) {
        float v[16];
        tc_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)((rt * OZ_L + d) * OZ_BN + half * 16), v);
        const float w = __int_as_float((127 - 7 * d) << 23);  // 2^(-7 d)
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (d == 0) {
            xh[i] = v[i];
            xl[i] = 0.f;
          } else {
            const float x = v[i] * w;
            const float sum = __fadd_rn(xh[i], x);
            const float bb = __fsub_rn(sum, xh[i]);
            const float e = __fadd_rn(__fsub_rn(xh[i], __fsub_rn(sum, bb)), __fsub_rn(x, bb));
            xh[i] = sum;
            xl[i] = __fadd_rn(xl[i], e);
          }
        }
      }
      if (row < n) {
        const int E = p.EA[((size_t)ch * RT) * OZ_M + row];
        const size_t o = ((size_t)ch * n + row) * ncol + col0 + half * 16;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (col0 + half * 16 + i >= ncol) break;
          const int k = E + s_F[half * 16 + i] - 14;  // scale 2^k
          const float h = xh[i] + xl[i], l = xl[i] - (h - xh[i]);  // renormalised (Fast2Sum)
          if (OUT_DF) {
            // two float powers of two (a float-float result lies in the
            // float range, so each half exponent stays within it)
            const int k1 = min(max(k / 2, -126), 127), k2 = min(max(k - k / 2, -126), 127);
            const float s1 = __int_as_float((127 + k1) << 23), s2 = __int_as_float((127 + k2) << 23);
            p.Ch[o + i] = h * s1 * s2;
            p.Cl[o + i] = l * s1 * s2;
          } else {
            p.C[o + i] = ((double)h + (double)l) * __longlong_as_double((long long)(1023 + k) << 52);
          }
        }
      }
    }
    // TMEM reads and s_F uses of this tile done before the next tile's
    // exponents and MMAs
    tc_fence_before();
    __syncthreads();
  }
  if (bail && tid == 0) {
    // after a wait ran out: still wait (bounded) for the copies issued and
    // the MMAs committed, so that nothing lands after the CTA has gone
    for (uint32_t q = g_seen; q < g_issued; ++q) mbar_wait(&bar_a[q % OZ_STAGES], (q / OZ_STAGES) & 1);
    tc_commit(&bar_done);
    mbar_wait(&bar_done, tl & 1);
    atomicOr(p.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  }
}

int g_oz_sms[64];
bool g_oz_attr[64];

}  // namespace

std::atomic<int> g_oz_expire_first{0};

bool oz_supported(const wpcd_problem *pr) { return pr->N >= 1 && pr->N <= OZ_MAX_RT * OZ_M; }

// the refinement products run on the tensor cores (digit planes) when N <=
// 256, unless WPCD_RESIDUAL_GEMM=ff selects the float-float SIMT kernels
bool oz_enabled() {
  const char *v = std::getenv("WPCD_RESIDUAL_GEMM");
  return !(v && std::strcmp(v, "ff") == 0);
}

// digit planes and row exponents of O and Vt, packed once per problem (host
// arithmetic in FP64, the same extraction as oz_digits)
wpcd_status oz_prepare(wpcd_problem *pr, cudaStream_t s) {
  if (pr->d.O_oz) return WPCD_OK;
  if (!oz_supported(pr)) return set_error(WPCD_EINVAL, "the digit-plane tensor-core GEMM needs N <= 256");
  const int N = pr->N, n_ch = pr->n_ch;
  const int RT = (N + OZ_M - 1) / OZ_M, nK = (N + OZ_KC - 1) / OZ_KC;
  const size_t plane = OZ_A_PLANE / 2;  // uint16 per (row tile, plane) block
  const size_t per_ch = (size_t)nK * RT * OZ_L * plane;
  std::vector<uint16_t> dig(per_ch * n_ch);
  std::vector<int> ex((size_t)n_ch * RT * OZ_M);
  uint16_t *out[2] = {nullptr, nullptr};
  int *outE[2] = {nullptr, nullptr};
  for (int which = 0; which < 2; ++which) {
    const std::vector<double> &A = which == 0 ? pr->O : pr->Vt;
    std::fill(dig.begin(), dig.end(), (uint16_t)0);
    std::fill(ex.begin(), ex.end(), 0);
    for (int ch = 0; ch < n_ch; ++ch)
      for (int i = 0; i < N; ++i) {
        const double *row = A.data() + ((size_t)ch * N + i) * N;
        double m = 0.0;
        for (int k = 0; k < N; ++k) m = std::max(m, std::fabs(row[k]));
        int E = 0;
        if (m > 0.0) std::frexp(m, &E);
        ex[(size_t)ch * RT * OZ_M + i] = E;
        const int rt = i / OZ_M, r = i % OZ_M;
        for (int k = 0; k < N; ++k) {
          double v = std::ldexp(row[k], -E);
          const int c = k / OZ_KC, kk = k % OZ_KC;
          for (int t = 0; t < OZ_L; ++t) {
            v *= 128.0;
            const double q = std::nearbyint(v);
            v -= q;
            uint16_t *blk = dig.data() + (size_t)ch * per_ch + (((size_t)c * RT + rt) * OZ_L + t) * plane;
            blk[oz_off(r, kk) / 2] = oz_bf16_bits((float)q);
          }
        }
      }
    WPCD_CUDA_TRY(dev_malloc(&out[which], sizeof(uint16_t) * dig.size()));
    WPCD_CUDA_TRY(dev_malloc(&outE[which], sizeof(int) * ex.size()));
    WPCD_CUDA_TRY(cudaMemcpyAsync(out[which], dig.data(), sizeof(uint16_t) * dig.size(), cudaMemcpyHostToDevice, s));
    WPCD_CUDA_TRY(cudaMemcpyAsync(outE[which], ex.data(), sizeof(int) * ex.size(), cudaMemcpyHostToDevice, s));
    WPCD_CUDA_TRY(cudaStreamSynchronize(s));  // host staging reused / freed
  }
  pr->d.O_oz = out[0];
  pr->d.Vt_oz = out[1];
  pr->d.O_ozE = outE[0];
  pr->d.Vt_ozE = outE[1];
  if (!pr->d.tc_err) {
    WPCD_CUDA_TRY(dev_malloc(&pr->d.tc_err, sizeof(int)));
    WPCD_CUDA_TRY(cudaMemsetAsync(pr->d.tc_err, 0, sizeof(int), s));
  }
  if (pr->device < 0 || pr->device >= 64) return set_error(WPCD_EINVAL, "device ordinal out of range");
  if (!g_oz_attr[pr->device]) {
    const int bytes = OZ_STAGES * (int)(OZ_MAX_RT * OZ_L * OZ_A_PLANE + OZ_L * OZ_B_PLANE);
    WPCD_CUDA_TRY(cudaFuncSetAttribute(oz_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    WPCD_CUDA_TRY(cudaFuncSetAttribute(oz_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    WPCD_CUDA_TRY(cudaDeviceGetAttribute(&g_oz_sms[pr->device], cudaDevAttrMultiProcessorCount, pr->device));
    g_oz_attr[pr->device] = true;
  }
  return WPCD_OK;
}

// C = A B for every channel block (A = O or Vt), B the float-float panel
// [n_ch][N][ncol]; C FP64 (C) or float-float (Ch, Cl)
wpcd_status oz_gemm(const wpcd_problem *pr, bool use_O, const float *Bh, const float *Bl, double *C, float *Ch,
                    float *Cl, int64_t ncol, cudaStream_t s) {
  if (!pr->d.O_oz) return set_error(WPCD_EINVAL, "digit-plane operands not prepared");
  if (ncol < 1) return set_error(WPCD_EINVAL, "empty panel");
  const int N = pr->N, n_ch = pr->n_ch;
  OzParams p{};
  p.n = N;
  p.RT = (N + OZ_M - 1) / OZ_M;
  p.nK = (N + OZ_KC - 1) / OZ_KC;
  p.n_cb = (int)((ncol + OZ_BN - 1) / OZ_BN);
  p.n_tiles = n_ch * p.n_cb;
  p.ncol = ncol;
  p.stage_bytes = (uint32_t)p.RT * OZ_L * OZ_A_PLANE + OZ_L * OZ_B_PLANE;
  p.A = use_O ? pr->d.O_oz : pr->d.Vt_oz;
  p.EA = use_O ? pr->d.O_ozE : pr->d.Vt_ozE;
  p.Bh = Bh;
  p.Bl = Bl;
  p.C = C;
  p.Ch = Ch;
  p.Cl = Cl;
  p.err = pr->d.tc_err;
  p.expire_first = g_oz_expire_first.load(std::memory_order_relaxed);
  int *F = nullptr;
  WPCD_CUDA_TRY(pool_malloc(&F, sizeof(int) * (size_t)n_ch * ncol, s));
  p.FB = F;
  oz_colexp_kernel<<<grid_for((int64_t)n_ch * ncol, 256), 256, 0, s>>>(n_ch, N, ncol, Bh, F);
  const int grid = std::min(p.n_tiles, std::max(1, g_oz_sms[pr->device]));
  const size_t smem = (size_t)OZ_STAGES * p.stage_bytes;
  if (Ch)
    oz_gemm_kernel<true><<<grid, OZ_THREADS, smem, s>>>(p);
  else
    oz_gemm_kernel<false><<<grid, OZ_THREADS, smem, s>>>(p);
  count_launches(2);
  pool_free(F, s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "digit-plane gemm launch");
}

}  // namespace wpcd
