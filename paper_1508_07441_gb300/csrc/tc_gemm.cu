// Tensor-core (tcgen05) version of the dense channel-block products of the
// K application (Sec. 3.3, Eq. kernel): for every channel block
//   C = A X'        A = Vt_ch or O_ch (N x N), X' = X or G1 o X (N x 2MB)
// with FP32 inputs and outputs, for the FP32 inner cycles of the mixed
// solve.  Each FP32 operand is split into two TF32 parts, x = hi + lo, and
// C accumulates hi*hi + hi*lo + lo*hi in FP32 (three kind::tf32 MMAs per
// K step; the lo*lo term is below FP32 resolution), which keeps about 21
// significant bits in every product.
//
// One CTA computes RT row tiles of 128 rows (all of C's rows, N <= 512)
// times 128 output columns, so X' is read once.  Per K chunk of 16:
//   - A (constant per problem, packed once into the MMA operand layout as
//     TF32 hi/lo blocks by tc_pack_kernel) arrives by one bulk async copy
//     (cp.async.bulk, completion counted on an mbarrier);
//   - the threads form X' (the G1 complex scaling fused in), split it into
//     TF32 hi/lo and store it in the operand layout;
//   - one thread issues the MMAs into TMEM accumulators (one 128 x BN
//     accumulator per row tile) and commits them to the stage's mbarrier,
//     which frees the stage for chunk + STAGES.
// The epilogue reads the accumulators with tcgen05.ld and writes C (or
// S - C).  Shared-memory operands use the no-swizzle K-major layout: 8-row
// groups of 512 B, each four 8 x 16 B core matrices along K (K-core stride
// 128 B, row-group stride 512 B).  Every mbarrier wait has an iteration
// limit; a wait that runs out sets the error word and the kernel still
// waits (bounded) for its MMAs before it frees TMEM and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "wpcd_internal.h"

namespace wpcd {
namespace {

constexpr int TC_M = 128;       // rows per MMA (TMEM lanes)
constexpr int TC_KC = 16;       // K per pipeline stage: two K = 8 MMA steps
constexpr int TC_THREADS = 256;
constexpr uint32_t TC_A_HALF = TC_M * TC_KC * 4;  // one TF32 part of one row tile: 8 KB
constexpr uint32_t TC_A_BLOCK = 2 * TC_A_HALF;    // hi + lo: 16 KB
constexpr uint32_t TC_KSTRIDE = 128;              // between core matrices along K
constexpr uint32_t TC_RSTRIDE = 512;              // between 8-row groups
constexpr int TC_MAX_STAGES = 3;
constexpr int TC_MAX_RAW = 4;  // raw panel chunks in flight (bulk-copy path)
constexpr long long TC_SPIN_LIMIT = 1LL << 22;

struct TcParams {
  int n, RT, nK, stages, raw_stages;
  int64_t ncol;
  uint32_t stage_bytes, raw_bytes, tmem_cols;
  const float *A;       // packed TF32 blocks [n_ch][nK][RT][hi | lo]
  const float2 *X, *G;  // [n_ch][n][ncol / 2] complex
  const float *S;       // epilogue S - C (SUB)
  float *C;
  int *err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, K-core stride (leading byte
// offset), row-group stride (stride byte offset), descriptor version 1,
// no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(TC_KSTRIDE >> 4) << 16) |
         ((uint64_t)(TC_RSTRIDE >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major,
// N = BN, M = 128
__host__ __device__ constexpr uint32_t tc_idesc(int BN) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (long long i = 0; i < TC_SPIN_LIMIT; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 16 consecutive 32-bit TMEM columns
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (row r, k) inside a [rows/8][KC/4][8][4] block
__host__ __device__ __forceinline__ uint32_t tc_off(int r, int k) {
  return (uint32_t)((r >> 3) * TC_RSTRIDE + (k >> 2) * TC_KSTRIDE + (r & 7) * 16 + (k & 3) * 4);
}

// A (FP64, [n_ch][n][n]) -> TF32 hi/lo blocks in the operand layout,
// [n_ch][nK][RT][hi (8 KB) | lo (8 KB)], zero outside n x n
__global__ void tc_pack_kernel(int n_ch, int n, int RT, int nK, const double *__restrict__ A,
                               float *__restrict__ out) {
  const int64_t total = (int64_t)n_ch * nK * RT * TC_M * TC_KC;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total; f += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(f % TC_KC);
    const int r = (int)((f / TC_KC) % TC_M);
    const int64_t blk = f / (TC_KC * TC_M);  // (ch * nK + c) * RT + rt
    const int rt = (int)(blk % RT);
    const int c = (int)((blk / RT) % nK);
    const int ch = (int)(blk / ((int64_t)RT * nK));
    const int row = rt * TC_M + r, col = c * TC_KC + k;
    const float x = (row < n && col < n) ? (float)A[((size_t)ch * n + row) * n + col] : 0.f;
    const uint32_t hi = to_tf32(x);
    const uint32_t lo = to_tf32(x - __uint_as_float(hi));
    char *base = reinterpret_cast<char *>(out) + (size_t)blk * TC_A_BLOCK + tc_off(r, k);
    *reinterpret_cast<uint32_t *>(base) = hi;
    *reinterpret_cast<uint32_t *>(base + TC_A_HALF) = lo;
  }
}

// RAW: the X (and G1) panel rows arrive by bulk async copies into a ring of
// raw chunks in shared memory, issued TC_MAX_RAW chunks ahead by one
// thread; otherwise each thread prefetches the next chunk into registers
template <int BN, bool SCALE_G, bool SUB, bool RAW>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(TcParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_a[TC_MAX_STAGES], bar_mma[TC_MAX_STAGES], bar_done;
  __shared__ __align__(8) uint64_t bar_raw[TC_MAX_RAW];
  __shared__ uint32_t tmem_holder;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ch = blockIdx.z;
  const int n = p.n, RT = p.RT, nK = p.nK, NS = p.stages;
  const int64_t ncol = p.ncol, col0 = (int64_t)blockIdx.x * BN;
  const uint32_t b_half = (uint32_t)BN * TC_KC * 4;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&bar_a[s], 1);
      mbar_init(&bar_mma[s], 1);
    }
    mbar_init(&bar_done, 1);
    if (RAW)
      for (int r = 0; r < p.raw_stages; ++r) mbar_init(&bar_raw[r], 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_holder;
  const uint32_t idesc = tc_idesc(BN);
  bool ok = true;

  const float2 *X = p.X + (size_t)ch * n * (ncol / 2);
  const float2 *G = SCALE_G ? p.G + (size_t)ch * n * (ncol / 2) : nullptr;
  // X' chunk c: rows k = c*KC .. c*KC+15, output columns col0 .. col0+BN-1.
  // Item (kg, nn): operand row nn (output column col0 + nn), K group kg
  // (4 rows); consecutive lanes take consecutive nn, so each store
  // instruction of a warp fills 512 contiguous bytes.
  constexpr int ITEMS = (TC_KC / 4) * BN / TC_THREADS;
  // register path: the raw values of chunk c + 1 are loaded while chunk c
  // is converted
  auto load_chunk = [&](int c, float2 (&xv)[ITEMS][4], float2 (&gv)[ITEMS][4]) {
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int item = tid + it * TC_THREADS;
      const int nn = item % BN, kg = item / BN;
      const int64_t gc = col0 + nn;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = c * TC_KC + kg * 4 + q;
        const bool in = k < n && gc < ncol;
        const size_t o = (size_t)k * (ncol / 2) + (gc >> 1);
        xv[it][q] = in ? X[o] : make_float2(0.f, 0.f);
        if (SCALE_G) gv[it][q] = in ? G[o] : make_float2(0.f, 0.f);
      }
    }
  };
  // bulk-copy path: raw chunk c (rows of X, then of G1; BN floats each,
  // the valid columns only) into ring slot c % raw_stages
  unsigned char *raw0 = smem + (size_t)NS * p.stage_bytes;
  const int valid_cols = (int)min((int64_t)BN, ncol - col0);  // a multiple of 4 on this path
  auto issue_raw = [&](int c) {
    const int r = c % p.raw_stages;
    unsigned char *dst = raw0 + (size_t)r * p.raw_bytes;
    const int rows = min(TC_KC, n - c * TC_KC);
    const uint32_t row_bytes = (uint32_t)valid_cols * 4;
    const uint32_t total = (uint32_t)rows * row_bytes * (SCALE_G ? 2u : 1u);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar_raw[r])),
                 "r"(total)
                 : "memory");
    for (int k = 0; k < rows; ++k) {
      const float *src = reinterpret_cast<const float *>(X) + (size_t)(c * TC_KC + k) * ncol + col0;
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(dst + (size_t)k * BN * 4)),
                   "l"(src), "r"(row_bytes), "r"(smem_u32(&bar_raw[r]))
                   : "memory");
      if (SCALE_G) {
        const float *gsrc = reinterpret_cast<const float *>(G) + (size_t)(c * TC_KC + k) * ncol + col0;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(dst + (size_t)(TC_KC + k) * BN * 4)),
            "l"(gsrc), "r"(row_bytes), "r"(smem_u32(&bar_raw[r]))
            : "memory");
      }
    }
  };
  int a_last = -1, raw_last = -1;  // thread 0: last chunks whose copies it saw complete
  float2 xv[ITEMS][4], gv[ITEMS][4];
  if (RAW) {
    if (tid == 0)
      for (int c = 0; c < min(p.raw_stages, nK); ++c) issue_raw(c);
  } else {
    load_chunk(0, xv, gv);
  }
  for (int c = 0; c < nK; ++c) {
    const int s = c % NS;
    const uint32_t use = (uint32_t)(c / NS);
    unsigned char *st = smem + (size_t)s * p.stage_bytes;
    // the MMAs of chunk c - NS read this stage
    if (c >= NS && ok) ok = mbar_wait(&bar_mma[s], (use - 1) & 1);
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)RT * TC_A_BLOCK;
      const float *src = p.A + ((size_t)ch * nK + c) * RT * (TC_A_BLOCK / 4);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar_a[s])), "r"(bytes)
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(st)),
                   "l"(src), "r"(bytes), "r"(smem_u32(&bar_a[s]))
                   : "memory");
    }
    float2 xn[ITEMS][4], gn[ITEMS][4];
    if (RAW) {
      const int r = c % p.raw_stages;
      if (ok) ok = mbar_wait(&bar_raw[r], (uint32_t)(c / p.raw_stages) & 1);
      if (ok) raw_last = c;
      const float2 *rx = reinterpret_cast<const float2 *>(raw0 + (size_t)r * p.raw_bytes);
      const float2 *rg = rx + TC_KC * BN / 2;
#pragma unroll
      for (int it = 0; it < ITEMS; ++it) {
        const int item = tid + it * TC_THREADS;
        const int nn = item % BN, kg = item / BN;
        const bool col_in = nn < valid_cols;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int kl = kg * 4 + q;
          const bool in = col_in && c * TC_KC + kl < n;
          xv[it][q] = in ? rx[kl * (BN / 2) + (nn >> 1)] : make_float2(0.f, 0.f);
          if (SCALE_G) gv[it][q] = in ? rg[kl * (BN / 2) + (nn >> 1)] : make_float2(0.f, 0.f);
        }
      }
    } else if (c + 1 < nK) {
      load_chunk(c + 1, xn, gn);
    }
    unsigned char *bhi = st + (size_t)RT * TC_A_BLOCK, *blo = bhi + b_half;
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int item = tid + it * TC_THREADS;
      const int nn = item % BN, kg = item / BN;
      const bool odd = ((col0 + nn) & 1) != 0;
      float v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 x = xv[it][q];
        if (SCALE_G) {
          const float2 g = gv[it][q];
          v[q] = odd ? (g.x * x.y + g.y * x.x) : (g.x * x.x - g.y * x.y);
        } else {
          v[q] = odd ? x.y : x.x;
        }
      }
      uint4 h, l;
      h.x = to_tf32(v[0]);
      h.y = to_tf32(v[1]);
      h.z = to_tf32(v[2]);
      h.w = to_tf32(v[3]);
      l.x = to_tf32(v[0] - __uint_as_float(h.x));
      l.y = to_tf32(v[1] - __uint_as_float(h.y));
      l.z = to_tf32(v[2] - __uint_as_float(h.z));
      l.w = to_tf32(v[3] - __uint_as_float(h.w));
      const uint32_t off = tc_off(nn, kg * 4);
      *reinterpret_cast<uint4 *>(bhi + off) = h;
      *reinterpret_cast<uint4 *>(blo + off) = l;
    }
    if (!RAW && c + 1 < nK) {
#pragma unroll
      for (int it = 0; it < ITEMS; ++it)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xv[it][q] = xn[it][q];
          if (SCALE_G) gv[it][q] = gn[it][q];
        }
    }
    // generic-proxy stores -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      // every thread has read raw slot c % raw_stages: refill it
      if (RAW && c + p.raw_stages < nK) issue_raw(c + p.raw_stages);
      if (ok) ok = mbar_wait(&bar_a[s], use & 1);
      if (ok) a_last = c;
      const uint32_t a0 = smem_u32(st), b0 = smem_u32(bhi);
#pragma unroll 1
      for (int rt = 0; rt < RT; ++rt) {
        const uint32_t d = tmem + (uint32_t)(rt * BN);
#pragma unroll
        for (int ks = 0; ks < TC_KC / 8; ++ks) {
          const uint32_t ko = (uint32_t)ks * 2 * TC_KSTRIDE;
          const uint64_t ahi = umma_desc(a0 + rt * TC_A_BLOCK + ko);
          const uint64_t alo = umma_desc(a0 + rt * TC_A_BLOCK + TC_A_HALF + ko);
          const uint64_t bh = umma_desc(b0 + ko), bl = umma_desc(b0 + b_half + ko);
          tc_mma(d, ahi, bh, idesc, (c > 0 || ks > 0) ? 1u : 0u);
          tc_mma(d, ahi, bl, idesc, 1u);
          tc_mma(d, alo, bh, idesc, 1u);
        }
      }
      tc_commit(&bar_mma[s]);
    }
  }
  if (tid == 0) {
    // after a wait ran out, still wait (bounded) for the copies this CTA
    // issued, so that none lands in shared memory after the CTA has gone
    for (int c = a_last + 1; c < nK; ++c) mbar_wait(&bar_a[c % NS], (uint32_t)(c / NS) & 1);
    if (RAW)
      for (int c = raw_last + 1; c < nK; ++c)
        mbar_wait(&bar_raw[c % p.raw_stages], (uint32_t)(c / p.raw_stages) & 1);
    tc_commit(&bar_done);
  }
  // always wait (bounded) for the MMAs before TMEM is read or freed
  const bool done = mbar_wait(&bar_done, 0);
  ok = ok && done;
  tc_fence_after();
  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, half w / 4 of the columns
  const int lg = warp & 3, half = warp >> 2;
  // a thread's 16 columns of one row go out as four 16-byte stores when the
  // row start is 16-byte aligned (ncol a multiple of 4) and all 16 exist
  const bool vec_out = ncol % 4 == 0;
  for (int rt = 0; rt < RT; ++rt) {
    const int row = rt * TC_M + lg * 32 + lane;
    for (int cb = half * (BN / 2); cb < (half + 1) * (BN / 2); cb += 16) {
      const size_t o = ((size_t)ch * n + min(row, n - 1)) * ncol + col0 + cb;
      const bool full = vec_out && col0 + cb + 16 <= ncol;
      float4 sv[4];
      if (SUB && full && row < n)  // issue the S loads before the TMEM read
#pragma unroll
        for (int q = 0; q < 4; ++q) sv[q] = *reinterpret_cast<const float4 *>(p.S + o + 4 * q);
      float v[16];
      tc_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(rt * BN + cb), v);
      if (row < n && done) {
        if (full) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float4 w = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            if (SUB) w = make_float4(sv[q].x - w.x, sv[q].y - w.y, sv[q].z - w.z, sv[q].w - w.w);
            *reinterpret_cast<float4 *>(p.C + o + 4 * q) = w;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (col0 + cb + j < ncol) p.C[o + j] = SUB ? p.S[o + j] - v[j] : v[j];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
  if (!ok && lane == 0) atomicOr(p.err, 1);
}

struct TcShape {
  int RT, BN, nK, stages, raw_stages;
  uint32_t stage_bytes, raw_bytes, tmem_cols;
};

// 128 output columns per CTA, all N rows (RT tiles of 128); operand stages
// of one K chunk (A hi/lo for every row tile, the panel's hi/lo), two or
// three of them, then a ring of raw panel chunks (rows of X and G1) for
// the bulk-copy path: at most 192 KB, one CTA per SM
TcShape tc_shape(int n) {
  TcShape sh{};
  sh.RT = (n + TC_M - 1) / TC_M;
  sh.BN = 128;
  sh.nK = (n + TC_KC - 1) / TC_KC;
  sh.stage_bytes = (uint32_t)sh.RT * TC_A_BLOCK + 2u * (uint32_t)sh.BN * TC_KC * 4;
  sh.stages = 3 * sh.stage_bytes <= 96u * 1024 ? 3 : 2;
  sh.raw_bytes = 2u * TC_KC * sh.BN * 4;
  sh.raw_stages = sh.stages * sh.stage_bytes + TC_MAX_RAW * sh.raw_bytes <= 192u * 1024 ? TC_MAX_RAW : 2;
  const int cols = sh.RT * sh.BN;
  sh.tmem_cols = 32;
  while ((int)sh.tmem_cols < cols) sh.tmem_cols <<= 1;
  return sh;
}

}  // namespace

bool tc_supported(const wpcd_problem *pr) { return pr->N >= 1 && pr->N <= 4 * TC_M; }

// the FP32 channel-block products run on the tensor cores unless
// WPCD_GEMM=simt selects the FP32 SIMT kernel
bool tc_enabled() {
  const char *v = std::getenv("WPCD_GEMM");
  return !(v && std::strcmp(v, "simt") == 0);
}

// pack O and Vt into the tensor-core operand layout once per problem
wpcd_status tc_prepare(wpcd_problem *pr, cudaStream_t s) {
  if (pr->d.O_tc) return WPCD_OK;
  if (!tc_supported(pr)) return set_error(WPCD_EINVAL, "tensor-core GEMM needs N <= 512");
  const TcShape sh = tc_shape(pr->N);
  const size_t bytes = (size_t)pr->n_ch * sh.nK * sh.RT * TC_A_BLOCK;
  WPCD_CUDA_TRY(cudaMalloc(&pr->d.O_tc, bytes));
  WPCD_CUDA_TRY(cudaMalloc(&pr->d.Vt_tc, bytes));
  WPCD_CUDA_TRY(cudaMalloc(&pr->d.tc_err, sizeof(int)));
  WPCD_CUDA_TRY(cudaMemsetAsync(pr->d.tc_err, 0, sizeof(int), s));
  const int64_t total = (int64_t)pr->n_ch * sh.nK * sh.RT * TC_M * TC_KC;
  tc_pack_kernel<<<grid_for(total, 256), 256, 0, s>>>(pr->n_ch, pr->N, sh.RT, sh.nK, pr->d.O, pr->d.O_tc);
  tc_pack_kernel<<<grid_for(total, 256), 256, 0, s>>>(pr->n_ch, pr->N, sh.RT, sh.nK, pr->d.Vt, pr->d.Vt_tc);
  count_launches(2);
  // the shared-memory limit is an attribute of the kernel on each device
  static bool attr_set[64] = {};
  if (pr->device < 0 || pr->device >= 64) return set_error(WPCD_EINVAL, "device ordinal out of range");
  if (!attr_set[pr->device]) {
    // the largest stage set of any shape (tc_shape: at most 192 KB); the
    // static barriers and the TMEM address take part of the rest
    const int max_bytes = 192 * 1024;
    WPCD_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<128, true, false, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes));
    WPCD_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<128, false, false, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes));
    WPCD_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<128, false, true, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes));
    WPCD_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<128, true, false, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes));
    WPCD_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<128, false, false, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes));
    WPCD_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<128, false, true, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes));
    attr_set[pr->device] = true;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "tensor-core pack");
}

// C = A X' (or S - A X') for every channel block; FP32 vectors in the
// batched layout ([n_ch][N][ncol] real, ncol = 2 M B)
wpcd_status tc_gemm(const wpcd_problem *pr, bool use_O, const float *G, const float *X, const float *S, float *C,
                    int64_t ncol, cudaStream_t s) {
  if (!pr->d.O_tc) return set_error(WPCD_EINVAL, "tensor-core operands not prepared");
  const TcShape sh = tc_shape(pr->N);
  TcParams p{};
  p.n = pr->N;
  p.RT = sh.RT;
  p.nK = sh.nK;
  p.stages = sh.stages;
  p.ncol = ncol;
  p.stage_bytes = sh.stage_bytes;
  p.tmem_cols = sh.tmem_cols;
  p.A = use_O ? pr->d.O_tc : pr->d.Vt_tc;
  p.X = reinterpret_cast<const float2 *>(X);
  p.G = reinterpret_cast<const float2 *>(G);
  p.S = S;
  p.C = C;
  p.err = pr->d.tc_err;
  p.raw_stages = sh.raw_stages;
  p.raw_bytes = sh.raw_bytes;
  // bulk copies need 16-byte aligned panel rows: ncol a multiple of 4 and
  // aligned bases (every row, and every column tile, then starts aligned)
  const bool raw = ncol % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                   (!G || (reinterpret_cast<uintptr_t>(G) & 15) == 0);
  const size_t smem = (size_t)sh.stages * sh.stage_bytes + (raw ? (size_t)sh.raw_stages * sh.raw_bytes : 0);
  dim3 grid((unsigned)((ncol + sh.BN - 1) / sh.BN), 1, pr->n_ch);
#define WPCD_TC_LAUNCH(RAW)                                                 \
  do {                                                                      \
    if (G)                                                                  \
      tc_gemm_kernel<128, true, false, RAW><<<grid, TC_THREADS, smem, s>>>(p);  \
    else if (S)                                                             \
      tc_gemm_kernel<128, false, true, RAW><<<grid, TC_THREADS, smem, s>>>(p);  \
    else                                                                    \
      tc_gemm_kernel<128, false, false, RAW><<<grid, TC_THREADS, smem, s>>>(p); \
  } while (0)
  if (raw)
    WPCD_TC_LAUNCH(true);
  else
    WPCD_TC_LAUNCH(false);
#undef WPCD_TC_LAUNCH
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "tensor-core gemm launch");
}

// nonzero if a tensor-core GEMM of this problem ran out of a wait limit
wpcd_status tc_check(const wpcd_problem *pr, cudaStream_t s) {
  if (!pr->d.tc_err) return WPCD_OK;
  int h = 0;
  WPCD_CUDA_TRY(cudaMemcpyAsync(&h, pr->d.tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  if (h) return set_error(WPCD_ETIMEOUT, "tensor-core GEMM wait limit reached");
  return WPCD_OK;
}

}  // namespace wpcd
