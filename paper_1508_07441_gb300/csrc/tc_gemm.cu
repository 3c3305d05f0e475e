// Tensor-core (tcgen05) version of the dense channel-block products of the
// K application (Sec. 3.3, Eq. kernel): for every channel block
//   C = A X'        A = Vt_ch or O_ch (N x N), X' = X or G1 o X (N x 2MB)
// with FP32 inputs and outputs, for the FP32 inner cycles of the mixed
// solve.  Each FP32 operand is split into two TF32 parts, x = hi + lo, and
// C accumulates hi*hi + hi*lo + lo*hi in FP32 (three kind::tf32 MMAs per
// K step; the lo*lo term is below FP32 resolution), which keeps about 21
// significant bits in every product.
//
// An output tile is RT row tiles of 128 rows (all of C's rows, N <= 512)
// times 128 output columns, so X' is read once.  Per K chunk of 16:
//   - A (constant per problem, packed once into the MMA operand layout as
//     TF32 hi/lo blocks by tc_pack_kernel) arrives by one bulk async copy
//     (cp.async.bulk, completion counted on an mbarrier);
//   - X' (the G1 complex scaling fused in) is formed, split into TF32 hi/lo
//     and stored in the operand layout;
//   - one thread issues the MMAs into TMEM accumulators (one 128 x 128
//     accumulator per row tile) and commits them to the stage's mbarrier,
//     which frees the stage.
// The epilogue reads the accumulators with tcgen05.ld and writes C (or
// S - C).  Aligned panels run in a persistent warp-specialised kernel (one
// CTA per SM, rings of A, raw-panel and operand stages, double-buffered
// accumulators); other panels in a one-tile-per-CTA kernel.  Shared-memory operands use the no-swizzle K-major layout: 8-row
// groups of 512 B, each four 8 x 16 B core matrices along K (K-core stride
// 128 B, row-group stride 512 B).  Every mbarrier wait has an iteration
// limit; a wait that runs out sets the error word and the kernel still
// waits (bounded) for its MMAs before it frees TMEM and returns.
#include <cuda.h>  // CUtensorMap (encoded through the runtime's driver entry point)
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>

#include "common.cuh"
#include "tc_ptx.cuh"
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

struct TcParams {
  int n, RT, nK, stages;
  int64_t ncol;
  uint32_t stage_bytes, tmem_cols;
  const float *A;       // packed TF32 blocks [n_ch][nK][RT][hi | lo]
  const float2 *X, *G;  // [n_ch][n][ncol / 2] complex
  const float *S;       // epilogue S - C (SUB)
  float *C;
  int *err;
  int vec_out;          // C (and S) rows 16-byte aligned: float4 epilogue
};

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


__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
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

// Panels that are not 16-byte aligned (the persistent kernel below takes
// the aligned ones): one CTA per 128-column tile, every thread converts
// chunk c while it holds the raw values of chunk c + 1 in registers
template <int BN, bool SCALE_G, bool SUB>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(TcParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_a[TC_MAX_STAGES], bar_mma[TC_MAX_STAGES], bar_done;
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
  // the raw values of chunk c + 1 are loaded while chunk c is converted
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
  int a_last = -1;  // thread 0: last chunk whose A copy it saw complete
  float2 xv[ITEMS][4], gv[ITEMS][4];
  load_chunk(0, xv, gv);
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
    if (c + 1 < nK) {
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
    if (c + 1 < nK) {
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
  const bool vec_out = p.vec_out != 0;
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

// ---------------------------------------------------------------------------
// Persistent warp-specialised version for 16-byte aligned panels: one CTA
// per SM walks the (channel, 128-column) output tiles; its warps take fixed
// roles and hand work over through mbarrier rings, so that copies, format
// conversion, MMAs and the epilogue of different chunks and tiles overlap:
//   warp 0      producer: bulk async copies of the packed A chunks (ring of
//               nsa stages) and tensor (TMA) copies of the raw X / G1 panel
//               chunks, one 16-row x 128-column box each (ring of nr)
//   warp 1      MMA issuer (one thread) and TMEM owner: 3 TF32 MMAs per
//               K step and row tile; commits free the A and B stages and,
//               after a tile's last chunk, hand the accumulator to the
//               epilogue
//   warps 2-5   converters: raw chunk -> G1 o X -> TF32 hi/lo in the
//               operand layout (ring of nsb B stages)
//   warps 6-9   epilogue: TMEM -> registers -> C (or S - C); warp w reads
//               TMEM lanes 32 (w % 4) .. +31
// The accumulators are double-buffered in TMEM when 2 RT 128 columns fit
// (N <= 256), so the epilogue of tile i overlaps the MMAs of tile i + 1.
// Every wait is bounded and also gives up once another role has set the
// CTA's abort flag; before the CTA exits, the producer waits (bounded) for
// every copy it issued and the MMA thread for every MMA it issued.
// ---------------------------------------------------------------------------
constexpr int WS_THREADS = 320;
constexpr int WS_MAX_A = 3, WS_MAX_B = 3, WS_MAX_R = 8;
constexpr int WS_BN = 128;
constexpr uint32_t WS_B_HALF = WS_BN * TC_KC * 4;  // one TF32 part of a B stage: 8 KB
constexpr uint32_t WS_B_STAGE = 2 * WS_B_HALF;
constexpr int WS_CONV = 128;                       // converter threads
constexpr int WS_EPI = 128;                        // epilogue threads

struct TcWsParams {
  int RT, n_tiles, nsa, nsb, nr, n_acc;  // RT: the largest row-tile count of any tile
  uint32_t raw_bytes, tmem_cols;
  int *err;
  int expire_role;  // -1, or the role (WsRole) whose first wait runs out at once
};

enum WsRole { WS_PRODUCER = 0, WS_MMA = 1, WS_CONVERTER = 2, WS_EPILOGUE = 3 };

// one output tile: 128 columns (col0 ..) of one channel block C = A X'
// ([n][ncol] floats at C), A packed as [nK][RT][hi | lo] TF32 blocks; the
// panel chunks come from rows y0 + 16 c of the tensor maps
struct WsTile {
  int n, RT, nK, y0;
  int64_t ncol, col0;
  const float *A, *S;
  float *C;
  const CUtensorMap *tmx, *tmg;
};

// the tiles of one problem: t -> (channel, column block)
struct WsTilesOne {
  CUtensorMap tmx, tmg;  // X and G1 as [n_ch n rows][ncol floats], box 16 x 128
  int n, RT, nK, n_cb;
  int64_t ncol;
  const float *A, *S;
  float *C;
  __device__ __forceinline__ WsTile get(int t) const {
    WsTile T;
    const int ch = t / n_cb;
    T.n = n;
    T.RT = RT;
    T.nK = nK;
    T.y0 = ch * n;
    T.ncol = ncol;
    T.col0 = (int64_t)(t % n_cb) * WS_BN;
    T.A = A + (size_t)ch * nK * RT * (TC_A_BLOCK / 4);
    const size_t blk = (size_t)ch * n * ncol;
    T.S = S ? S + blk : nullptr;
    T.C = C + blk;
    T.tmx = &tmx;
    T.tmg = &tmg;
    return T;
  }
};

// the tiles of a group of problems (the grouped solve): problem g owns
// tiles toff[g] .. toff[g+1]-1 over (channel, column block) of its segment
constexpr int WS_GROUP_MAX = WPCD_GROUP_MAX;
struct alignas(64) WsProb {
  CUtensorMap tmx, tmg;  // the segment's X and G1 as [n_ch n rows][ncol floats]
  const float *A;        // packed A of the problem (all channels)
  int64_t off;           // float offset of the segment in the group vectors
  int64_t ncol;
  int n, RT, nK, n_cb;
};
struct WsTilesGroup {
  WsProb p[WS_GROUP_MAX];
  int toff[WS_GROUP_MAX + 1];
  int n_prob;
  const float *S;
  float *C;
  __device__ __forceinline__ WsTile get(int t) const {
    int lo = 0, hi = n_prob - 1;  // largest g with toff[g] <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (toff[mid] <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    const WsProb &q = p[lo];
    const int lt = t - toff[lo], ch = lt / q.n_cb;
    WsTile T;
    T.n = q.n;
    T.RT = q.RT;
    T.nK = q.nK;
    T.y0 = ch * q.n;
    T.ncol = q.ncol;
    T.col0 = (int64_t)(lt % q.n_cb) * WS_BN;
    T.A = q.A + (size_t)ch * q.nK * q.RT * (TC_A_BLOCK / 4);
    const size_t blk = (size_t)q.off + (size_t)ch * q.n * q.ncol;
    T.S = S ? S + blk : nullptr;
    T.C = C + blk;
    T.tmx = &q.tmx;
    T.tmg = &q.tmg;
    return T;
  }
};

struct WsBars {
  uint64_t a_full[WS_MAX_A], a_empty[WS_MAX_A], b_full[WS_MAX_B], b_empty[WS_MAX_B];
  uint64_t r_full[WS_MAX_R], r_empty[WS_MAX_R], t_full[2], t_empty[2], fin;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// one 2-D box of a tensor map at (x = column, y = row) into shared memory;
// x is a multiple of 128 floats (512 bytes), rows past the end read zeros
__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bounded wait that also ends when another role has aborted; running out
// of the limit aborts the CTA and sets the error word
__device__ __forceinline__ bool ws_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err,
                                        long long limit) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  atomicOr(err, 1);
  return false;
}

// Tiles: WsTilesOne or WsTilesGroup (a parameter in the constant bank, so
// that the tensor maps it holds have the address the TMA copies need)
template <bool SCALE_G, bool SUB, class Tiles>
__global__ void __launch_bounds__(WS_THREADS, 1)
    tc_gemm_ws_kernel(const __grid_constant__ Tiles tiles, TcWsParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) WsBars bars;
  __shared__ uint32_t tmem_holder;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int RTM = p.RT;  // A stage and accumulator stride (largest RT)
  unsigned char *a_ring = smem;
  unsigned char *b_ring = smem + (size_t)p.nsa * RTM * TC_A_BLOCK;
  unsigned char *r_ring = b_ring + (size_t)p.nsb * WS_B_STAGE;
  const int my_tiles = (p.n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;

  if (tid == 0) {
    for (int i = 0; i < p.nsa; ++i) {
      mbar_init(&bars.a_full[i], 1);
      mbar_init(&bars.a_empty[i], 1);
    }
    for (int i = 0; i < p.nsb; ++i) {
      mbar_init(&bars.b_full[i], WS_CONV);
      mbar_init(&bars.b_empty[i], 1);
    }
    for (int i = 0; i < p.nr; ++i) {
      mbar_init(&bars.r_full[i], 1);
      mbar_init(&bars.r_empty[i], WS_CONV);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars.t_full[i], 1);
      mbar_init(&bars.t_empty[i], WS_EPI);
    }
    mbar_init(&bars.fin, 1);
    abort_flag = 0;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_holder;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      WaitLimit lim(p.expire_role == WS_PRODUCER);
      int last_a[WS_MAX_A], last_r[WS_MAX_R];
      for (int i = 0; i < WS_MAX_A; ++i) last_a[i] = -1;
      for (int i = 0; i < WS_MAX_R; ++i) last_r[i] = -1;
      bool ok = true;
      int q = 0;
      for (int lt = 0; lt < my_tiles && ok; ++lt) {
        const WsTile T = tiles.get((int)blockIdx.x + lt * (int)gridDim.x);
        for (int c = 0; c < T.nK; ++c, ++q) {
          const int sr = q % p.nr;
          if (q >= p.nr && !(ok = ws_wait(&bars.r_empty[sr], (uint32_t)(q / p.nr - 1) & 1, &abort_flag, p.err, lim.next())))
            break;
          // the whole box counts, zero-filled parts included; rows of the
          // next channel that a last chunk reaches are masked by the converters
          unsigned char *dst = r_ring + (size_t)sr * p.raw_bytes;
          expect_tx(&bars.r_full[sr], TC_KC * WS_BN * 4 * (SCALE_G ? 2u : 1u));
          tma_2d(dst, T.tmx, (int)T.col0, T.y0 + c * TC_KC, &bars.r_full[sr]);
          if (SCALE_G) tma_2d(dst + TC_KC * WS_BN * 4, T.tmg, (int)T.col0, T.y0 + c * TC_KC, &bars.r_full[sr]);
          last_r[sr] = q;
          const int sa = q % p.nsa;
          if (q >= p.nsa && !(ok = ws_wait(&bars.a_empty[sa], (uint32_t)(q / p.nsa - 1) & 1, &abort_flag, p.err, lim.next())))
            break;
          const uint32_t abytes = (uint32_t)T.RT * TC_A_BLOCK;
          expect_tx(&bars.a_full[sa], abytes);
          bulk_g2s(a_ring + (size_t)sa * RTM * TC_A_BLOCK, T.A + (size_t)c * T.RT * (TC_A_BLOCK / 4), abytes,
                   &bars.a_full[sa]);
          last_a[sa] = q;
        }
      }
      // every issued copy lands before the CTA exits
      for (int i = 0; i < p.nsa; ++i)
        if (last_a[i] >= 0) mbar_wait(&bars.a_full[i], (uint32_t)(last_a[i] / p.nsa) & 1);
      for (int i = 0; i < p.nr; ++i)
        if (last_r[i] >= 0) mbar_wait(&bars.r_full[i], (uint32_t)(last_r[i] / p.nr) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = tc_idesc(WS_BN);
      WaitLimit lim(p.expire_role == WS_MMA);
      bool ok = true;
      int q = 0;
      for (int lt = 0; lt < my_tiles && ok; ++lt) {
        const int buf = lt % p.n_acc;
        if (lt >= p.n_acc && !(ok = ws_wait(&bars.t_empty[buf], (uint32_t)(lt / p.n_acc - 1) & 1, &abort_flag, p.err,
                                          lim.next())))
          break;
        tc_fence_after();
        const WsTile T = tiles.get((int)blockIdx.x + lt * (int)gridDim.x);
        const uint32_t d0 = tmem + (uint32_t)(buf * RTM * WS_BN);
        for (int c = 0; c < T.nK; ++c, ++q) {
          const int sa = q % p.nsa, sb = q % p.nsb;
          if (!(ok = ws_wait(&bars.a_full[sa], (uint32_t)(q / p.nsa) & 1, &abort_flag, p.err, lim.next()))) break;
          if (!(ok = ws_wait(&bars.b_full[sb], (uint32_t)(q / p.nsb) & 1, &abort_flag, p.err, lim.next()))) break;
          tc_fence_after();
          const uint32_t a0 = smem_u32(a_ring + (size_t)sa * RTM * TC_A_BLOCK);
          const uint32_t b0 = smem_u32(b_ring + (size_t)sb * WS_B_STAGE);
#pragma unroll 1
          for (int rt = 0; rt < T.RT; ++rt) {
            const uint32_t d = d0 + (uint32_t)(rt * WS_BN);
#pragma unroll
            for (int ks = 0; ks < TC_KC / 8; ++ks) {
              const uint32_t ko = (uint32_t)ks * 2 * TC_KSTRIDE;
              const uint64_t ahi = umma_desc(a0 + rt * TC_A_BLOCK + ko);
              const uint64_t alo = umma_desc(a0 + rt * TC_A_BLOCK + TC_A_HALF + ko);
              const uint64_t bh = umma_desc(b0 + ko), bl = umma_desc(b0 + WS_B_HALF + ko);
              tc_mma(d, ahi, bh, idesc, (c > 0 || ks > 0) ? 1u : 0u);
              tc_mma(d, ahi, bl, idesc, 1u);
              tc_mma(d, alo, bh, idesc, 1u);
            }
          }
          tc_commit(&bars.a_empty[sa]);
          tc_commit(&bars.b_empty[sb]);
        }
        if (ok) tc_commit(&bars.t_full[buf]);
      }
      // every issued MMA completes before TMEM is freed
      tc_commit(&bars.fin);
      mbar_wait(&bars.fin, 0);
    }
  } else if (warp < 6) {
    // ---------------- converters ----------------
    const int ct = tid - 64;
    constexpr int ITEMS = (TC_KC / 4) * WS_BN / WS_CONV;
    WaitLimit lim(p.expire_role == WS_CONVERTER);
    bool ok = true;
    int q = 0;
    for (int lt = 0; lt < my_tiles && ok; ++lt) {
      const WsTile T = tiles.get((int)blockIdx.x + lt * (int)gridDim.x);
      const int64_t col0 = T.col0;
      const int valid_cols = (int)min((int64_t)WS_BN, T.ncol - col0);
      for (int c = 0; c < T.nK; ++c, ++q) {
        const int sr = q % p.nr, sb = q % p.nsb;
        if (!(ok = ws_wait(&bars.r_full[sr], (uint32_t)(q / p.nr) & 1, &abort_flag, p.err, lim.next()))) break;
        const float2 *rx = reinterpret_cast<const float2 *>(r_ring + (size_t)sr * p.raw_bytes);
        const float2 *rg = rx + TC_KC * WS_BN / 2;
        float2 xv[ITEMS][4], gv[ITEMS][4];
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
          const int item = ct + it * WS_CONV;
          const int nn = item % WS_BN, kg = item / WS_BN;
          const bool col_in = nn < valid_cols;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const int kl = kg * 4 + qq;
            const bool in = col_in && c * TC_KC + kl < T.n;
            xv[it][qq] = in ? rx[kl * (WS_BN / 2) + (nn >> 1)] : make_float2(0.f, 0.f);
            if (SCALE_G) gv[it][qq] = in ? rg[kl * (WS_BN / 2) + (nn >> 1)] : make_float2(0.f, 0.f);
          }
        }
        if (q >= p.nsb && !(ok = ws_wait(&bars.b_empty[sb], (uint32_t)(q / p.nsb - 1) & 1, &abort_flag, p.err, lim.next())))
          break;
        unsigned char *bhi = b_ring + (size_t)sb * WS_B_STAGE, *blo = bhi + WS_B_HALF;
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
          const int item = ct + it * WS_CONV;
          const int nn = item % WS_BN, kg = item / WS_BN;
          const bool odd = ((col0 + nn) & 1) != 0;
          float v[4];
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const float2 x = xv[it][qq];
            if (SCALE_G) {
              const float2 g = gv[it][qq];
              v[qq] = odd ? (g.x * x.y + g.y * x.x) : (g.x * x.x - g.y * x.y);
            } else {
              v[qq] = odd ? x.y : x.x;
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
        // generic-proxy stores -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&bars.b_full[sb]);
        // the raw slot is released only now that the values read from it
        // have been stored: released right after the reads, it was refilled
        // under them whenever the producer ran ahead on raw slots (one raw
        // slot, or more A stages than raw slots), and products differed from
        // run to run
        mbar_arrive(&bars.r_empty[sr]);
      }
    }
  } else {
    // ---------------- epilogue ----------------
    const int lg = warp & 3;
    WaitLimit lim(p.expire_role == WS_EPILOGUE);
    bool ok = true;
    for (int lt = 0; lt < my_tiles && ok; ++lt) {
      const WsTile T = tiles.get((int)blockIdx.x + lt * (int)gridDim.x);
      const int n = T.n;
      const int64_t col0 = T.col0, ncol = T.ncol;
      const int buf = lt % p.n_acc;
      ok = ws_wait(&bars.t_full[buf], (uint32_t)(lt / p.n_acc) & 1, &abort_flag, p.err, lim.next());
      // the TMEM loads below are warp-collective: the warp decides together
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      tc_fence_after();
      for (int rt = 0; rt < T.RT; ++rt) {
        const int row = rt * TC_M + lg * 32 + lane;
        for (int cb = 0; cb < WS_BN; cb += 16) {
          const size_t o = (size_t)min(row, n - 1) * ncol + col0 + cb;
          // ncol % 4 == 0 and 16-byte aligned C and S on this path
          const bool full = col0 + cb + 16 <= ncol;
          float4 sv[4];
          if (SUB && full && row < n)  // the S loads go out before the TMEM read
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) sv[qq] = *reinterpret_cast<const float4 *>(T.S + o + 4 * qq);
          float v[16];
          __syncwarp();  // the TMEM load is warp-collective
          tc_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(buf * RTM * WS_BN + rt * WS_BN + cb), v);
          if (row < n) {
            if (full) {
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                float4 w = make_float4(v[4 * qq], v[4 * qq + 1], v[4 * qq + 2], v[4 * qq + 3]);
                if (SUB) w = make_float4(sv[qq].x - w.x, sv[qq].y - w.y, sv[qq].z - w.z, sv[qq].w - w.w);
                *reinterpret_cast<float4 *>(T.C + o + 4 * qq) = w;
              }
            } else {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (col0 + cb + j < ncol) T.C[o + j] = SUB ? T.S[o + j] - v[j] : v[j];
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&bars.t_empty[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
}

struct TcWsShape {
  int nsa, nsb, nr, n_acc;
  uint32_t raw_bytes, smem, tmem_cols;
};

// rings for the persistent kernel: A stages (RT 16 KB blocks each), three
// B stages of 16 KB, as many raw panel chunks as fit in 216 KB (at most 8);
// two accumulator buffers when they fit in the 512 TMEM columns
TcWsShape tc_ws_shape(int RT, bool scale_g) {
  TcWsShape w{};
  w.raw_bytes = (uint32_t)TC_KC * WS_BN * 4 * (scale_g ? 2u : 1u);
  w.nsa = RT <= 2 ? 3 : 2;
  w.nsb = WS_MAX_B;
  const uint32_t used = (uint32_t)w.nsa * RT * TC_A_BLOCK + (uint32_t)w.nsb * WS_B_STAGE;
  w.nr = (int)std::min<uint32_t>(WS_MAX_R, (216u * 1024 - used) / w.raw_bytes);
  w.smem = used + (uint32_t)w.nr * w.raw_bytes;
  w.n_acc = 2 * RT * WS_BN <= 512 ? 2 : 1;
  const int cols = w.n_acc * RT * WS_BN;
  w.tmem_cols = 32;
  while ((int)w.tmem_cols < cols) w.tmem_cols <<= 1;
  return w;
}

struct TcShape {
  int RT, BN, nK, stages;
  uint32_t stage_bytes, tmem_cols;
};

// 128 output columns per CTA, all N rows (RT tiles of 128); operand stages
// of one K chunk (A hi/lo for every row tile, the panel's hi/lo), two or
// three of them: at most 192 KB, one CTA per SM
TcShape tc_shape(int n) {
  TcShape sh{};
  sh.RT = (n + TC_M - 1) / TC_M;
  sh.BN = 128;
  sh.nK = (n + TC_KC - 1) / TC_KC;
  sh.stage_bytes = (uint32_t)sh.RT * TC_A_BLOCK + 2u * (uint32_t)sh.BN * TC_KC * 4;
  sh.stages = 3 * sh.stage_bytes <= 96u * 1024 ? 3 : 2;
  const int cols = sh.RT * sh.BN;
  sh.tmem_cols = 32;
  while ((int)sh.tmem_cols < cols) sh.tmem_cols <<= 1;
  return sh;
}

}  // namespace

std::atomic<int> g_ws_expire_role{-1};

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// [rows][ncol] FP32 panel, 16 x 128 boxes, zero fill outside
bool panel_map(CUtensorMap *m, const float *base, int64_t rows, int64_t ncol) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)ncol, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ncol * 4};
  const cuuint32_t box[2] = {WS_BN, TC_KC};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// per device: kernel attributes set, SM count (the persistent grid)
bool attr_set[64] = {};
int sm_count[64] = {};

// the persistent kernel over a tile source: rings sized for the largest
// row-tile count RT, one CTA per SM (at most one per tile)
template <class Tiles>
wpcd_status launch_ws(const Tiles &tiles, int n_tiles, int RT, bool scale_g, bool sub, int *err, int device,
                      cudaStream_t s) {
  const TcWsShape w = tc_ws_shape(RT, scale_g);
  TcWsParams q{};
  q.RT = RT;
  q.n_tiles = n_tiles;
  q.nsa = w.nsa;
  q.nsb = w.nsb;
  q.nr = w.nr;
  q.n_acc = w.n_acc;
  q.raw_bytes = w.raw_bytes;
  q.tmem_cols = w.tmem_cols;
  q.err = err;
  q.expire_role = g_ws_expire_role.load(std::memory_order_relaxed);
  const int grid = std::max(1, std::min(n_tiles, sm_count[device] > 0 ? sm_count[device] : 152));
  if (scale_g)
    tc_gemm_ws_kernel<true, false, Tiles><<<grid, WS_THREADS, w.smem, s>>>(tiles, q);
  else if (sub)
    tc_gemm_ws_kernel<false, true, Tiles><<<grid, WS_THREADS, w.smem, s>>>(tiles, q);
  else
    tc_gemm_ws_kernel<false, false, Tiles><<<grid, WS_THREADS, w.smem, s>>>(tiles, q);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "tensor-core gemm launch");
}

// the shared-memory limit of the persistent kernels (tc_ws_shape: at most 216 KB)
template <class Tiles>
cudaError_t set_ws_attributes() {
  const int ws_bytes = 216 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(tc_gemm_ws_kernel<true, false, Tiles>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                ws_bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(tc_gemm_ws_kernel<false, true, Tiles>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                ws_bytes)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(tc_gemm_ws_kernel<false, false, Tiles>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              ws_bytes);
}


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
  WPCD_CUDA_TRY(dev_malloc(&pr->d.O_tc, bytes));
  WPCD_CUDA_TRY(dev_malloc(&pr->d.Vt_tc, bytes));
  if (!pr->d.tc_err) {  // shared with the digit-plane products (oz_gemm.cu)
    WPCD_CUDA_TRY(dev_malloc(&pr->d.tc_err, sizeof(int)));
    WPCD_CUDA_TRY(cudaMemsetAsync(pr->d.tc_err, 0, sizeof(int), s));
  }
  const int64_t total = (int64_t)pr->n_ch * sh.nK * sh.RT * TC_M * TC_KC;
  tc_pack_kernel<<<grid_for(total, 256), 256, 0, s>>>(pr->n_ch, pr->N, sh.RT, sh.nK, pr->d.O, pr->d.O_tc);
  tc_pack_kernel<<<grid_for(total, 256), 256, 0, s>>>(pr->n_ch, pr->N, sh.RT, sh.nK, pr->d.Vt, pr->d.Vt_tc);
  count_launches(2);
  // the shared-memory limit is an attribute of the kernel on each device
  if (pr->device < 0 || pr->device >= 64) return set_error(WPCD_EINVAL, "device ordinal out of range");
  if (!attr_set[pr->device]) {
    // the largest stage set of any shape (tc_shape: at most 192 KB); the
    // static barriers and the TMEM address take part of the rest
    const int max_bytes = 192 * 1024;
    WPCD_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<128, true, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes));
    WPCD_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<128, false, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes));
    WPCD_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<128, false, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes));
    WPCD_CUDA_TRY(set_ws_attributes<WsTilesOne>());
    WPCD_CUDA_TRY(set_ws_attributes<WsTilesGroup>());
    WPCD_CUDA_TRY(cudaDeviceGetAttribute(&sm_count[pr->device], cudaDevAttrMultiProcessorCount, pr->device));
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
  auto aligned16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  // 16-byte aligned C and S rows: float4 epilogue stores and loads
  const bool vec_out = ncol % 4 == 0 && aligned16(C) && (!S || aligned16(S));
  // bulk copies need 16-byte aligned panel rows: ncol a multiple of 4 and
  // aligned bases (every row, and every column tile, then starts aligned)
  const bool raw = vec_out && aligned16(X) && (!G || aligned16(G));
  if (raw) {
    WsTilesOne tiles{};
    tiles.n = pr->N;
    tiles.RT = sh.RT;
    tiles.nK = sh.nK;
    tiles.n_cb = (int)((ncol + WS_BN - 1) / WS_BN);
    tiles.ncol = ncol;
    tiles.A = p.A;
    tiles.S = S;
    tiles.C = C;
    const int64_t rows = (int64_t)pr->n_ch * pr->N;
    if (!panel_map(&tiles.tmx, X, rows, ncol) || (G && !panel_map(&tiles.tmg, G, rows, ncol)))
      return set_error(WPCD_ECUDA, "tensor map encoding failed");
    wpcd_status st = launch_ws(tiles, pr->n_ch * tiles.n_cb, sh.RT, G != nullptr, S != nullptr, p.err, pr->device, s);
    if (st != WPCD_OK) return st;
  } else {
    p.vec_out = vec_out;
    const size_t smem = (size_t)sh.stages * sh.stage_bytes;
    dim3 grid((unsigned)((ncol + sh.BN - 1) / sh.BN), 1, pr->n_ch);
    if (G)
      tc_gemm_kernel<128, true, false><<<grid, TC_THREADS, smem, s>>>(p);
    else if (S)
      tc_gemm_kernel<128, false, true><<<grid, TC_THREADS, smem, s>>>(p);
    else
      tc_gemm_kernel<128, false, false><<<grid, TC_THREADS, smem, s>>>(p);
  }
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "tensor-core gemm launch");
}

// C = A X' (or S - A X') for every (problem, channel) block of a group in
// one persistent launch; problem g's vectors are the segment at float
// offset off[g] of X, G, S and C ([n_ch][N][ncol] floats), 16-byte aligned
// with ncol % 4 == 0; every problem prepared (tc_prepare), N <= 512
wpcd_status tc_gemm_group(const TcGroupProb *gp, int n_prob, bool use_O, const float *G, const float *X,
                          const float *S, float *C, cudaStream_t s) {
  if (n_prob < 1 || n_prob > WS_GROUP_MAX) return set_error(WPCD_EINVAL, "bad tensor-core group size");
  auto aligned16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  // about 21 KB: held on the heap, passed by value as the kernel parameter
  std::unique_ptr<WsTilesGroup> tiles(new WsTilesGroup());
  tiles->n_prob = n_prob;
  tiles->S = S;
  tiles->C = C;
  tiles->toff[0] = 0;
  int RTmax = 1;
  for (int g = 0; g < n_prob; ++g) {
    const wpcd_problem *pr = gp[g].pr;
    const int64_t off = gp[g].off, ncol = gp[g].ncol;
    if (!pr->d.O_tc || !tc_supported(pr)) return set_error(WPCD_EINVAL, "tensor-core operands not prepared");
    if (ncol % 4 != 0 || !aligned16(X + off) || !aligned16(C + off) || (G && !aligned16(G + off)) ||
        (S && !aligned16(S + off)))
      return set_error(WPCD_EINVAL, "tensor-core group segments must be 16-byte aligned");
    const TcShape sh = tc_shape(pr->N);
    WsProb &q = tiles->p[g];
    q.A = use_O ? pr->d.O_tc : pr->d.Vt_tc;
    q.off = off;
    q.ncol = ncol;
    q.n = pr->N;
    q.RT = sh.RT;
    q.nK = sh.nK;
    q.n_cb = (int)((ncol + WS_BN - 1) / WS_BN);
    const int64_t rows = (int64_t)pr->n_ch * pr->N;
    if (!panel_map(&q.tmx, X + off, rows, ncol) || (G && !panel_map(&q.tmg, G + off, rows, ncol)))
      return set_error(WPCD_ECUDA, "tensor map encoding failed");
    tiles->toff[g + 1] = tiles->toff[g] + pr->n_ch * q.n_cb;
    RTmax = std::max(RTmax, sh.RT);
  }
  const wpcd_problem *pr0 = gp[0].pr;
  wpcd_status st = launch_ws(*tiles, tiles->toff[n_prob], RTmax, G != nullptr, S != nullptr, pr0->d.tc_err,
                             pr0->device, s);
  if (st != WPCD_OK) return st;
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WPCD_OK : cuda_error(e, "tensor-core group gemm launch");
}

// nonzero if a tensor-core GEMM of this problem ran out of a wait limit
// since the last check or clear; the word is cleared for the next operation
wpcd_status tc_check(const wpcd_problem *pr, cudaStream_t s) {
  if (!pr->d.tc_err) return WPCD_OK;
  int h = 0;
  WPCD_CUDA_TRY(cudaMemcpyAsync(&h, pr->d.tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  WPCD_CUDA_TRY(cudaStreamSynchronize(s));
  if (!h) return WPCD_OK;
  WPCD_CUDA_TRY(cudaMemsetAsync(pr->d.tc_err, 0, sizeof(int), s));
  return set_error(WPCD_ETIMEOUT, "tensor-core GEMM wait limit reached");
}

// a clean error word at the start of an operation that ends in tc_check, so
// that a word left set by an operation that returned early is not reported
// against the next one
wpcd_status tc_clear(const wpcd_problem *pr, cudaStream_t s) {
  if (pr->d.tc_err) WPCD_CUDA_TRY(cudaMemsetAsync(pr->d.tc_err, 0, sizeof(int), s));
  return WPCD_OK;
}

}  // namespace wpcd
