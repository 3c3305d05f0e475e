// Step 2 of the numerical scheme (Sec. 3.3; Sec. 4.2): the lattice
// permutation matrix P0 of Eq. perm / Eq. gal, assembled on the device by
// quadrature-node binning, in two passes.  Values are summed in a fixed
// order (no floating-point atomics), so the result is bit-reproducible.
//
//   count pass  one CTA per source cell c = (i, j).  Every GL node (a, b, x)
//               of the cell is mapped through the recoupled momenta
//                 p'^2 = fma((0.75 p) q, y, (p p) 0.25 + (q q) 0.5625)
//                 q'^2 = fma(-(p q),     y, (p p) + (q q) 0.25)
//               (FP64, each product rounded on its own) and binned against
//               the squared edges held in shared memory (compared as int64
//               bit patterns: the order of non-negative doubles), by binary
//               search for the first y node of each (p, q) pair and short
//               walks for the rest (p'^2, q'^2 are monotone in y).  The
//               distinct targets (the paper's pre-selection) are counted in
//               a shared hash set and ranked; a stable counting sort by rank
//               leaves the packed keys (target << nbits | node) in ascending
//               order in global memory for the fill pass.
//   scan        exclusive scan of the counts -> row_ptr.
//   fill pass   one CTA per source cell.  The sorted keys are re-read; each
//               node's value w p^2 q^2 P_l(y) P_l'(y') is formed for every
//               (l, l') pair and summed per target by a block-wide segmented
//               scan (warp shuffles + a cross-warp carry), then normalised by
//               sqrt((2l+1)(2l'+1)) / sqrt(B_i Bq_j B_i' Bq_j') and written
//               to block-CSR (pair-major values).
//
// FP64 mode computes y' and the node values in FP64.  FP32C mode forms the
// recoupled squares from float pairs (FP64-class, rounded once to FP32),
// the rest in FP32, and accumulates with error-free transformations (TwoSum
// float-float pairs); only the binning uses FP64.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "wpcd_internal.h"

namespace wpcd {
namespace {

constexpr int kThreads = 256;  // count pass: threads per source cell
constexpr int kFill = 128;     // fill pass: threads per source cell (np2 / 128 sorted elements each)
constexpr uint32_t kInvalid = 0xFFFFFFFFu;

struct AsmParams {
  int N, M, n_p, n_q, n_x, n_nodes, np2, nbits, n_ch, n_pairs;
  uint64_t nx_magic;  // ceil(2^32 / n_x): node / n_x by a multiply and a shift
  int stage_rows;     // fill: rows staged in shared memory (the longest row), 0: direct writes
  int slot_bits;      // count pass: hash set of 2^slot_bits slots, filled to half at most
  int *err;           // count pass: set when a cell's distinct targets overflow the set
  int warp_runs;      // n_x a multiple of 32 and the y nodes ascending: a warp step is one
                      // (p, q) pair's consecutive y nodes, with monotone targets
  int pl[kMaxPairs], plp[kMaxPairs];
  double cnorm[kMaxPairs];  // sqrt((2l+1)(2l'+1))
  const double *pe2, *qe2, *pn, *wp, *qn, *wq, *yn, *wy, *rsb;
};

// shared-memory index of element n of a per-node array read both as runs of
// R consecutive elements per thread and as 32 consecutive elements per warp:
// one pad word per 32 puts the runs of the 32 lanes on distinct banks
__device__ __forceinline__ int pad32(int n) { return n + (n >> 5); }

// n / d for 0 <= n < 2^13 and d <= 2^13 from magic = ceil(2^32 / d): with
// magic d = 2^32 + r, 0 <= r < d, the product n magic / 2^32 exceeds n / d by
// n r / (d 2^32) < 1 / d, too little to reach the next integer
__device__ __forceinline__ int div_magic(int n, uint64_t magic) { return (int)(((uint64_t)n * magic) >> 32); }

__device__ __forceinline__ int bin_search(const long long *e2, int n, long long x) {
  // number of interior squared edges e2[1..n-1] that are <= x
  int lo = 0;
  int step = 1;
  while (step * 2 <= n - 1) step *= 2;
  for (; step >= 1; step >>= 1) {
    int cand = lo + step;
    lo = (cand <= n - 1 && e2[cand] <= x) ? cand : lo;
  }
  return lo;
}

// p'^2 = A y + Bp and q'^2 = C y + D for one (p, q) node pair
struct BinConst {
  double A, Bp, C, D;
};

constexpr int kWarps = kThreads / 32;

// exclusive prefix sum of v[0 .. n) in shared memory, in place; called by
// every thread after v is written, returns after a barrier
__device__ void block_exclusive_scan(int *v, int n, int *warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int chunk = (n + kThreads - 1) / kThreads;
  const int b = min(n, (int)threadIdx.x * chunk), e = min(n, b + chunk);
  int s = 0;
  for (int k = b; k < e; ++k) s += v[k];
  int incl = s;
  for (int d = 1; d < 32; d <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += u;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  int run = incl - s;
  for (int w = 0; w < warp; ++w) run += warp_tot[w];
  for (int k = b; k < e; ++k) {
    const int t = v[k];
    v[k] = run;
    run += t;
  }
  __syncthreads();
}

// insert a key into a shared hash set of 2^bits slots (multiplicative hash,
// linear probing; the set has at least twice as many slots as keys): the
// key's slot, fresh if it was not there yet
__device__ __forceinline__ int set_insert(uint32_t *table, int bits, uint32_t key, bool &fresh) {
  const uint32_t mask = (1u << bits) - 1u;
  uint32_t h = (key * 2654435761u) >> (32 - bits);
  fresh = false;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const uint32_t old = atomicCAS(&table[h], kInvalid, key);
    if (old == kInvalid) {
      fresh = true;
      return (int)h;
    }
    if (old == key) return (int)h;
    h = (h + 1) & mask;
  }
  return -1;
}

// Count pass of one source cell (R = np2 / kThreads nodes per thread).
// Every node is binned (thread t: nodes t R .. t R + R - 1, a binary search
// for the first node of each (p, q) pair, then walks along its y nodes);
// the distinct targets go into a shared hash set, each node keeping its
// target's slot; a target's rank is the number of smaller distinct targets;
// then a stable counting sort places the nodes rank by rank in node order
// (node n = warp * 32 R + k * 32 + lane here: within a warp by warp-match,
// across warps by per-(warp, rank) counts).  The result, the packed keys
// (target << nbits | node) in ascending order, is the one a full sort of
// the keys gives, without sorting them.
template <int R>
__global__ void __launch_bounds__(kThreads) count_kernel(AsmParams P, int64_t *counts, uint32_t *sorted) {
  extern __shared__ __align__(16) unsigned char smem[];
  long long *pe2 = reinterpret_cast<long long *>(smem);
  long long *qe2 = pe2 + (P.N + 1);
  BinConst *abk = reinterpret_cast<BinConst *>(qe2 + (P.M + 1));  // per (a, b)
  double *ys = reinterpret_cast<double *>(abk + P.n_p * P.n_q);
  // 2 S words: the hash set (S slots) and the ranks by slot, then the
  // per-warp counts [kWarps][S / 2] (a cell has at most S / 2 distinct targets)
  const int S = 1 << P.slot_bits, WS = S / 2;
  uint32_t *table = reinterpret_cast<uint32_t *>(ys + P.n_x);
  uint16_t *wc = reinterpret_cast<uint16_t *>(table);
  uint32_t *keys = table + 2 * S;                       // distinct targets, then the sorted keys
  int *off = reinterpret_cast<int *>(keys + P.np2 + P.np2 / 32);  // per-rank counts, then offsets
  __shared__ int n_distinct, n_fill, n_valid, overflow, warp_tot[kWarps];

  const int c = blockIdx.x;
  const int i = c / P.M, j = c % P.M;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int np2 = P.np2;
  for (int k = threadIdx.x; k <= P.N; k += kThreads) pe2[k] = __double_as_longlong(P.pe2[k]);
  for (int k = threadIdx.x; k <= P.M; k += kThreads) qe2[k] = __double_as_longlong(P.qe2[k]);
  for (int ab = threadIdx.x; ab < P.n_p * P.n_q; ab += kThreads) {
    int a = ab / P.n_q, b = ab % P.n_q;
    double p = P.pn[i * P.n_p + a], q = P.qn[j * P.n_q + b];
    // canonical rounding order of the recoupled squares (no contraction)
    double A = __dmul_rn(__dmul_rn(0.75, p), q);
    double Bp = __dadd_rn(__dmul_rn(__dmul_rn(p, p), 0.25), __dmul_rn(__dmul_rn(q, q), 0.5625));
    double C = -__dmul_rn(p, q);
    double D = __dadd_rn(__dmul_rn(p, p), __dmul_rn(__dmul_rn(q, q), 0.25));
    abk[ab] = BinConst{A, Bp, C, D};
  }
  for (int x = threadIdx.x; x < P.n_x; x += kThreads) ys[x] = P.yn[x];
  for (int k = threadIdx.x; k < S; k += kThreads) table[k] = kInvalid;
  if (threadIdx.x == 0) {
    n_distinct = 0;
    n_fill = 0;
    n_valid = 0;
    overflow = 0;
  }
  __syncthreads();
  // bin the nodes, thread t taking nodes t R .. t R + R - 1: consecutive y
  // nodes of one (p, q) pair, along which p'^2 and q'^2 are monotone, so
  // after a binary search for the first node of each pair the bins follow
  // by short walks (both directions: the y order is not assumed)
  const long long pmax2 = pe2[P.N], qmax2 = qe2[P.M];
  const int bits = P.slot_bits;
  // the distinct targets go into the hash set here too (once per run of
  // equal targets along the thread's nodes); each node keeps its slot
  uint32_t *tg = reinterpret_cast<uint32_t *>(off);  // targets by node index
  int *ts = reinterpret_cast<int *>(keys);           // their hash slots by node index
  {
    int bp = 0, bq = 0, prev_ab = -1, prev_slot = -1, my_valid = 0;
    uint32_t prev_t = kInvalid;
#pragma unroll 1
    for (int k = 0; k < R; ++k) {
      const int n = (int)threadIdx.x * R + k;
      uint32_t t = kInvalid;
      if (n < P.n_nodes) {
        const int ab = div_magic(n, P.nx_magic);
        const BinConst bc = abk[ab];
        const double y = ys[n - ab * P.n_x];
        const long long xp = __double_as_longlong(__fma_rn(bc.A, y, bc.Bp));
        const long long xq = __double_as_longlong(__fma_rn(bc.C, y, bc.D));
        if (ab != prev_ab) {
          bp = bin_search(pe2, P.N, xp);
          bq = bin_search(qe2, P.M, xq);
          prev_ab = ab;
        } else {
          while (bp < P.N - 1 && pe2[bp + 1] <= xp) ++bp;
          while (bp > 0 && pe2[bp] > xp) --bp;
          while (bq < P.M - 1 && qe2[bq + 1] <= xq) ++bq;
          while (bq > 0 && qe2[bq] > xq) --bq;
        }
        if (xp <= pmax2 && xq <= qmax2) t = (uint32_t)(bp * P.M + bq);
      }
      int sl = -1;
      if (t != kInvalid) {
        ++my_valid;
        if (t == prev_t) {
          sl = prev_slot;
        } else {
          bool fresh;
          sl = set_insert(table, bits, t, fresh);
          if (fresh) atomicAdd(&n_distinct, 1);
          if (sl < 0) overflow = 1;
        }
      }
      prev_t = t;
      prev_slot = sl;
      tg[pad32(n)] = t;
      ts[pad32(n)] = sl;
    }
    if (my_valid) atomicAdd(&n_valid, my_valid);
  }
  __syncthreads();
  // node n = warp * 32 R + k * 32 + lane from here on, so that each warp
  // holds consecutive nodes
  uint32_t tgt[R];
  int slot[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    tgt[k] = tg[pad32(warp * 32 * R + k * 32 + lane)];
    slot[k] = ts[pad32(warp * 32 * R + k * 32 + lane)];
  }
  __syncthreads();
  // the distinct targets (list) with their slots; the rank of each is the
  // number of smaller ones (a row has tens to a few hundred), stored by slot
  const int nr = n_distinct;
  if (overflow || nr > WS) {  // uniform (shared values after a barrier): the host reruns with a larger set
    if (threadIdx.x == 0) {
      atomicOr(P.err, 1);
      counts[c] = 0;
    }
    return;
  }
  uint32_t *rank_of = table + S;  // by slot
  int *lslot = off;                      // the targets by node index are in registers now
  for (int k = threadIdx.x; k < S; k += kThreads) {
    const uint32_t v = table[k];
    if (v != kInvalid) {
      const int at = atomicAdd(&n_fill, 1);
      keys[at] = v;
      lslot[at] = k;
    }
  }
  __syncthreads();
  for (int m = threadIdx.x; m < nr; m += kThreads) {
    const uint32_t v = keys[m];
    int r = 0;
    for (int q = 0; q < nr; ++q) r += keys[q] < v ? 1 : 0;
    rank_of[lslot[m]] = (uint32_t)r;
  }
  __syncthreads();
  int rk[R];
#pragma unroll
  for (int k = 0; k < R; ++k) rk[k] = slot[k] >= 0 ? (int)rank_of[slot[k]] : -1;
  __syncthreads();
  // the hash set is dead: per-warp counts per rank in its place
  for (int r = threadIdx.x; r < nr; r += kThreads)
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wc[w * WS + r] = 0;
  __syncthreads();
  // within the warp: nodes of one rank in lane order, k by k.  When n_x is
  // a multiple of 32 the lanes of a step are consecutive y nodes of one
  // (p, q) pair, whose targets are monotone, so the lanes of one rank are
  // contiguous and found from the run heads; else by warp-match
  const unsigned lower = (1u << lane) - 1u;
  const bool contiguous = P.warp_runs != 0;
  int lp[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int r = rk[k];
    unsigned peers;
    if (contiguous) {
      const int up = __shfl_up_sync(0xffffffffu, r, 1);
      const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || up != r);
      const unsigned le = lower | (1u << lane);
      const int h = 31 - __clz(heads & le);                       // my run's head
      const unsigned after = heads & ~le;                           // heads after me
      const int e = after ? __ffs(after) - 1 : 32;                  // next run's head
      peers = (e >= 32 ? 0xffffffffu : ((1u << e) - 1u)) & ~((1u << h) - 1u);
    } else {
      peers = __match_any_sync(0xffffffffu, r);
    }
    const int base = r >= 0 ? (int)wc[warp * WS + r] : 0;
    __syncwarp();
    if (r >= 0 && (peers & lower) == 0) wc[warp * WS + r] = (uint16_t)(base + __popc(peers));
    __syncwarp();
    lp[k] = base + __popc(peers & lower);
  }
  __syncthreads();
  // per rank: the offsets of the warps within the rank, and its node count
  for (int r = threadIdx.x; r < nr; r += kThreads) {
    int s = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const int t = wc[w * WS + r];
      wc[w * WS + r] = (uint16_t)s;
      s += t;
    }
    off[r] = s;
  }
  __syncthreads();
  block_exclusive_scan(off, nr, warp_tot);
  // place the keys; the invalid nodes fill the tail
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int r = rk[k];
    if (r >= 0) {
      const int n = warp * 32 * R + k * 32 + lane;
      keys[off[r] + wc[warp * WS + r] + lp[k]] = (tgt[k] << P.nbits) | (uint32_t)n;
    }
  }
  for (int k = n_valid + threadIdx.x; k < np2; k += kThreads) keys[k] = kInvalid;
  __syncthreads();
  for (int k = threadIdx.x; k < np2; k += kThreads) sorted[(size_t)c * np2 + k] = keys[k];
  if (threadIdx.x == 0) {
    counts[c] = nr;
    atomicMax(reinterpret_cast<unsigned long long *>(counts + P.N * P.M), (unsigned long long)nr);  // longest row
  }
}

// single-CTA exclusive scan of n counts into row_ptr[n + 1]
__global__ void __launch_bounds__(1024) scan_kernel(const int64_t *counts, int n, int64_t *row_ptr) {
  __shared__ int64_t part[1024];
  const int T = 1024;
  int chunk = (n + T - 1) / T;
  int b = threadIdx.x * chunk, e = min(n, b + chunk);
  int64_t s = 0;
  for (int k = b; k < e; ++k) s += counts[k];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < T; off <<= 1) {
    int64_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = part[threadIdx.x] - s;
  for (int k = b; k < e; ++k) {
    row_ptr[k] = run;
    run += counts[k];
  }
  if (threadIdx.x == T - 1) row_ptr[n] = part[T - 1];
}

// ---- accumulators -----------------------------------------------------------
struct Acc64 {
  double v;
  __device__ void zero() { v = 0.0; }
  __device__ void fma(double a, double b) { v = ::fma(a, b, v); }
  __device__ void add(const Acc64 &o) { v += o.v; }
  __device__ double value() const { return v; }
  __device__ double result() const { return v; }
  __device__ Acc64 shfl_up(int d) const { Acc64 r; r.v = __shfl_up_sync(0xffffffffu, v, d); return r; }
};

// float-float accumulator (Knuth TwoSum): hi + lo carries the sum exactly
// up to the rounding of lo
struct AccFF {
  float hi, lo;
  __device__ void zero() { hi = 0.f; lo = 0.f; }
  __device__ static void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  }
  __device__ void add(float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ void fma(float a, float b) { add(__fmul_rn(a, b)); }
  __device__ void add(const AccFF &o) {
    float s, e;
    two_sum(hi, o.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, o.lo));
    two_sum(s, e, hi, lo);
  }
  __device__ double value() const { return (double)hi + (double)lo; }
  __device__ float result() const { return __fadd_rn(hi, lo); }  // rounded once to FP32
  __device__ AccFF shfl_up(int d) const {
    AccFF r;
    r.hi = __shfl_up_sync(0xffffffffu, hi, d);
    r.lo = __shfl_up_sync(0xffffffffu, lo, d);
    return r;
  }
};

template <bool F64>
struct NodeVal;
template <>
struct NodeVal<true> {
  using real = double;
  using Acc = Acc64;
};
template <>
struct NodeVal<false> {
  using real = float;
  using Acc = AccFF;
};

// P_0 .. P_{NCH-1} at y by the three-term recurrence
template <typename real, int NCH>
__device__ __forceinline__ void legendre_n(real y, real *P) {
  P[0] = real(1);
  if (NCH > 1) P[1] = y;
#pragma unroll
  for (int n = 1; n + 1 < NCH; ++n)
    P[n + 1] = (real(2 * n + 1) / real(n + 1)) * y * P[n] - (real(n) / real(n + 1)) * P[n - 1];
}

__device__ __forceinline__ float mul_r(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_r(double a, double b) { return __dmul_rn(a, b); }

// a b + c in the operands' own precision (no promotion of floats to double)
__device__ __forceinline__ float fma_r(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return __fma_rn(a, b, c); }

// W P_0 .. W P_{NCH-1} at y (the weight folded into the recurrence; hW =
// W / 2, the term P_0 / 2 of the first step, given)
template <typename real, int NCH>
__device__ __forceinline__ void legendre_w(real y, real W, real hW, real *P) {
  P[0] = W;
  if (NCH > 1) P[1] = W * y;
  if (NCH > 2) P[2] = fma_r(real(1.5) * y, P[1], -hW);
#pragma unroll
  for (int n = 2; n + 1 < NCH; ++n)
    P[n + 1] = (real(2 * n + 1) / real(n + 1)) * y * P[n] - (real(n) / real(n + 1)) * P[n - 1];
}

// 1/sqrt(d) for d > 0 in FP64 by one Newton-Raphson step r <- r + r (1 -
// d r^2) / 2 from the FP32 reciprocal square root of d: for a seed with
// relative error e the step leaves about 1.5 e^2 (the seed is within 3e-7,
// so the result within about 2e-13).  The seed's float is formed from d's
// exponent and leading mantissa bits, and the FP32 result widened, by
// integer operations, so that no conversion occupies the FP64 pipe; d
// outside 2^-99 .. 2^99 takes the FP64 rsqrt
__device__ __forceinline__ double rsqrt_newton(double d) {
  const long long b = __double_as_longlong(d);
  const int ex = (int)((b >> 52) & 0x7ff) - 1023;
  if (ex < -99 || ex > 99) return rsqrt(d);
  const unsigned fb = ((unsigned)(ex + 127) << 23) | (unsigned)((b >> 29) & 0x7fffff);
  const unsigned rb = __float_as_uint(rsqrtf(__uint_as_float(fb)));
  const double r = __longlong_as_double(((long long)((int)((rb >> 23) & 0xff) - 127 + 1023) << 52) |
                                        ((long long)(rb & 0x7fffff) << 29));
  const double e = fma(-(d * r), r, 1.0);  // 1 - d r^2
  // r / 2 by decrementing the exponent (r is normal): no FP64 multiply
  const double half_r = __longlong_as_double(__double_as_longlong(r) - (1LL << 52));
  return fma(half_r, e, r);
}

// Per (p, q) node pair constants of one source cell (FP64):
//   p'^2 = A y + Bp,  q'^2 = C y + D,  p'.q' = nA y + nB,  and the weight
//   wp wq.  Shared by the n_x y-nodes of the pair.
struct __align__(16) PairConst {
  double A, Bp, C, D, nA, nB, W, hW;  // hW = W / 2
};

// The FP32C form: each FP64 constant as an unevaluated float pair hi + lo
// (hi the nearest float, lo the nearest float to the rest: 48 bits)
struct __align__(16) PairConstF {
  float Ah, Al, Bh, Bl, Ch, Cl, Dh, Dl, nAh, nAl, nBh, nBl, W, hW, pad[2];
};

__device__ __forceinline__ float2 split_ff(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

// float-pair arithmetic (hi + lo, |lo| <= ulp(hi) / 2; intrinsics, so no
// contraction): products by Dekker's TwoProduct (FMA), sums by Knuth's TwoSum
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, __fmaf_rn(a.x, b.x, -p)));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ float2 ff_mul_f(float2 a, float b) {
  const float p = __fmul_rn(a.x, b);
  return fast_two_sum(p, __fmaf_rn(a.y, b, __fmaf_rn(a.x, b, -p)));
}
__device__ __forceinline__ float2 ff_scale2(float2 a, float pow2) {  // exact
  return make_float2(a.x * pow2, a.y * pow2);
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  return fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}

// a y + b for float pairs a, y, b, rounded to a float: the product of the
// high parts exactly (Dekker's TwoProduct by FMA), its sum with b's high
// part exactly (Knuth's TwoSum), then the small terms; the result is the
// FP64-class value rounded once to FP32 (intrinsics: no contraction)
__device__ __forceinline__ float ff_mad(float ah, float al, float yh, float yl, float bh, float bl) {
  const float ph = __fmul_rn(ah, yh);
  const float pl = __fmaf_rn(ah, yh, -ph);
  const float sh = __fadd_rn(ph, bh);
  const float bb = __fsub_rn(sh, ph);
  const float e = __fadd_rn(__fsub_rn(ph, __fsub_rn(sh, bb)), __fsub_rn(bh, bb));
  float t = __fmaf_rn(ah, yl, pl);
  t = __fmaf_rn(al, yh, t);
  t = __fadd_rn(t, __fadd_rn(bl, e));
  return __fadd_rn(sh, t);
}

template <bool F64, int NCH>
__global__ void __launch_bounds__(kFill) fill_kernel(AsmParams P, const uint32_t *sorted,
                                                        const int64_t *row_ptr, int32_t *col,
                                                        typename NodeVal<F64>::real *val,
                                                        int64_t nnz) {
  using real = typename NodeVal<F64>::real;
  using Acc = typename NodeVal<F64>::Acc;
  constexpr int NPAIR = pair_count(NCH);
  extern __shared__ __align__(16) unsigned char smem[];
  PairConst *pc = reinterpret_cast<PairConst *>(smem);            // [n_p * n_q] (FP64)
  PairConstF *pcf = reinterpret_cast<PairConstF *>(smem);         // [n_p * n_q] (FP32C)
  float2 *ysp = reinterpret_cast<float2 *>(pc + P.n_p * P.n_q);   // y as a float pair [n_x]
  real *Pyw = reinterpret_cast<real *>(ysp + P.n_x);               // w_y P_l(y) [n_x][NCH]
  uint32_t *keys = reinterpret_cast<uint32_t *>(Pyw + P.n_x * NCH + 2);  // [np2]
  // the row's staged sums [stage_rows][NPAIR] and targets [stage_rows]
  real *st_val =
      reinterpret_cast<real *>((reinterpret_cast<uintptr_t>(keys + P.np2 + P.np2 / 32) + 15) & ~(uintptr_t)15);
  int32_t *st_col = reinterpret_cast<int32_t *>(st_val + (size_t)P.stage_rows * NPAIR);
  __shared__ Acc wtot[kFill / 32][NPAIR];
  __shared__ int wflag[kFill / 32];
  __shared__ int whead[kFill / 32];

  const int c = blockIdx.x;
  const int i = c / P.M, j = c % P.M;
  const int R = P.np2 / kFill;  // consecutive sorted elements per thread
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t mask = (1u << P.nbits) - 1u;
  const int nbits = P.nbits;

  for (int ab = threadIdx.x; ab < P.n_p * P.n_q; ab += kFill) {
    int a = ab / P.n_q, b = ab % P.n_q;
    double p = P.pn[i * P.n_p + a], q = P.qn[j * P.n_q + b];
    if (!F64) {
      // the same constants in float-pair arithmetic from p and q split
      // once (FP64-class, a handful of FP64 instructions per pair)
      const float2 pf = split_ff(p), qf = split_ff(q);
      const float2 pp = ff_mul(pf, pf), qq = ff_mul(qf, qf), pq = ff_mul(pf, qf);
      const float2 A = ff_mul_f(pq, 0.75f);
      const float2 Bp = ff_add(ff_scale2(pp, 0.25f), ff_mul_f(qq, 0.5625f));
      const float2 D = ff_add(pp, ff_scale2(qq, 0.25f));
      const float2 nB = ff_add(ff_mul_f(qq, 0.375f), ff_scale2(pp, -0.5f));
      PairConstF f;
      f.Ah = A.x, f.Al = A.y;
      f.Bh = Bp.x, f.Bl = Bp.y;
      f.Ch = -pq.x, f.Cl = -pq.y;
      f.Dh = D.x, f.Dl = D.y;
      f.nAh = -0.5f * pq.x, f.nAl = -0.5f * pq.y;
      f.nBh = nB.x, f.nBl = nB.y;
      f.W = (float)P.wp[i * P.n_p + a] * (float)P.wq[j * P.n_q + b];
      f.hW = 0.5f * f.W;
      pcf[ab] = f;
      continue;
    }
    PairConst k;
    k.A = __dmul_rn(__dmul_rn(0.75, p), q);
    k.Bp = __dadd_rn(__dmul_rn(__dmul_rn(p, p), 0.25), __dmul_rn(__dmul_rn(q, q), 0.5625));
    k.C = -__dmul_rn(p, q);
    k.D = __dadd_rn(__dmul_rn(p, p), __dmul_rn(__dmul_rn(q, q), 0.25));
    k.nA = -0.5 * p * q;
    k.nB = 0.375 * q * q - 0.5 * p * p;
    k.W = P.wp[i * P.n_p + a] * P.wq[j * P.n_q + b];
    k.hW = 0.5 * k.W;
    pc[ab] = k;
  }
  for (int x = threadIdx.x; x < P.n_x; x += kFill) {
    real Pl[NCH];
    legendre_n<real, NCH>((real)P.yn[x], Pl);
#pragma unroll
    for (int l = 0; l < NCH; ++l) Pyw[x * NCH + l] = (real)P.wy[x] * Pl[l];
    ysp[x] = split_ff(P.yn[x]);
  }
  // keys at pad32(n): each thread reads a run of R consecutive keys
  for (int n = threadIdx.x; n < P.np2; n += kFill) keys[pad32(n)] = sorted[(size_t)c * P.np2 + n];
  __syncthreads();

  auto is_head = [&](int e) {
    uint32_t k = keys[pad32(e)];
    return k != kInvalid && (e == 0 || (keys[pad32(e - 1)] >> nbits) != (k >> nbits));
  };
  // add the contributions of sorted element e to every (l, l') pair:
  // acc[m] += (w_y P_l(y)) (W_pq P_l'(y')), the first factor from a table
  // the two factors of every pair's term of element e: Pyw row x, W P_l'(y')
  auto factors = [&](int e, real *WPl2) -> int {
    const int node = (int)(keys[pad32(e)] & mask);
    const int ab = div_magic(node, P.nx_magic), x = node - ab * P.n_x;
    real yp, W, hW;
    if (F64) {
      const PairConst &k = pc[ab];
      const double y = P.yn[x];
      double p2 = fma(k.A, y, k.Bp), q2 = fma(k.C, y, k.D), num = fma(k.nA, y, k.nB);
      double den2 = p2 * q2;  // both >= 0 up to rounding; guarded below (sign by the bits)
      yp = __double_as_longlong(den2) > 0 ? num * rsqrt_newton(den2) : 0.0;
      W = k.W;
      hW = k.hW;
    } else {
      // recoupled squares and p'.q' to FP64-class accuracy from float pairs
      // (no FP64 instruction), each rounded once to FP32; the rest in FP32
      const PairConstF &k = pcf[ab];
      const float2 y = ysp[x];
      const float p2 = ff_mad(k.Ah, k.Al, y.x, y.y, k.Bh, k.Bl);
      const float q2 = ff_mad(k.Ch, k.Cl, y.x, y.y, k.Dh, k.Dl);
      const float num = ff_mad(k.nAh, k.nAl, y.x, y.y, k.nBh, k.nBl);
      float den2 = p2 * q2;
      float cc = den2 > 0.f ? num * rsqrtf(den2) : 0.f;
      yp = (real)fminf(1.f, fmaxf(-1.f, cc));
      W = k.W;
      hW = k.hW;
    }
    legendre_w<real, NCH>(yp, W, hW, WPl2);
    return x;
  };
  auto accumulate = [&](int e, Acc *acc) {
    real WPl2[NCH];  // W_pq P_l'(y')
    const int x = factors(e, WPl2);
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) acc[m].fma(Pyw[x * NCH + pair_first(NCH, m)], WPl2[pair_second(NCH, m)]);
  };
  // FP32C: the rounded products of element e (AccFF::fma adds the same)
  auto products = [&](int e, real *v) {
    real WPl2[NCH];
    const int x = factors(e, WPl2);
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) v[m] = mul_r(Pyw[x * NCH + pair_first(NCH, m)], WPl2[pair_second(NCH, m)]);
  };

  // step A: segment ranks from an integer scan of the head flags
  const int e0 = threadIdx.x * R;
  int nhead = 0;
  for (int r = 0; r < R; ++r) nhead += is_head(e0 + r) ? 1 : 0;
  int hscan = nhead;
  for (int d = 1; d < 32; d <<= 1) {
    int hu = __shfl_up_sync(0xffffffffu, hscan, d);
    if (lane >= d) hscan += hu;
  }
  if (lane == 31) whead[warp] = hscan;
  __syncthreads();
  int hbase = 0;
  for (int w = 0; w < warp; ++w) hbase += whead[w];
  const int seg0 = hbase + hscan - nhead;  // heads before this thread
  const int64_t base = row_ptr[c];
  const int64_t lim = row_ptr[c + 1];
  const double rs_src = P.rsb[c];

  const bool staged = P.stage_rows > 0;
  auto write_seg = [&](int seg, uint32_t k, const Acc *sum) {
    int64_t o = base + seg;
    if (staged) {
      if (o < lim) {
        st_col[seg] = (int32_t)(k >> nbits);
#pragma unroll
        for (int m = 0; m < NPAIR; ++m) st_val[seg * NPAIR + m] = sum[m].result();
      }
    } else if (o < lim) {
      int t = (int)(k >> nbits);
      col[o] = t;
      double nrm = rs_src * P.rsb[t];
#pragma unroll
      for (int m = 0; m < NPAIR; ++m) val[(size_t)m * nnz + o] = (real)(sum[m].value() * nrm * P.cnorm[m]);
    }
  };

  // step B: one pass over my elements; segments that open and close here are
  // written at once, the leading one (continuing from earlier threads) waits
  Acc run[NPAIR], lead[NPAIR];
#pragma unroll
  for (int m = 0; m < NPAIR; ++m) {
    run[m].zero();
    lead[m].zero();
  }
  int flag = 0, local_heads = 0, lead_tail = 0;
  uint32_t lead_key = 0;
  // a window of (previous, current) keys: one shared-memory load per element
  uint32_t kprev = e0 > 0 ? keys[pad32(e0 - 1)] : kInvalid, k = keys[pad32(e0)];
  // FP32C: the next element's products are formed while the current one is
  // added (independent work for the scheduler); same sums as AccFF::fma
  real v_cur[NPAIR], v_nxt[NPAIR];
  if constexpr (!F64) {
    if (k != kInvalid) products(e0, v_cur);
  }
  for (int r = 0; r < R; ++r) {
    const int e = e0 + r;
    if (k == kInvalid) break;
    const uint32_t knext = e + 1 < P.np2 ? keys[pad32(e + 1)] : kInvalid;
    const uint32_t tk = k >> nbits;
    if constexpr (!F64) {
      if (r + 1 < R && knext != kInvalid) products(e + 1, v_nxt);
    }
    if (e == 0 || (kprev >> nbits) != tk) {
      flag = 1;
      ++local_heads;
#pragma unroll
      for (int m = 0; m < NPAIR; ++m) run[m].zero();
    }
    if constexpr (F64) {
      accumulate(e, run);
    } else {
#pragma unroll
      for (int m = 0; m < NPAIR; ++m) run[m].add(v_cur[m]);
    }
    if (knext == kInvalid || (knext >> nbits) != tk) {
      if (flag) {
        write_seg(seg0 + local_heads - 1, k, run);
      } else {
#pragma unroll
        for (int m = 0; m < NPAIR; ++m) lead[m] = run[m];
        lead_tail = 1;
        lead_key = k;
      }
    }
    kprev = k;
    k = knext;
    if constexpr (!F64) {
#pragma unroll
      for (int m = 0; m < NPAIR; ++m) v_cur[m] = v_nxt[m];
    }
  }
  // step C: segmented scan of (flag, sum of the segment open at my end)
  Acc agg[NPAIR];
#pragma unroll
  for (int m = 0; m < NPAIR; ++m) agg[m] = run[m];
  int f = flag;
  for (int d = 1; d < 32; d <<= 1) {
    int fu = __shfl_up_sync(0xffffffffu, f, d);
    Acc su[NPAIR];
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) su[m] = agg[m].shfl_up(d);
    if (lane >= d) {
      if (!f) {
#pragma unroll
        for (int m = 0; m < NPAIR; ++m) agg[m].add(su[m]);
      }
      f |= fu;
    }
  }
  if (lane == 31) {
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) wtot[warp][m] = agg[m];
    wflag[warp] = f;
  }
  __syncthreads();
  Acc carry[NPAIR];
#pragma unroll
  for (int m = 0; m < NPAIR; ++m) carry[m].zero();
  int cflag = 0;
  for (int w = warp - 1; w >= 0 && !cflag; --w) {
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) carry[m].add(wtot[w][m]);
    cflag = wflag[w];
  }
  if (!f) {
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) agg[m].add(carry[m]);
  }
  // exclusive value for this thread = inclusive value of the previous one
  Acc excl[NPAIR];
#pragma unroll
  for (int m = 0; m < NPAIR; ++m) excl[m] = agg[m].shfl_up(1);
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) excl[m] = carry[m];
  }
  // step D: close the leading segment with the carry from earlier threads
  if (lead_tail) {
#pragma unroll
    for (int m = 0; m < NPAIR; ++m) lead[m].add(excl[m]);
    write_seg(seg0 - 1, lead_key, lead);
  }
  if (!staged) return;  // uniform over the CTA
  // normalise and write the row: consecutive threads, consecutive elements
  __syncthreads();
  const int n_seg = (int)(lim - base);
  for (int sg = threadIdx.x; sg < n_seg; sg += kFill) col[base + sg] = st_col[sg];
  for (int idx = threadIdx.x; idx < n_seg * NPAIR; idx += kFill) {
    const int m = idx / n_seg, sg = idx - m * n_seg;
    const double scale = rs_src * P.rsb[st_col[sg]] * P.cnorm[m];
    val[(size_t)m * nnz + base + sg] = (real)((double)st_val[sg * NPAIR + m] * scale);
  }
}

template <int R>
cudaError_t launch_count(const AsmParams &P, int n_cells, size_t smem, cudaStream_t s, int64_t *counts,
                         uint32_t *sorted) {
  cudaError_t e = cudaFuncSetAttribute(count_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_kernel<R><<<n_cells, kThreads, smem, s>>>(P, counts, sorted);
  return cudaGetLastError();
}

template <bool F64, int NCH>
void launch_fill(const AsmParams &P, int n_cells, size_t smem, cudaStream_t s, const uint32_t *sorted,
                 const int64_t *row_ptr, int32_t *col, void *val, int64_t nnz) {
  using real = typename NodeVal<F64>::real;
  auto kern = fill_kernel<F64, NCH>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<n_cells, kFill, smem, s>>>(P, sorted, row_ptr, col, reinterpret_cast<real *>(val), nnz);
}

template <bool F64>
wpcd_status dispatch_fill(const AsmParams &P, int n_cells, size_t smem, cudaStream_t s,
                          const uint32_t *sorted, const int64_t *row_ptr, int32_t *col, void *val,
                          int64_t nnz) {
  switch (P.n_ch) {
    case 1: launch_fill<F64, 1>(P, n_cells, smem, s, sorted, row_ptr, col, val, nnz); break;
    case 2: launch_fill<F64, 2>(P, n_cells, smem, s, sorted, row_ptr, col, val, nnz); break;
    case 3: launch_fill<F64, 3>(P, n_cells, smem, s, sorted, row_ptr, col, val, nnz); break;
    case 4: launch_fill<F64, 4>(P, n_cells, smem, s, sorted, row_ptr, col, val, nnz); break;
    case 5: launch_fill<F64, 5>(P, n_cells, smem, s, sorted, row_ptr, col, val, nnz); break;
    default: return set_error(WPCD_EINVAL, "unsupported number of channels");
  }
  return WPCD_OK;
}

}  // namespace

wpcd_status assemble(wpcd_grid *g, int n_ch, int prec, cudaStream_t s, wpcd_P **out) {
  if (prec != WPCD_FP64 && prec != WPCD_FP32C) return set_error(WPCD_EINVAL, "prec must be WPCD_FP64 or WPCD_FP32C");
  if (n_ch < 1 || n_ch > 5) return set_error(WPCD_EINVAL, "n_ch must be in [1, 5]");
  WPCD_CUDA_TRY(cudaSetDevice(g->device));
  AsmParams P{};
  P.N = g->N;
  P.M = g->M;
  P.n_p = g->n_p;
  P.n_q = g->n_q;
  P.n_x = g->n_x;
  P.n_nodes = g->n_p * g->n_q * g->n_x;
  P.nx_magic = ((1ull << 32) + (uint64_t)g->n_x - 1) / (uint64_t)g->n_x;
  P.warp_runs = g->n_x % 32 == 0 && g->y_ascending;
  int np2 = kThreads;
  while (np2 < P.n_nodes) np2 *= 2;
  P.np2 = np2;
  int nbits = 0;
  while ((1 << nbits) < np2) ++nbits;
  P.nbits = nbits;
  P.n_ch = n_ch;
  P.n_pairs = pair_count(n_ch);
  for (int m = 0; m < P.n_pairs; ++m) {
    P.pl[m] = pair_first(n_ch, m);
    P.plp[m] = pair_second(n_ch, m);
    P.cnorm[m] = sqrt((2.0 * P.pl[m] + 1.0) * (2.0 * P.plp[m] + 1.0));
  }
  P.pe2 = g->pe2;
  P.qe2 = g->qe2;
  P.pn = g->pn;
  P.wp = g->wp;
  P.qn = g->qn;
  P.wq = g->wq;
  P.yn = g->yn;
  P.wy = g->wy;
  P.rsb = g->rsb;
  const int n_cells = P.N * P.M;
  if (np2 > 8192) return set_error(WPCD_EINVAL, "too many quadrature nodes per cell (max 8192)");
  if ((int64_t)n_cells << nbits >= (int64_t)1 << 32)
    return set_error(WPCD_EINVAL, "lattice too large for 32-bit packed node keys");

  cudaEvent_t ev0, ev1, evc, evs;
  WPCD_CUDA_TRY(cudaEventCreate(&ev0));
  WPCD_CUDA_TRY(cudaEventCreate(&ev1));
  WPCD_CUDA_TRY(cudaEventCreate(&evc));
  WPCD_CUDA_TRY(cudaEventCreate(&evs));
  int64_t *counts = nullptr;
  uint32_t *sorted = nullptr;
  wpcd_P *Pm = new wpcd_P();
  Pm->grid = g;
  Pm->device = g->device;
  Pm->n_ch = n_ch;
  Pm->prec = prec;
  Pm->n_pairs = P.n_pairs;
  Pm->work = (int64_t)n_cells * P.n_nodes;  // every node of every cell mapped once
  auto fail = [&](wpcd_status st) {
    dev_free(counts);
    dev_free(sorted);
    dev_free(Pm->row_ptr);
    dev_free(Pm->col);
    dev_free(Pm->val64);
    dev_free(Pm->val32);
    delete Pm;
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaEventDestroy(evc);
    cudaEventDestroy(evs);
    return st;
  };
  cudaError_t e;
  // counts[n_cells]: the longest row; counts[n_cells + 1]: the overflow word
  if ((e = dev_malloc(&counts, sizeof(int64_t) * (n_cells + 2))) != cudaSuccess)
    return fail(cuda_error(e, "cudaMalloc counts"));
  if ((e = dev_malloc(&sorted, sizeof(uint32_t) * (size_t)n_cells * np2)) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc sorted keys"));
  if ((e = dev_malloc(&Pm->row_ptr, sizeof(int64_t) * (n_cells + 1))) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc row_ptr"));

  cudaEventRecord(ev0, s);
  // the count pass's hash set: 4 (N + M) slots (at least 512), which the
  // distinct targets of a cell fill to half at most in practice; a cell
  // that overflows it sets the error word and the pass runs again with
  // 2 np2 slots, which no cell can overflow (it has at most np2 targets)
  int full_bits = 1;
  while ((1 << full_bits) < 2 * np2) ++full_bits;
  int bits0 = 9;
  while ((1 << bits0) < 4 * (P.N + P.M) && bits0 < full_bits) ++bits0;
  if (bits0 > full_bits) bits0 = full_bits;
  P.err = reinterpret_cast<int *>(counts + n_cells + 1);
  int64_t nnz = 0, longest = 0;
  for (int attempt = 0;; ++attempt) {
    P.slot_bits = attempt == 0 ? bits0 : full_bits;
    // edges, node constants, y nodes; hash set and ranks (2 S words, then
    // the per-warp counts), keys and per-rank offsets (np2 + np2 / 32 each)
    const size_t smem_count = sizeof(long long) * (P.N + P.M + 2) + sizeof(BinConst) * P.n_p * P.n_q +
                              sizeof(double) * P.n_x +
                              sizeof(uint32_t) * (2 * ((size_t)1 << P.slot_bits) + 2 * (size_t)np2 + np2 / 16);
    if (smem_count > 227 * 1024)
      return fail(set_error(WPCD_EINVAL, "lattice edges and node count exceed shared memory"));
    if ((e = cudaMemsetAsync(counts + n_cells, 0, 2 * sizeof(int64_t), s)) != cudaSuccess)
      return fail(cuda_error(e, "counts clear"));
    switch (np2 / kThreads) {
      case 1: e = launch_count<1>(P, n_cells, smem_count, s, counts, sorted); break;
      case 2: e = launch_count<2>(P, n_cells, smem_count, s, counts, sorted); break;
      case 4: e = launch_count<4>(P, n_cells, smem_count, s, counts, sorted); break;
      case 8: e = launch_count<8>(P, n_cells, smem_count, s, counts, sorted); break;
      case 16: e = launch_count<16>(P, n_cells, smem_count, s, counts, sorted); break;
      default: e = launch_count<32>(P, n_cells, smem_count, s, counts, sorted); break;
    }
    if (e != cudaSuccess) return fail(cuda_error(e, "count pass launch"));
    cudaEventRecord(evc, s);
    scan_kernel<<<1, 1024, 0, s>>>(counts, n_cells, Pm->row_ptr);
    cudaEventRecord(evs, s);
    count_launches(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_error(e, "count/scan launch"));
    int64_t flag = 0;
    if ((e = cudaMemcpyAsync(&nnz, Pm->row_ptr + n_cells, sizeof(int64_t), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(&longest, counts + n_cells, sizeof(int64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&flag, counts + n_cells + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
      return fail(cuda_error(e, "nnz readback"));
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(cuda_error(e, "count pass"));
    if (!flag) break;
    if (P.slot_bits == full_bits) return fail(set_error(WPCD_ECUDA, "count pass: hash set overflow"));
  }
  Pm->nnz = nnz;
  size_t nz = nnz > 0 ? (size_t)nnz : 1;
  if ((e = dev_malloc(&Pm->col, sizeof(int32_t) * nz)) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc col"));
  void *val = nullptr;
  if (prec == WPCD_FP64) {
    if ((e = dev_malloc(&Pm->val64, sizeof(double) * nz * P.n_pairs)) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc val"));
    val = Pm->val64;
  } else {
    if ((e = dev_malloc(&Pm->val32, sizeof(float) * nz * P.n_pairs)) != cudaSuccess) return fail(cuda_error(e, "cudaMalloc val"));
    val = Pm->val32;
  }
  size_t rsz = prec == WPCD_FP64 ? sizeof(double) : sizeof(float);
  size_t smem_fill = sizeof(PairConst) * (size_t)P.n_p * P.n_q + sizeof(float2) * P.n_x +
                     rsz * ((size_t)P.n_x * P.n_ch + 2) + sizeof(uint32_t) * (np2 + np2 / 32);
  smem_fill = (smem_fill + 15) & ~(size_t)15;
  // each row's sums staged in shared memory (values, target), then
  // normalised and written by all threads together, when the longest fits
  const size_t stage = 16 + (size_t)longest * ((size_t)P.n_pairs * rsz + sizeof(int32_t));
  P.stage_rows = smem_fill + stage <= 200 * 1024 ? (int)longest : 0;
  if (P.stage_rows) smem_fill += stage;
  wpcd_status st = prec == WPCD_FP64
                       ? dispatch_fill<true>(P, n_cells, smem_fill, s, sorted, Pm->row_ptr, Pm->col, val, nnz)
                       : dispatch_fill<false>(P, n_cells, smem_fill, s, sorted, Pm->row_ptr, Pm->col, val, nnz);
  if (st != WPCD_OK) return fail(st);
  count_launches(1);
  cudaEventRecord(ev1, s);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_error(e, "fill launch"));
  if ((e = cudaEventSynchronize(ev1)) != cudaSuccess) return fail(cuda_error(e, "fill pass"));
  cudaEventElapsedTime(&Pm->ms, ev0, ev1);
  cudaEventElapsedTime(&Pm->ms_phase[0], ev0, evc);
  cudaEventElapsedTime(&Pm->ms_phase[1], evc, evs);
  cudaEventElapsedTime(&Pm->ms_phase[2], evs, ev1);
  dev_free(counts);
  dev_free(sorted);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  cudaEventDestroy(evc);
  cudaEventDestroy(evs);
  grid_retain(g);  // P0 keeps its lattice alive
  *out = Pm;
  return WPCD_OK;
}

}  // namespace wpcd
