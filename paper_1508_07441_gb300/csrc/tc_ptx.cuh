// PTX pieces shared by the tcgen05 kernels (tc_gemm.cu, oz_gemm.cu):
// shared-memory addresses, bounded mbarrier waits, tcgen05 fences, commit
// to an mbarrier and the 32-lane TMEM load.  Each translation unit gets its
// own copy (unnamed namespace).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace wpcd {
namespace {

constexpr long long TC_SPIN_LIMIT = 1LL << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
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
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit = TC_SPIN_LIMIT) {
  for (long long i = 0; i < limit; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

// The spin limit of one thread's successive waits.  The host can give the
// first wait of one role a limit of zero, so that it runs out on valid input
// and the abort path is exercised without a fault; every later wait, and
// every wait that drains copies or MMAs in flight, keeps the full limit.
struct WaitLimit {
  long long first;
  __device__ __forceinline__ explicit WaitLimit(bool expire_first) : first(expire_first ? 0 : TC_SPIN_LIMIT) {}
  __device__ __forceinline__ long long next() {
    const long long l = first;
    first = TC_SPIN_LIMIT;
    return l;
  }
};

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

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

}  // namespace
}  // namespace wpcd
