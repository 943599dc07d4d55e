// Asynchronous-copy helpers shared by the kernels that stage data with the
// bulk-copy engine: mbarrier set-up, transaction counts, 1-D bulk copies
// global -> shared, and a bounded wait (a wait that gives up returns false so
// the kernel can raise its error flag instead of spinning forever).
#pragma once
#include <stdint.h>

#include "debug.cuh"

namespace sapmg {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Completes `bytes` of the barrier's expected transactions without a copy.
__device__ __forceinline__ void mbar_complete_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
#ifdef MG_DEBUG
  // both addresses and the size must be multiples of 16 bytes; a copy that is
  // not is skipped and its bytes completed by hand, so the wait still ends
  const uint32_t bad = (smem_u32(dst) | (uint32_t)reinterpret_cast<uintptr_t>(src) | bytes) & 15u;
  if (!MG_CHECK(kBulkCopy, bad, 1)) {
    mbar_complete_tx(bar, bytes);
    return;
  }
#endif
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase completed, false after `spins` tries
// (kMaxSpins by default).
constexpr int kMaxSpins = 1 << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int spins = kMaxSpins) {
  for (int i = 0; i < spins; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// The device error word of a context: err[0] is the flag a wait that gave up
// raises, err[1] the bound on the main-loop waits of the bulk-copy kernels
// (kMaxSpins unless a test lowers it to drive the timeout path; the drain
// waits after a failure always use kMaxSpins).
__device__ __forceinline__ int wait_spins(const int* err) { return err[1]; }


}  // namespace sapmg
