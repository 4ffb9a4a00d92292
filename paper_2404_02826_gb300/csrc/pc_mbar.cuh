// Shared-memory barrier (mbarrier) and bulk-copy helpers, inline PTX, used by
// the partition's double-buffered tile copies (csrc/k_scatter.cu) and by the
// self-test of the bounded wait (csrc/pc_selftest.cu).  Internal.
#pragma once

#include <cstdint>

#include "pc_internal.cuh"

namespace pcx {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for the copy into one buffer; bounded: after `limit` polls the error
// bit is set and the wait is repeated once more, as long, before it returns
// (a copy in flight always completes; the second wait lets it land).  Returns
// whether the wait gave up; the caller then stops using the buffer.
__device__ __forceinline__ bool wait_buffer(unsigned long long *bar, uint32_t parity, uint32_t *err,
                                            uint32_t limit = kBarSpinLimit) {
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++spins > limit) {
      if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
      spins = 0;
      while (!mbar_try_wait(bar, parity) && ++spins < limit) {
      }
      return true;
    }
  }
  return false;
}

// Waits, bounded, for a copy whose data will not be used (a block leaving
// early lets its copies in flight land first); sets no error bit.
__device__ __forceinline__ void drain_buffer(unsigned long long *bar, uint32_t parity, uint32_t limit = kBarSpinLimit) {
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity) && ++spins < limit) {
  }
}

}  // namespace pcx
