// bulk.cuh -- mbarrier and bulk asynchronous copy (the non-tensor TMA form) helpers in inline
// PTX, shared by the solve kernels (internal).
#pragma once
#include <stdint.h>

#include "lockstep.cuh"

namespace pimpc {
namespace bulk {

using ls::kWaitLimit;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Hint: bring [src, src + bytes) into L2 (16-byte aligned, a multiple of 16 bytes); no
// completion to wait for, no shared memory written.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Orders this thread's earlier generic-proxy accesses (and those it has observed) before later
// async-proxy (bulk copy) accesses, for both shared and global memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait on an mbarrier phase (every thread polls); false and an error flag on timeout.
__device__ inline bool mbar_wait(uint64_t *bar, uint32_t parity, Ctl *c) {
  long long k = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++k > kWaitLimit) {
      atomicExch(&c->err, 2);
      return false;
    }
  }
  return true;
}

}  // namespace bulk
}  // namespace pimpc
