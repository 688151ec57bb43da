// Tensor-memory-accelerator (TMA) copies and mbarrier waits for sm_100-class
// GPUs, as inline PTX: tiled bulk-tensor loads global -> shared memory whose
// completion is counted in bytes on a shared-memory mbarrier. Every mbarrier
// wait is bounded in time so that a copy that never lands ends the kernel with
// an error bit instead of a hang.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rlbm_common.h"

namespace rlbm {

constexpr unsigned long long kWaitLimitNs = kDefaultWaitNs;  // one second
// limits below this poll with the non-suspending test_wait, so that a short
// limit runs out on the first copy still in flight (failure-detection tests)
constexpr unsigned long long kPollBelowNs = 1000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make initialised barriers visible to the async proxy (the TMA unit).
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrive once and announce `bytes` of incoming transactions.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// 4D tiled copy of one box at element coordinates (c0, c1, c2, c3) of the
// tensor map into shared memory.
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-suspending test of the phase of parity `parity`.
__device__ __forceinline__ bool mbar_poll(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait until the phase of parity `parity` has completed; false once limit_ns
// have passed (a limit under kPollBelowNs polls without suspending).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned long long limit_ns = kWaitLimitNs) {
  const unsigned long long t0 = global_ns();
  if (limit_ns < kPollBelowNs) {
    for (;;) {
      if (mbar_poll(bar, parity)) return true;
      if (global_ns() - t0 > limit_ns) return false;
    }
  }
  if (mbar_test(bar, parity)) return true;
  for (unsigned it = 1;; ++it) {
    if (mbar_test(bar, parity)) return true;
    if ((it & 63u) == 0u && global_ns() - t0 > limit_ns) return false;
  }
}

}  // namespace rlbm
