// Tensor-memory-access (TMA) row gathers for the correction passes.
//
// A warp gathers the tile rows of 32 in-edges at a time with four-row
// `cp.async.bulk.tensor ... tile::gather4` copies into its own shared-memory
// slots, completed on an mbarrier (transaction-count completion).  Every wait
// is bounded by the global timer: when it runs out the kernel records a status
// word, lets the copies it already issued land, and stops.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace ppr {

// status word bits written by a kernel whose wait ran out
constexpr unsigned kTmaWaitTimeout = 1u;
constexpr unsigned long long kTmaWaitLimitNs = 500000000ull;  // 0.5 s

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait for the phase of parity `parity` to complete; false when the time
// limit runs out (the caller records the status and stops)
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
  if (mbar_try_wait(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned i = 1;; ++i) {
    if (mbar_try_wait(b, parity)) return true;
    if ((i & 63u) == 0 && global_ns() - t0 > kTmaWaitLimitNs) return false;
  }
}
// order this thread's earlier generic-proxy accesses to shared memory before
// later asynchronous-proxy writes (a slot is read, then refilled by TMA)
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// four rows y0..y3 of a 2-D tensor (box one row high, x = column start) into
// consecutive rows of dst; completes on bar with the copied bytes
__device__ __forceinline__ void tma_gather4(void* dst, const CUtensorMap* map, int x, int y0, int y1, int y2, int y3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace ppr
