// Bounded waits on shared-memory mbarriers, used by every kernel of the
// library that waits for an asynchronous copy or for tensor-core work.
//
// A wait gives up after a time limit (%globaltimer), raises the CTA's abort
// flag and the context's device error flag (reported to the host as
// CE_ETIMEOUT), and returns false; the caller then stops issuing work and
// leaves in an orderly way.  No wait can hang the GPU, and nothing traps.
#pragma once

#include <cstdint>

namespace ce {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits until the phase with the given parity of the mbarrier at shared
// address `bar` has completed.  On expiry (or when another thread of the CTA
// has already aborted) raises *abort, sets *err = 1 and returns false.
__device__ __forceinline__ bool bounded_wait(uint32_t bar, uint32_t parity, volatile int *abort,
                                             int *err, uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (global_timer() - t0 > limit_ns) {
      *abort = 1;
      atomicExch(err, 1);
      return false;
    }
  }
  return true;
}

// Wait used only after an abort, to let a CTA's own copies and tensor-core
// work finish before its shared memory and TMEM are released (bounded too).
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity,
                                           uint64_t limit_ns = kWaitLimitNs) {
  const uint64_t t0 = global_timer();
  while (!mbar_try_wait(bar, parity))
    if (global_timer() - t0 > limit_ns) return;
}

}  // namespace ce
