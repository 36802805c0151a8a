// pft_tma.cuh -- asynchronous bulk copies (the TMA engine's non-tensor form) between
// global and shared memory, completed on shared-memory mbarriers.
//
// A CTA stages a tile with cp.async.bulk: one elected thread arms an mbarrier with the
// number of bytes to expect and issues the copies; every thread then waits on the
// barrier's phase.  Every wait here is bounded: after kWaitNs nanoseconds of the global
// timer it records the failure in a global error word and gives up, so a lost completion
// cannot hang the GPU.
// Copies need 16-byte aligned source and destination addresses and a size that is a
// multiple of 16 bytes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pft {

constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s: far beyond any real copy

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make barrier initialisation visible to the async proxy (the bulk copies complete on it).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// One poll: true once the phase with parity `parity` has completed.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with parity `parity`.  On expiry sets *err (if given) to
// `code` and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err, int code) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_test(bar, parity)) {
    if (global_ns() - t0 > kWaitNs) {
      if (err) atomicExch(err, code);
      return false;
    }
  }
  return true;
}

// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned),
// counted against the transaction count of `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace pft
