// bulk.cuh -- one-shot bulk copies from global into shared memory (the
// Blackwell/Hopper bulk-copy engine, completion tracked by an mbarrier), and
// bulk prefetches into L2.  Every wait is bounded.
#pragma once
#include "common.cuh"

namespace bp {

constexpr uint32_t kBulkWaitLimit = 1u << 21;  // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// An mbarrier with one expected arrival per phase (the issuing thread).
__device__ __forceinline__ void bulk_bar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// `src` to shared `dst`; the phase of `bar` completes when the bytes landed.
// The proxy fence orders this thread's earlier generic accesses to the buffer
// (made warp-wide by a __syncwarp before the call) before the async write.
__device__ __forceinline__ void bulk_load(uint32_t bar, uint32_t dst, const void *src,
                                          uint32_t bytes) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Wait for the phase of `bar` with parity `parity`; false after
// kBulkWaitLimit polls.
__device__ __forceinline__ bool bulk_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kBulkWaitLimit; i++) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, "
        "p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Pull `bytes` (a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

}  // namespace bp
