// Bulk asynchronous global -> shared copies completing on an mbarrier (sm_90 and later, inline PTX).
//
// Rules the callers keep: source and destination addresses 16-byte aligned, sizes multiples of 16
// bytes; the barrier is initialised by one thread, made visible to the async proxy, and waited on
// by every thread that reads the destination.  Waits are bounded: a wait that runs out returns
// false and the caller records the failure instead of spinning forever.
#pragma once

#include <stdint.h>

namespace hhg {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  // make the initialised barrier visible to the asynchronous (bulk copy) proxy
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// this thread's arrival, announcing `bytes` of copies that will complete on the barrier
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// bulk prefetch of a global range into L2 (no completion to wait for); address 16-byte aligned,
// size a multiple of 16
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// wait for completion of the barrier phase with the given parity; false after max_tries polls
// (each poll may suspend the thread for a hardware-defined time)
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int max_tries) {
  for (int it = 0; it < max_tries; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace hhg
