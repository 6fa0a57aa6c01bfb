// async.cuh -- mbarrier, bulk-copy (TMA engine, 1-D) and bounded-wait helpers shared
// by the kernels that stream the resident DB through shared memory.
//
// Every barrier wait is bounded (about one second of %globaltimer): a wait that
// runs out returns false, and the caller records it in the per-device error word
// instead of spinning forever.
#pragma once
#include <cstdint>

namespace gbpir {
namespace async {

constexpr uint64_t kWaitNs = 1000000000ull;  // bound on every barrier wait
// try_wait with a suspend-time hint: a waiting thread sleeps in hardware until the
// phase completes (or the hint elapses) instead of spinning on issue slots.
constexpr uint32_t kSuspendHintNs = 100000;

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}

// Waits for the completion of phase `parity`; false once kWaitNs has passed.  A
// failed poll backs off with __nanosleep so that waiting warps leave the issue
// slots to the warps doing the work.
__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t k = 1;; ++k) {
    __nanosleep(64);
    if (mbar_try_wait(bar, parity)) return true;
    if ((k & 15) == 0 && gtimer() - t0 > kWaitNs) return false;
  }
}

// 1-D bulk copy global -> shared, completing `bytes` transaction bytes on `bar`;
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar,
                                         uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar), "l"(policy)
      : "memory");
}

// The same copy delivered to every CTA of the cluster set in ctaMask: at dst's offset
// in each one's shared memory, completing `bytes` on the barrier at bar's offset there.
__device__ __forceinline__ void bulk_g2s_multicast(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar,
                                                   uint16_t cta_mask, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4, %5;" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar), "h"(cta_mask), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

}  // namespace async
}  // namespace gbpir
