// Bulk asynchronous copies global -> shared (cp.async.bulk, the TMA unit's
// untiled form) completed on a shared-memory mbarrier, with waits bounded in
// wall-clock time.
#pragma once

#include <cstdint>

namespace ibg {

// IB_ETIMEOUT of include/ib.h: recorded per instance when a wait runs out
constexpr int32_t ASYNC_TIMEOUT = 7;
// wall-clock limit of one wait (ns)
constexpr unsigned long long ASYNC_WAIT_NS = 1000000000ULL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// One thread initialises the barrier for one arrival (its own expect_tx) and
// makes the initialisation visible to the async proxy before any copy names it.
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The arrival of the issuing thread, announcing the bytes the copies will deliver.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// An arrival without copies: completes the current phase of a one-arrival
// barrier at once (a stage that receives nothing this time round).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
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

// Wait for the phase with the given parity to complete, for at most
// ASYNC_WAIT_NS.  Returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0; it < (1u << 30); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > ASYNC_WAIT_NS) return false;
  }
  return false;
}

// The wait for the copies of a CTA (by one thread, followed by a CTA barrier):
// on a timeout the instance's error word is set, and the thread waits once more
// (again bounded) so that the CTA does not retire with its copies in flight.
__device__ __forceinline__ void mbar_wait_or_flag(uint64_t* bar, uint32_t parity, int32_t* err) {
  if (mbar_wait_bounded(bar, parity)) return;
  atomicMax(err, ASYNC_TIMEOUT);
  mbar_wait_bounded(bar, parity);
}

}  // namespace ibg
