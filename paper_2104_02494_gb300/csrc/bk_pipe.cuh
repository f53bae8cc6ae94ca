// Asynchronous bulk-copy pipeline primitives (sm_90 and later, used on sm_103a):
// shared-memory mbarriers, 1D bulk copies (cp.async.bulk) and tiled tensor
// copies (cp.async.bulk.tensor) from global to shared memory, whose completion
// is counted in bytes on an mbarrier ("complete_tx").
//
// A ring of NS shared-memory stages is filled by one producer thread and read by
// the consumer warps.  Stage k has two barriers: full[k] (one producer arrival
// plus the copied bytes) and empty[k] (one arrival per consumer warp).  Use u
// of a stage completes phase u of its barriers, so a waiter of use u waits for
// parity u & 1.
//
// Every wait is bounded: after kWaitCycles SM clock cycles (about 1 s at
// 2 GHz) it gives up, and the caller records BK_TIMEOUT, stops its work and
// lets the kernel end normally.  A wait also gives up early once another
// thread of the CTA has raised the CTA's abort flag.
#pragma once

#include <cstdint>
#include <cuda.h>

#include "bk_common.cuh"

namespace bk {

constexpr long long kWaitCycles = 1ll << 31;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make the initialised barriers visible to the async (copy) proxy; call once by
// the initialising thread, followed by a CTA barrier.
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Producer: arrive on `bar` and announce `bytes` of copies that will complete on it.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// Bounded wait for phase `parity` of `bar`.  Returns false when it gave up
// (time limit, or *abort set by another thread of the CTA).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

// 1D bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Tiled 4D tensor copy of the tensor map's box at coordinates (c0, c1, c2, c3)
// (c0 innermost) into shared memory, completing on `bar`.  Out-of-range
// elements of the box are filled with zeros; the barrier counts the whole box.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// Tiled 2D tensor copy of the box at (c0, c1) (c0 innermost), as tma_load_4d.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Record a timed-out wait: the status word (if any) gets BK_TIMEOUT and the stop
// word (if any) a non-zero value, so that the kernels after this one return.
__device__ __forceinline__ void report_timeout(int* status, int* stop) {
  if (status) atomicExch(status, (int)BK_TIMEOUT);
  if (stop) atomicExch(stop, (int)kDoneStopped);
}

}  // namespace bk
