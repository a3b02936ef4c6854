// Tensor-memory-accelerator (TMA) tile loads into shared memory with an mbarrier, in inline
// PTX for sm_103a.  One elected thread arms the barrier with the expected byte count and
// issues the tile copies; every thread then waits on the barrier's phase.  Waits are
// bounded: a wait that gives up returns false and the caller reports it to the host instead
// of spinning on.

#pragma once

#include <cstdint>

namespace holo {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// One arrival (the issuing thread's expect_tx) completes a phase together with the bytes.
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity; false after kMbarTries unsuccessful tries
// (each try suspends the thread for a bounded, hardware-chosen time), far longer than any
// tile copy takes.
constexpr int kMbarTries = 1 << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < kMbarTries; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 2-D tile load: box of the tensor map at element coordinates (x inner, y outer) into
// dst, completing bytes on bar.  x * element size must be a multiple of 16 bytes; rows
// outside the tensor are filled with zeros (and still counted as transferred bytes).
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// L2 prefetch (a hint: nothing is written to shared memory and nothing waits on it):
// l2_prefetch_bulk fetches the 16-byte-aligned hull of [p, p + bytes) with one bulk request;
// the hull must lie inside one allocation (every buffer here starts 256-byte aligned and
// has a size that is a multiple of 16 bytes).
__device__ __forceinline__ void l2_prefetch_bulk(const void* p, uint32_t bytes) {
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(p) & ~static_cast<uintptr_t>(15);
  const uintptr_t a1 =
      (reinterpret_cast<uintptr_t>(p) + bytes + 15) & ~static_cast<uintptr_t>(15);
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((uint32_t)(a1 - a0))
               : "memory");
}

}  // namespace holo
