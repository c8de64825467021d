// Tensor-memory-accelerator (TMA) loads and mbarrier completion for the batched 2-D kernel, as
// inline PTX (sm_90 and later; used here on sm_103a).  One thread issues a tiled 2-D copy of a box
// of a global array (described by a CUtensorMap in global memory) into shared memory; the copy
// signals its byte count on an mbarrier in shared memory, on which every thread of the CTA waits.
// Coordinates outside the tensor read as zero (the homogeneous Dirichlet values of the grid).
// No cluster multicast: every copy lands in the issuing CTA's own shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace whv {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the copy engine
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// arrive once and add `bytes` to the transaction count of the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Wait for the completion of the phase with the given parity, at most `limit` polls (each
// try_wait may suspend the thread for a short, hardware-defined time).  False if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 2-D tiled copy of the box whose first element is at (x, y) of the tensor `map` (a CUtensorMap
// in global memory, 64-byte aligned) into dst (shared memory); completes `bar`.  x times the
// element size must be a multiple of 16 bytes; out-of-range elements read as zero.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_addr(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// order this thread's generic-proxy global writes with later async-proxy (TMA) accesses
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

}  // namespace whv
