// Tile loads by the tensor memory accelerator (TMA) into a CTA's own shared memory, completed
// on an mbarrier in the same CTA, and the host-side encoding of the tensor maps they read.
//
// A load copies one box of a tensor map (up to three dimensions here, element size 8 bytes:
// an FP32 complex value) from global memory into shared memory without the CTA's threads;
// the barrier's phase completes when all of the box's bytes have landed. Every wait is bounded
// (about a second of SM clock); a wait that runs out counts itself in a device counter that the
// host reads (tma_wait_errors) and its CTA stops without touching memory again.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace hom {

// waits that give up after this many SM cycles (about 1 s at 2 GHz)
constexpr long long kTmaWaitCycles = 1LL << 31;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// orders this thread's earlier shared-memory accesses (and barrier initialisations) before
// later accesses of the async proxy (the TMA unit) to the same memory
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// one arrival on the barrier that also announces `bytes` of asynchronous copies to come
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// box of the 3-D tensor map at element coordinates (x, y, z) into dst (128-byte aligned)
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// true once the barrier's phase of the given parity has completed; false if that takes longer
// than kTmaWaitCycles
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = smem_addr(bar);
  const long long t0 = clock64();
  while (true) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > kTmaWaitCycles) return false;
  }
}

// Host: a 3-D tiled map over 8-byte elements, dims {C, rows, batches} with row stride es and
// batch stride bs (elements), box {box_c, box_rows, 1}; out-of-range elements of a box read
// as zero. False when the layout breaks a rule of the TMA unit (base address or a stride not a
// multiple of 16 bytes, a box row not a multiple of 16 bytes, a box side above 256) or the
// driver has no encoder.
bool tma_map_3d(CUtensorMap* map, const void* base, long long C, long long rows,
                long long batches, long long es, long long bs, int box_c, int box_rows);

// device counter of TMA waits that ran out (all TMA kernels of the library); reset = zero it
unsigned tma_wait_errors(bool reset);

}  // namespace hom
