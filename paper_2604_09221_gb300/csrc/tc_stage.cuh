// tc_stage.cuh -- staging of a triangulation's tables into shared memory:
// one cp.async.bulk copy (global -> shared, no multicast) that completes on
// an mbarrier, polled with a bounded number of tries.  Used by the
// table-driven kernels (kernels.cu) and the warp-per-instance kernels
// (warp_kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"

namespace tcurve {
namespace {

constexpr long kWaitIters = 1L << 22;  // bounded spin on the table mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Stage the triangulation tables into shared memory (step (a)).  Every wait
// is bounded; on time-out the block reports kErrTimeout and returns false.
__device__ bool stage_tables(uint32_t *stab, const uint32_t *gtab, uint32_t bytes, uint64_t *bar,
                             uint32_t *err) {
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, bytes);
    bulk_g2s(stab, gtab, bytes, bar);
  }
  bool ok = false;
  for (long it = 0; it < kWaitIters && !ok; ++it) ok = mbar_try_wait(bar, 0);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
    // let a late copy land before the block's shared memory is released
    for (long it = 0; it < kWaitIters && !ok; ++it) ok = mbar_try_wait(bar, 0);
    return false;
  }
  return true;
}

}  // namespace
}  // namespace tcurve
