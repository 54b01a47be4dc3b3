// mbarrier-counted bulk copies (cp.async.bulk, the TMA's one-dimensional
// form) and the bounded wait every kernel of this library uses on an
// mbarrier.  Device helpers shared by the FP32 GEMM kernels (fused.cu) and
// the tensor-core contraction (tc_gemm.cu).
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace wino {

// An mbarrier expecting one arrival per phase.
__device__ __forceinline__ void mbar_init1(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar));
}
// The phase's one arrival, which also sets the bytes its copies will bring.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
// One bulk copy global -> shared (both 16-byte aligned, bytes a multiple of
// 16), completion counted on `bar` in bytes.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// Waits for phase `parity` of `bar` to complete, at most `max_polls` polls
// (each suspends the thread for a bounded time); false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  int max_polls = kWaitPolls) {
  for (int it = 0; it < max_polls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace wino
