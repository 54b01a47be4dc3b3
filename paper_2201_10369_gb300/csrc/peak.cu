// peak.cu -- throughput probes of the SM's arithmetic pipes.
//
// The FP32 layer, the sweep and the FP64 reference are bound by plain ALU
// arithmetic, so their rooflines need the rate the pipes actually sustain on
// this part at its present clocks, not a figure derived from unit counts.
// Each probe is a grid of independent fused multiply-add chains that keeps
// every SM's pipe busy and touches no memory in its loop:
//   WINO_PIPE_FP32    fma.rn.f32      (1 FMA = 2 flops per lane)
//   WINO_PIPE_FP32X2  fma.rn.f32x2    (2 FMAs = 4 flops per lane; the packed
//                                      form the FP32 layer's contraction uses)
//   WINO_PIPE_FP64    fma.rn.f64      (1 FMA = 2 flops per lane)
// Every chain is a dependent sequence acc = acc * b + c with b, c loop
// invariant and opaque to the compiler (inline PTX), 16 chains per thread so
// the pipe's latency is covered by independent work within one warp.
#include <cuda_runtime.h>

#include "../../include/wino.h"
#include "common.cuh"

namespace wino {

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_pipe_peak(int iters, float bf, float cf,
                                                        double bd, double cd, double* sink) {
  if (KIND == WINO_PIPE_FP64) {
    double acc[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc[j] = (double)(threadIdx.x + j);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int j = 0; j < kChains; ++j)
        asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(acc[j]) : "d"(bd), "d"(cd));
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += acc[j];
    if (s == 12345.678) sink[0] = s;  // keeps the chains live; never true for these inputs
  } else if (KIND == WINO_PIPE_FP32X2) {
    unsigned long long acc[kChains], b2, c2;
    asm("mov.b64 %0, {%1, %1};" : "=l"(b2) : "f"(bf));
    asm("mov.b64 %0, {%1, %1};" : "=l"(c2) : "f"(cf));
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
      const float v = (float)(threadIdx.x + j);
      asm("mov.b64 %0, {%1, %1};" : "=l"(acc[j]) : "f"(v));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int j = 0; j < kChains; ++j)
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[j]) : "l"(b2), "l"(c2));
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
      float lo, hi;
      asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[j]));
      s += lo + hi;
    }
    if (s == 12345.678f) sink[0] = s;
  } else {
    float acc[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc[j] = (float)(threadIdx.x + j);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int j = 0; j < kChains; ++j)
        asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(acc[j]) : "f"(bf), "f"(cf));
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += acc[j];
    if (s == 12345.678f) sink[0] = s;
  }
}

}  // namespace

}  // namespace wino

using namespace wino;

extern "C" int wino_pipe_peak(int kind, int iters, int blocks_per_sm, double* tflops,
                              double* ms, void* cuda_stream) {
  if (!tflops || !ms || iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 8 ||
      (kind != WINO_PIPE_FP32 && kind != WINO_PIPE_FP32X2 && kind != WINO_PIPE_FP64)) {
    set_error("wino_pipe_peak: kind must be WINO_PIPE_FP32/FP32X2/FP64, iters >= 1, "
              "1 <= blocks_per_sm <= 8, outputs non-NULL");
    return WINO_EINVAL;
  }
  if (!wino_device_ok()) return WINO_EUNSUPPORTED;
  int dev = 0, sms = 0;
  WINO_CUDA_TRY(cudaGetDevice(&dev));
  WINO_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  void* sink = nullptr;
  int rc = scratch_get(kScratchStats, 64, &sink);
  if (rc != WINO_OK) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t a = nullptr, b = nullptr;
  WINO_CUDA_TRY(cudaEventCreate(&a));
  cudaError_t e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    (void)cudaEventDestroy(a);
    return cuda_fail(e, "cudaEventCreate");
  }
  const unsigned grid = (unsigned)(sms * blocks_per_sm);
  // b slightly below 1 and c small keep every value finite and normal
  const float bf = 0.999999f, cf = 1e-3f;
  const double bd = 0.9999999999, cd = 1e-3;
  e = cudaEventRecord(a, st);
  if (e == cudaSuccess) {
    if (kind == WINO_PIPE_FP32)
      k_pipe_peak<WINO_PIPE_FP32><<<grid, kThreads, 0, st>>>(iters, bf, cf, bd, cd, (double*)sink);
    else if (kind == WINO_PIPE_FP32X2)
      k_pipe_peak<WINO_PIPE_FP32X2><<<grid, kThreads, 0, st>>>(iters, bf, cf, bd, cd,
                                                                (double*)sink);
    else
      k_pipe_peak<WINO_PIPE_FP64><<<grid, kThreads, 0, st>>>(iters, bf, cf, bd, cd, (double*)sink);
    note_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  (void)cudaEventDestroy(a);
  (void)cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "wino_pipe_peak launch");
  const double fma_per_lane = (kind == WINO_PIPE_FP32X2) ? 2.0 : 1.0;
  const double flops = 2.0 * fma_per_lane * kChains * (double)iters * (double)grid * kThreads;
  *ms = t;
  *tflops = flops / (t * 1e-3) / 1e12;
  return WINO_OK;
}
