// tc_gemm.cu -- precision form of the contraction on tcgen05 (filled in below).
#include <cuda_runtime.h>

#include "../../include/wino.h"
#include "common.cuh"

namespace wino {

int layer_forward_tc(const float* x, const float* w, float* y, const LayerGeom& g,
                     const LayerMats& M, int dtype, void* ws, size_t ws_bytes, cudaStream_t st) {
  set_error("tensor-core forms not built yet");
  return WINO_EUNSUPPORTED;
}

}  // namespace wino
