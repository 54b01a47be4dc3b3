// noalloc.cu -- the FP32 Winograd layer for callers that cannot allocate
// device memory.
//
// Who needs it: code that runs while a stream is being captured into a CUDA
// graph in global capture mode (cudaMalloc is not permitted then), plug-ins
// running inside a framework whose caching allocator has already reserved
// the device memory they would ask for, and latency-critical loops whose
// rules forbid allocation after start-up.  wino_conv2d takes its scratch
// from cudaMalloc on first use (or from wino_set_workspace); this entry point
// instead uses one fixed array of device memory that is part of the library
// image, so no call allocates.
//
// The scratch holds the transformed filters V[alpha^2][C][K] of the fused
// FP32 kernel (fused.cu).  Every call overwrites the part it uses before
// reading it, so nothing has to start at zero.  All calls share the one
// array: calls whose GPU work overlaps (different streams, or different
// host threads, without ordering between them) race on it.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <string>

#include "../../include/wino.h"
#include "common.cuh"

namespace wino {

int layer_forward_fused(const float* x, const float* w, float* y, const LayerGeom& g,
                        const LayerMats& M, void* ws, size_t ws_bytes, cudaStream_t st);
size_t fused_workspace_bytes(const LayerGeom& g);

// The scratch array: WINO_NOALLOC_SCRATCH_FLOATS floats, 256-byte aligned,
// present on every device that loads the library until the process exits.
static __device__ __align__(256) float g_noalloc_scratch[WINO_NOALLOC_SCRATCH_FLOATS];

namespace {
constexpr int kMaxDevices = 16;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {nullptr};  // device address, per device
}  // namespace

// Device address of the scratch array on the current device.  In host code
// the symbol names a host-side stand-in, never the device memory, so the
// address is looked up once per device (with that device current).
static int noalloc_scratch(void** out) {
  int dev = 0;
  WINO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device index out of range");
    return WINO_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return WINO_OK;
}

}  // namespace wino

using namespace wino;

extern "C" int wino_conv2d_f32_noalloc(const void* x, const void* w, void* y, int N, int C,
                                       int K, int H, int W, int pad, const double* points,
                                       int m, int r, void* cuda_stream) {
  if (r != 3 || (m != 2 && m != 4 && m != 6) || N < 0 || C < 1 || K < 1 || H < 1 || W < 1 ||
      pad < 0 || K % 64 != 0) {
    set_error("wino_conv2d_f32_noalloc supports r = 3, m in {2, 4, 6}, K a multiple of 64");
    return WINO_EINVAL;
  }
  if (!points) {
    set_error("points is NULL");
    return WINO_EINVAL;
  }
  const int alpha = m + r - 1;
  const double need = (double)alpha * alpha * C * K;
  if (need > (double)WINO_NOALLOC_SCRATCH_FLOATS) {
    set_error("layer needs " + std::to_string((long long)need) +
              " floats of scratch; the fixed array holds " +
              std::to_string(WINO_NOALLOC_SCRATCH_FLOATS) + " (alpha^2 * C * K must not exceed it)");
    return WINO_EINVAL;
  }
  // point set: exactly one +inf, the rest finite; sorted ascending
  double fin[kMaxAlpha];
  int n_inf = 0, nf = 0;
  for (int i = 0; i < alpha; ++i) {
    const double p = points[i];
    if (isnan(p) || (isinf(p) && p < 0)) {
      set_error("points must be finite or +INFINITY");
      return WINO_EINVAL;
    }
    if (isinf(p))
      ++n_inf;
    else
      fin[nf++] = p;
  }
  if (n_inf != 1) {
    set_error("exactly one point must be +INFINITY");
    return WINO_EINVAL;
  }
  sort_points(fin, nf);
  double ATd[kMaxAlpha * kMaxAlpha], Gd[kMaxAlpha * kMaxR], BTd[kMaxAlpha * kMaxAlpha];
  if (!build_matrices<double>(fin, m, r, ATd, Gd, BTd)) {
    set_error("two finite points coincide (singular Vandermonde system)");
    return WINO_ESINGULAR;
  }
  LayerMats M;
  memset(&M, 0, sizeof(M));
  for (int i = 0; i < m * alpha; ++i) M.AT[i] = (float)ATd[i];
  for (int i = 0; i < alpha * r; ++i) M.G[i] = (float)Gd[i];
  for (int i = 0; i < alpha * alpha; ++i) M.BT[i] = (float)BTd[i];
  M.m = m;
  M.r = r;
  M.alpha = alpha;
  LayerGeom g;
  g.dim = 2;
  g.N = N;
  g.C = C;
  g.K = K;
  g.H = H;
  g.W = W;
  g.pad = pad;
  g.Ho = H + 2 * pad - r + 1;
  g.Wo = W + 2 * pad - r + 1;
  if (g.Ho < 1 || g.Wo < 1) {
    set_error("kernel larger than the padded input");
    return WINO_EINVAL;
  }
  g.th = (g.Ho + m - 1) / m;
  g.tw = (g.Wo + m - 1) / m;
  g.T = (int64_t)N * g.th * g.tw;
  g.F = alpha * alpha;
  if (N == 0) return WINO_OK;
  if (!x || !w || !y) {
    set_error("x, w and y must be device pointers");
    return WINO_EINVAL;
  }
  // the device check is cached per device (no property query per call)
  if (!wino_device_ok()) return WINO_EUNSUPPORTED;
  void* scratch = nullptr;
  int st = noalloc_scratch(&scratch);
  if (st != WINO_OK) return st;
  const size_t bytes = (size_t)WINO_NOALLOC_SCRATCH_FLOATS * sizeof(float);
  st = layer_forward_fused((const float*)x, (const float*)w, (float*)y, g, M, scratch, bytes,
                           (cudaStream_t)cuda_stream);
  if (st == kFallback) {
    set_error("shape not supported by the fused kernel");
    return WINO_EINVAL;
  }
  return st;
}
