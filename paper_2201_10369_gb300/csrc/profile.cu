// profile.cu -- optional CUDA-event timing of the library's own kernels.
// When enabled (wino_profile_enable), each launch site records a start and a
// stop event on the stream the kernel is launched on; wino_profile_read sums
// the elapsed times per kernel name.  Off by default; recording is skipped
// while the stream is being captured into a graph.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "../../include/wino.h"
#include "common.cuh"

namespace wino {

static const char* kKernelNames[kNumKernelIds] = {
    "filter_transform", "input_transform", "wino_gemm",  "output_transform", "fused_layer",
    "tc_gemm",          "tc_transform",    "sweep_eval", "sweep_prepare",    "direct_f64",
    "error_stats",      "mlp",             "sweep_order"};

namespace {
struct Rec {
  int id;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return e;
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    (void)cudaGetLastError();
    return true;
  }
  return cs != cudaStreamCaptureStatusNone;
}
}  // namespace

ProfScope::ProfScope(int id, cudaStream_t st) : id_(id), st_(st), a_(nullptr) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (capturing(st)) return;
  a_ = get_event();
  if (a_) (void)cudaEventRecord((cudaEvent_t)a_, st);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = get_event();
  if (!b) return;
  (void)cudaEventRecord(b, st_);
  g_recs.push_back(Rec{id_, (cudaEvent_t)a_, b});
}

}  // namespace wino

using namespace wino;

extern "C" {

int wino_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  return WINO_OK;
}

int wino_profile_read(const char* kernel, double* total_ms, int* launches) {
  if (!kernel || !total_ms || !launches) {
    set_error("invalid arguments to wino_profile_read");
    return WINO_EINVAL;
  }
  int id = -1;
  for (int i = 0; i < kNumKernelIds; ++i)
    if (strcmp(kernel, kKernelNames[i]) == 0) id = i;
  if (id < 0) {
    set_error("unknown kernel name");
    return WINO_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  double ms = 0.0;
  int n = 0;
  std::vector<Rec> keep;
  for (const Rec& r : g_recs) {
    if (r.id != id) {
      keep.push_back(r);
      continue;
    }
    cudaError_t e = cudaEventSynchronize(r.b);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    ms += t;
    ++n;
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.swap(keep);
  *total_ms = ms;
  *launches = n;
  return WINO_OK;
}

}  // extern "C"
