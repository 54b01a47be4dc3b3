// common.cuh -- internal declarations shared by the library's translation
// units (not part of the public ABI; see include/wino.h for that).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/wino.h"
#include "construct.cuh"

namespace wino {

// FP32 transform matrices of one point set, passed to layer kernels by
// value (they live in the kernel-parameter constant bank, so unrolled
// transforms read them as instruction operands).
constexpr int kMaxR = 7;
struct LayerMats {
  float AT[kMaxAlpha * kMaxAlpha];  // [m][alpha]
  float G[kMaxAlpha * kMaxR];       // [alpha][r]
  float BT[kMaxAlpha * kMaxAlpha];  // [alpha][alpha]
  int m, r, alpha;
};

// Layer geometry (stride 1, zero padding).  dim 1: H = Ho = th = 1.
struct LayerGeom {
  int dim, N, C, K, H, W, pad, Ho, Wo, th, tw;
  int64_t T;  // tiles = N * th * tw
  int F;      // frequencies = alpha^dim
};

// Internal return code: "no specialised kernel for this shape, use the
// general path" (never returned through the ABI).
constexpr int kFallback = 1;

// Filter transform of one (c, k) kernel g (r taps in 1D, r x r in 2D), FP32
// in the layer's fixed order: 1D v_i = sum_q G[i][q] g[q]; 2D W = G g, then
// V[i][j] = sum_q W[i][q] G[j][q]; every sum from zero with fmaf, inner
// index ascending.  sink(f, v) receives frequency f = i (1D) or i alpha + j.
template <class Sink>
__device__ __forceinline__ void filter_transform_one(const float* __restrict__ g, int dim,
                                                     const LayerMats& M, Sink sink) {
  const int A = M.alpha, r = M.r;
  const int taps = (dim == 1) ? r : r * r;
  float gl[kMaxR * kMaxR];
  for (int i = 0; i < taps; ++i) gl[i] = g[i];
  if (dim == 1) {
    for (int i = 0; i < A; ++i) {
      float acc = 0.0f;
      for (int q = 0; q < r; ++q) acc = fmaf(M.G[i * r + q], gl[q], acc);
      sink(i, acc);
    }
    return;
  }
  float Wk[kMaxAlpha * kMaxR];
  for (int i = 0; i < A; ++i)
    for (int q = 0; q < r; ++q) {
      float acc = 0.0f;
      for (int l = 0; l < r; ++l) acc = fmaf(M.G[i * r + l], gl[l * r + q], acc);
      Wk[i * r + q] = acc;
    }
  for (int i = 0; i < A; ++i)
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
      for (int q = 0; q < r; ++q) acc = fmaf(Wk[i * r + q], M.G[j * r + q], acc);
      sink(i * A + j, acc);
    }
}

// V = G g G^T of one (c, k) kernel with compile-time sizes, in the FP32
// layer's order (W = G g, l ascending; then V = W G^T, q ascending; every sum
// from zero with fmaf), so the values equal the FP32 filter transform's.
template <int MM>
__device__ __forceinline__ void filter_fixed(const float* g9, const LayerMats& M,
                                             float (&v)[(MM + 2) * (MM + 2)]) {
  constexpr int A = MM + 2, R = 3;
  float gl[R * R];
#pragma unroll
  for (int i = 0; i < R * R; ++i) gl[i] = g9[i];
  float Wk[A][R];
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int q = 0; q < R; ++q) {
      float acc = 0.0f;
#pragma unroll
      for (int l = 0; l < R; ++l) acc = fmaf(M.G[i * R + l], gl[l * R + q], acc);
      Wk[i][q] = acc;
    }
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < R; ++q) acc = fmaf(Wk[i][q], M.G[j * R + q], acc);
      v[i * A + j] = acc;
    }
}

// Per-device int in device memory, zero until a kernel's bounded wait gives
// up (the kernel then stores 1 and abandons its tile); wino_wait_error
// reads and clears it.
int wait_error_flag(int** ptr);
// Polls of one bounded mbarrier wait in the layer kernels (~1 s).
constexpr int kWaitPolls = WINO_WAIT_POLLS;
// Runs the layer kernels' bounded mbarrier wait on a barrier nothing
// arrives at, `polls` polls, on stream st; sets the flag above and stores
// the device time of the polls (synchronises st).
int wait_probe(int polls, long long* elapsed_ns, cudaStream_t st);

// Error reporting (thread-local text, see wino_last_error).
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// Counts kernel launches (reported by wino_kernel_launches).
void note_launches(int n);

// Optional event timing of one kernel launch (profile.cu): construct right
// before the launch, destroy right after it.
enum KernelId {
  kKFilter = 0, kKInput, kKGemm, kKOutput, kKFused, kKTcGemm, kKTcTransform, kKSweepEval,
  kKSweepPrep, kKDirect, kKStats, kKMlp, kKSweepOrder, kNumKernelIds
};
class ProfScope {
 public:
  ProfScope(int id, cudaStream_t st);
  ~ProfScope();

 private:
  int id_;
  cudaStream_t st_;
  void* a_;
};

// The current device's side stream of the layer paths and its two events
// (created on first use): a layer call forks work that does not depend on
// the input (the filter transforms) onto it with `fork`, recorded on the
// caller's stream, and joins it back with `join` before the contraction.
int side_stream(cudaStream_t* aux, cudaEvent_t* fork, cudaEvent_t* join);

// Scratch owned by the library (grow-only, per purpose and device).
enum ScratchSlot { kScratchLayer = 0, kScratchSweep = 1, kScratchStats = 2, kScratchTC = 3,
                   kScratchMLP = 4, kNumScratch = 5 };
int scratch_get(int slot, size_t bytes, void** ptr);

// ---- layer path (layer.cu) ----------------------------------------------
size_t layer_workspace_bytes(const LayerGeom& g, int dtype);
int layer_forward_f32(const float* x, const float* w, float* y, const LayerGeom& g,
                      const LayerMats& M, void* ws, size_t ws_bytes, cudaStream_t st);

// ---- precision form (tc_gemm.cu) ----------------------------------------
int layer_forward_tc(const float* x, const float* w, float* y, const LayerGeom& g,
                     const LayerMats& M, int dtype, void* ws, size_t ws_bytes, cudaStream_t st);

// ---- references and reductions (reference.cu) ---------------------------
int direct_conv_f64(const float* x, const float* w, double* y, int dim, int N, int C, int K,
                    int H, int W, int pad, int r, cudaStream_t st);
int error_stats(const float* yhat, const double* y, int64_t n, double* out4_host,
                cudaStream_t st);

// ---- sweep (sweep.cu) -----------------------------------------------------
struct SweepSize {
  int dim, m, r;
  double d;
};
int error_sweep(const double* c_grid, int n_c, const SweepSize* sizes, int n_sizes,
                const unsigned char* subsets, int n_subsets, int trials, unsigned long long seed,
                int order, double* err_out, cudaStream_t st);
int pointset_error(int dim, int m, int r, const double* sorted, int n_sets, int trials,
                   unsigned long long seed, int order, double* err_out, cudaStream_t st);
int pointset_error_kron(int m, int r, const double* sorted, int n_sets, int trials,
                        unsigned long long seed, int pairwise, double* err_out, cudaStream_t st);
int instance_matrices(const double* c_grid, int n_c, const SweepSize& s, unsigned mask,
                      double* AT, double* G, double* BT, unsigned char* singular,
                      cudaStream_t st);

}  // namespace wino

#define WINO_CUDA_TRY(expr)                               \
  do {                                                    \
    cudaError_t e__ = (expr);                             \
    if (e__ != cudaSuccess) return ::wino::cuda_fail(e__, #expr); \
  } while (0)
