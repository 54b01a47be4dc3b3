// mlp.cu -- the learned surrogate of the point sweep: a 16-64-1 perceptron
// (GELU, erf form) predicting log10 of the sweep error of an instance from
// (m, r, subset mask, log c, dim), trained on the device by hand-written
// forward / backward / Adam kernels on labels the sweep itself produces.
// The paper's observation that the error curve over c is roughly smooth
// (Sec. 6.1) is what makes a surrogate useful: it ranks a dense c grid, and
// only the top candidates are evaluated by the exact sweep.
//
// Parameters: FP32 master copy p[1153] = [W1 64x16 | b1 64 | w2 64 | b2],
// BF16-rounded working copy pw (stored as floats) used by the forward and
// backward passes; Adam updates the masters and re-rounds pw.
// One training step = gradient kernel (blocks of 64 samples, per-block
// reduction in shared memory into that block's row of partial gradients;
// block 0 also advances the step counter, which lives on the device so an
// epoch can be captured once in a CUDA graph and replayed) + Adam kernel
// (one thread per parameter, which first adds the blocks' partials in block
// order).  No atomics: a training run is deterministic, the same weights
// from the same data, seed and schedule on every run.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "../../include/wino.h"
#include "common.cuh"

namespace wino {

constexpr int kIn = 16, kHid = 64;
constexpr int kNParam = kHid * kIn + kHid + kHid + 1;  // 1153
constexpr int kOffB1 = kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid;
constexpr int kGradBlock = 64;

__device__ __forceinline__ float gelu_f(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__global__ void k_mlp_round(const float* __restrict__ p, float* __restrict__ pw) {
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < kNParam; i += blockDim.x * gridDim.x)
    pw[i] = __bfloat162float(__float2bfloat16_rn(p[i]));
}

// MSE gradient of a batch at the working weights, per block: row b of
// part (kPartStride floats) receives the sum over block b's samples of
// d/dp (out - y)^2 / B and, in its last word, their squared residuals.
// With t non-null, block 0 advances the step counter.
constexpr int kPartStride = kNParam + 1;
__global__ void __launch_bounds__(kGradBlock) k_mlp_grad(const float* __restrict__ pw,
                                                         const float* __restrict__ X,
                                                         const float* __restrict__ y, int B,
                                                         float* __restrict__ part,
                                                         int* __restrict__ t) {
  __shared__ float sp[kNParam];
  __shared__ float sdz[kGradBlock][kHid + 1];
  __shared__ float sh[kGradBlock][kHid + 1];
  __shared__ float sx[kGradBlock][kIn + 1];
  __shared__ float sdo[kGradBlock];
  __shared__ float sr2[kGradBlock / 32];
  const int tid = threadIdx.x;
  if (t && blockIdx.x == 0 && tid == 0) *t += 1;
  for (int i = tid; i < kNParam; i += kGradBlock) sp[i] = pw[i];
  __syncthreads();
  const int s = blockIdx.x * kGradBlock + tid;
  float r2 = 0.0f;
  if (s < B) {
    float x[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) x[i] = X[(int64_t)s * kIn + i];
    float out = sp[kOffB2];
    float z[kHid];
#pragma unroll 4
    for (int j = 0; j < kHid; ++j) {
      float a = sp[kOffB1 + j];
#pragma unroll
      for (int i = 0; i < kIn; ++i) a = fmaf(sp[j * kIn + i], x[i], a);
      z[j] = a;
      const float h = gelu_f(a);
      sh[tid][j] = h;
      out = fmaf(sp[kOffW2 + j], h, out);
    }
    const float r = out - y[s];
    r2 = r * r;
    const float dout = 2.0f * r / (float)B;
    sdo[tid] = dout;
#pragma unroll 4
    for (int j = 0; j < kHid; ++j) sdz[tid][j] = dout * sp[kOffW2 + j] * gelu_grad_f(z[j]);
#pragma unroll
    for (int i = 0; i < kIn; ++i) sx[tid][i] = x[i];
  } else {
    sdo[tid] = 0.0f;
    for (int j = 0; j < kHid; ++j) {
      sdz[tid][j] = 0.0f;
      sh[tid][j] = 0.0f;
    }
    for (int i = 0; i < kIn; ++i) sx[tid][i] = 0.0f;
  }
  // squared residuals: warp shuffle, then the warps in order
  for (int o = 16; o > 0; o >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, o);
  if ((tid & 31) == 0) sr2[tid >> 5] = r2;
  __syncthreads();
  float* row = part + (int64_t)blockIdx.x * kPartStride;
  if (tid == 0) {
    float l = 0.0f;
    for (int w = 0; w < kGradBlock / 32; ++w) l += sr2[w];
    row[kNParam] = l;
  }
  // per-parameter sums over the block's samples
  for (int q = tid; q < kNParam; q += kGradBlock) {
    float acc = 0.0f;
    if (q < kOffB1) {
      const int j = q / kIn, i = q % kIn;
      for (int t = 0; t < kGradBlock; ++t) acc = fmaf(sdz[t][j], sx[t][i], acc);
    } else if (q < kOffW2) {
      const int j = q - kOffB1;
      for (int t = 0; t < kGradBlock; ++t) acc += sdz[t][j];
    } else if (q < kOffB2) {
      const int j = q - kOffW2;
      for (int t = 0; t < kGradBlock; ++t) acc = fmaf(sdo[t], sh[t][j], acc);
    } else {
      for (int t = 0; t < kGradBlock; ++t) acc += sdo[t];
    }
    row[q] = acc;
  }
}

// Sum of the blocks' partial gradients (and squared residuals) in block
// order: grad[i] = sum_b part[b][i], i < kNParam + 1.
__device__ __forceinline__ float sum_parts(const float* __restrict__ part, int nblocks, int i) {
  float g = 0.0f;
  for (int b = 0; b < nblocks; ++b) g += part[(int64_t)b * kPartStride + i];
  return g;
}
__global__ void k_mlp_reduce(const float* __restrict__ part, int nblocks,
                             float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kPartStride) grad[i] = sum_parts(part, nblocks, i);
}

// Adam, one thread per parameter: g = the blocks' partials added in block
// order; p <- p - lr mhat / (sqrt(vhat) + eps) at the step the gradient
// kernel counted; pw <- bf16(p).
__global__ void k_mlp_adam(float* __restrict__ p, float* __restrict__ pw,
                           const float* __restrict__ part, int nblocks, float* __restrict__ m,
                           float* __restrict__ v, const int* __restrict__ t, float lr) {
  const int step = *t;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kNParam) {
    const float g = sum_parts(part, nblocks, i);
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pw[i] = __bfloat162float(__float2bfloat16_rn(pi));
  }
}

__global__ void k_mlp_predict(const float* __restrict__ pw, const float* __restrict__ X,
                              int64_t n, float* __restrict__ out) {
  __shared__ float sp[kNParam];
  for (int i = threadIdx.x; i < kNParam; i += blockDim.x) sp[i] = pw[i];
  __syncthreads();
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[kIn];
#pragma unroll
  for (int i = 0; i < kIn; ++i) x[i] = X[s * kIn + i];
  float o = sp[kOffB2];
  for (int j = 0; j < kHid; ++j) {
    float a = sp[kOffB1 + j];
#pragma unroll
    for (int i = 0; i < kIn; ++i) a = fmaf(sp[j * kIn + i], x[i], a);
    o = fmaf(sp[kOffW2 + j], gelu_f(a), o);
  }
  out[s] = o;
}

// Features of an instance: [m/8, (r-3)/2, mask bits b0..b7, u, dim - 1, u^2,
// |u|, u^3, 0] with u = ln c / ln 20 (the spare inputs carry powers of the one
// continuous input).
struct MlpSizeInfo {
  int dim, m, r, pad;
};
__global__ void k_mlp_features(const MlpSizeInfo* __restrict__ sizes,
                               const wino_instance* __restrict__ inst, int64_t n,
                               float* __restrict__ X) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const wino_instance q = inst[s];
  const MlpSizeInfo z = sizes[q.size];
  float* x = X + s * kIn;
  x[0] = z.m * 0.125f;
  x[1] = (z.r - 3) * 0.5f;
#pragma unroll
  for (int b = 0; b < 8; ++b) x[2 + b] = (float)((q.mask >> b) & 1u);
  const float u = (float)(log(q.c) / log(20.0));
  x[10] = u;
  x[11] = (float)(z.dim - 1);
  x[12] = u * u;
  x[13] = fabsf(u);
  x[14] = u * u * u;
  x[15] = 0.0f;
}

// Features of a grid: row q = (size, mask) x every c of c_grid, row-major.
__global__ void k_mlp_grid_features(const MlpSizeInfo* __restrict__ sizes,
                                    const int* __restrict__ row_size,
                                    const unsigned char* __restrict__ row_mask, int n_rows,
                                    const double* __restrict__ cg, int n_c,
                                    float* __restrict__ X) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= (int64_t)n_rows * n_c) return;
  const int q = (int)(s / n_c), k = (int)(s % n_c);
  const MlpSizeInfo z = sizes[row_size[q]];
  const unsigned mk = row_mask[q];
  float* x = X + s * kIn;
  x[0] = z.m * 0.125f;
  x[1] = (z.r - 3) * 0.5f;
#pragma unroll
  for (int b = 0; b < 8; ++b) x[2 + b] = (float)((mk >> b) & 1u);
  const float u = (float)(log(cg[k]) / log(20.0));
  x[10] = u;
  x[11] = (float)(z.dim - 1);
  x[12] = u * u;
  x[13] = fabsf(u);
  x[14] = u * u * u;
  x[15] = 0.0f;
}

// The k smallest values of each row (ties by index), ascending: one block per
// row, bitonic sort of (value, index) pairs in shared memory.
__global__ void k_topk_rows(const float* __restrict__ vals, int cols, int k,
                            int* __restrict__ idx_out) {
  extern __shared__ unsigned char tk[];
  const int row = blockIdx.x;
  int P = 1;
  while (P < cols) P <<= 1;
  float* sv = reinterpret_cast<float*>(tk);
  int* si = reinterpret_cast<int*>(sv + P);
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const float v = (i < cols) ? vals[(int64_t)row * cols + i] : INFINITY;
    sv[i] = (v == v) ? v : INFINITY;  // NaN sorts last
    si[i] = i;
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const float a = sv[i], b = sv[j];
          const int ia = si[i], ib = si[j];
          const bool a_after_b = (a > b) || (a == b && ia > ib);
          if (a_after_b == up) {
            sv[i] = b;
            sv[j] = a;
            si[i] = ib;
            si[j] = ia;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < k; i += blockDim.x) idx_out[(int64_t)row * k + i] = si[i];
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
struct Mlp {
  float *p = nullptr, *pw = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
  int* t = nullptr;
  void* buf = nullptr;
  float* part = nullptr;  // per-block partial gradients (grown as needed)
  int part_blocks = 0;
};

// The handle's partial-gradient rows for `nblocks` gradient blocks.
static int mlp_part(Mlp* M, int nblocks, float** part) {
  if (nblocks > M->part_blocks) {
    if (M->part) {
      WINO_CUDA_TRY(cudaDeviceSynchronize());
      WINO_CUDA_TRY(cudaFree(M->part));
      M->part = nullptr;
      M->part_blocks = 0;
    }
    if (cudaMalloc(&M->part, (size_t)nblocks * kPartStride * sizeof(float)) != cudaSuccess) {
      (void)cudaGetLastError();
      M->part = nullptr;
      set_error("could not allocate the surrogate's gradient partials");
      return WINO_ENOMEM;
    }
    M->part_blocks = nblocks;
  }
  *part = M->part;
  return WINO_OK;
}

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace wino

using namespace wino;

extern "C" {

int wino_mlp_create(unsigned long long seed, void** out) {
  if (!out) {
    set_error("out is NULL");
    return WINO_EINVAL;
  }
  Mlp* M = new Mlp();
  const size_t n = kNParam;
  const size_t bytes = (5 * n + 64) * sizeof(float) + 64;
  if (cudaMalloc(&M->buf, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    delete M;
    set_error("could not allocate the surrogate's parameters");
    return WINO_ENOMEM;
  }
  float* b = (float*)M->buf;
  M->p = b;
  M->pw = b + n;
  M->m = b + 2 * n;
  M->v = b + 3 * n;
  M->grad = b + 4 * n;
  M->loss = b + 5 * n;
  M->t = (int*)(b + 5 * n + 16);
  // uniform(-a, a) initial weights, a = sqrt(6 / fan_in), biases 0
  std::vector<float> h(n, 0.0f);
  for (size_t i = 0; i < n; ++i) {
    const double u = (double)(mix64(seed + 0x9E3779B97F4A7C15ull * (i + 1)) >> 11) * 0x1p-53;
    if (i < (size_t)kOffB1)
      h[i] = (float)((2.0 * u - 1.0) * sqrt(6.0 / kIn));
    else if (i >= (size_t)kOffW2 && i < (size_t)kOffB2)
      h[i] = (float)((2.0 * u - 1.0) * sqrt(6.0 / kHid));
  }
  int rc = wino_mlp_set_params(M, h.data());
  if (rc != WINO_OK) {
    cudaFree(M->buf);
    delete M;
    return rc;
  }
  *out = M;
  return WINO_OK;
}

int wino_mlp_set_params(void* mlp, const float* params) {
  Mlp* M = (Mlp*)mlp;
  if (!M || !params) {
    set_error("invalid arguments to wino_mlp_set_params");
    return WINO_EINVAL;
  }
  WINO_CUDA_TRY(cudaMemcpy(M->p, params, kNParam * sizeof(float), cudaMemcpyHostToDevice));
  WINO_CUDA_TRY(cudaMemset(M->m, 0, 3 * kNParam * sizeof(float)));  // m, v, grad
  WINO_CUDA_TRY(cudaMemset(M->loss, 0, 64 * sizeof(float)));          // loss, t
  k_mlp_round<<<5, 256>>>(M->p, M->pw);
  note_launches(1);
  WINO_CUDA_TRY(cudaGetLastError());
  WINO_CUDA_TRY(cudaDeviceSynchronize());
  return WINO_OK;
}

int wino_mlp_get_params(void* mlp, float* params, int working) {
  Mlp* M = (Mlp*)mlp;
  if (!M || !params) {
    set_error("invalid arguments to wino_mlp_get_params");
    return WINO_EINVAL;
  }
  WINO_CUDA_TRY(cudaDeviceSynchronize());
  WINO_CUDA_TRY(cudaMemcpy(params, working ? M->pw : M->p, kNParam * sizeof(float),
                           cudaMemcpyDeviceToHost));
  return WINO_OK;
}

int wino_mlp_loss_grad(void* mlp, const float* X, const float* y, int B, float* grad_out,
                       double* loss_out, void* cuda_stream) {
  Mlp* M = (Mlp*)mlp;
  if (!M || !X || !y || B < 1 || !grad_out || !loss_out) {
    set_error("invalid arguments to wino_mlp_loss_grad");
    return WINO_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nb = (B + kGradBlock - 1) / kGradBlock;
  float* part = nullptr;
  int rc = mlp_part(M, nb, &part);
  if (rc != WINO_OK) return rc;
  {
    ProfScope ps(kKMlp, st);
    k_mlp_grad<<<nb, kGradBlock, 0, st>>>(M->pw, X, y, B, part, nullptr);
    k_mlp_reduce<<<(kPartStride + 255) / 256, 256, 0, st>>>(part, nb, M->grad);
    note_launches(2);
  }
  WINO_CUDA_TRY(cudaGetLastError());
  float ls = 0.0f;
  WINO_CUDA_TRY(cudaMemcpyAsync(grad_out, M->grad, kNParam * sizeof(float),
                                cudaMemcpyDeviceToHost, st));
  WINO_CUDA_TRY(cudaMemcpyAsync(&ls, M->grad + kNParam, sizeof(float), cudaMemcpyDeviceToHost,
                                st));
  WINO_CUDA_TRY(cudaStreamSynchronize(st));
  *loss_out = (double)ls / B;
  return WINO_OK;
}

int wino_mlp_train(void* mlp, const float* X, const float* y, int64_t n, int batch, int epochs,
                   float lr, void* cuda_stream) {
  Mlp* M = (Mlp*)mlp;
  if (!M || !X || !y || n < 1 || batch < 1 || epochs < 0 || !(lr > 0.0f)) {
    set_error("invalid arguments to wino_mlp_train");
    return WINO_EINVAL;
  }
  const int64_t steps = n / batch;  // whole batches only
  if (steps < 1) {
    set_error("fewer samples than one batch");
    return WINO_EINVAL;
  }
  const int nb = (batch + kGradBlock - 1) / kGradBlock;
  float* part = nullptr;
  {
    int rc = mlp_part(M, nb, &part);
    if (rc != WINO_OK) return rc;
  }
  cudaStream_t st = nullptr;
  WINO_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t ev = nullptr;
  WINO_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  // order after the caller's stream
  WINO_CUDA_TRY(cudaEventRecord(ev, (cudaStream_t)cuda_stream));
  WINO_CUDA_TRY(cudaStreamWaitEvent(st, ev, 0));
  // one epoch = `steps` (gradient, Adam) pairs, captured once, replayed
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  WINO_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  for (int64_t s = 0; s < steps; ++s) {
    k_mlp_grad<<<nb, kGradBlock, 0, st>>>(M->pw, X + s * batch * kIn, y + s * batch, batch,
                                          part, M->t);
    k_mlp_adam<<<(kNParam + 255) / 256, 256, 0, st>>>(M->p, M->pw, part, nb, M->m, M->v, M->t,
                                                      lr);
  }
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  {
    ProfScope ps(kKMlp, st);
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
      e = cudaGraphLaunch(exec, st);
      note_launches((int)(2 * steps));
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)cuda_stream, ev, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaEventDestroy(ev);
  cudaStreamDestroy(st);
  if (e != cudaSuccess) return cuda_fail(e, "wino_mlp_train");
  return WINO_OK;
}

int wino_mlp_predict(void* mlp, const float* X, int64_t n, float* out, void* cuda_stream) {
  Mlp* M = (Mlp*)mlp;
  if (!M || !X || !out || n < 0) {
    set_error("invalid arguments to wino_mlp_predict");
    return WINO_EINVAL;
  }
  if (n == 0) return WINO_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  ProfScope ps(kKMlp, st);
  k_mlp_predict<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M->pw, X, n, out);
  note_launches(1);
  WINO_CUDA_TRY(cudaGetLastError());
  return WINO_OK;
}

int wino_mlp_features(const wino_size* sizes, int n_sizes, const wino_instance* inst, int64_t n,
                      float* X, void* cuda_stream) {
  if (!sizes || n_sizes < 1 || n_sizes > 64 || !inst || n < 0 || !X) {
    set_error("invalid arguments to wino_mlp_features");
    return WINO_EINVAL;
  }
  if (n == 0) return WINO_OK;
  for (int64_t i = 0; i < n; ++i)
    if (inst[i].size < 0 || inst[i].size >= n_sizes || !(inst[i].c > 0.0)) {
      set_error("instance with a bad size index or c <= 0");
      return WINO_EINVAL;
    }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t bytes = 64 * sizeof(MlpSizeInfo) + (size_t)n * sizeof(wino_instance);
  void* base = nullptr;
  int rc = scratch_get(kScratchMLP, bytes, &base);
  if (rc != WINO_OK) return rc;
  MlpSizeInfo hs[64];
  for (int s = 0; s < n_sizes; ++s) hs[s] = MlpSizeInfo{sizes[s].dim, sizes[s].m, sizes[s].r, 0};
  MlpSizeInfo* ds = (MlpSizeInfo*)base;
  wino_instance* di = (wino_instance*)((char*)base + 64 * sizeof(MlpSizeInfo));
  WINO_CUDA_TRY(cudaMemcpyAsync(ds, hs, n_sizes * sizeof(MlpSizeInfo), cudaMemcpyHostToDevice, st));
  WINO_CUDA_TRY(
      cudaMemcpyAsync(di, inst, (size_t)n * sizeof(wino_instance), cudaMemcpyHostToDevice, st));
  k_mlp_features<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ds, di, n, X);
  note_launches(1);
  WINO_CUDA_TRY(cudaGetLastError());
  WINO_CUDA_TRY(cudaStreamSynchronize(st));  // the host instance array may be reused
  return WINO_OK;
}

int wino_mlp_grid_features(const wino_size* sizes, int n_sizes, const int* row_size,
                           const unsigned char* row_mask, int n_rows, const double* c_grid,
                           int n_c, float* X, void* cuda_stream) {
  if (!sizes || n_sizes < 1 || n_sizes > 64 || !row_size || !row_mask || n_rows < 0 ||
      !c_grid || n_c < 1 || !X) {
    set_error("invalid arguments to wino_mlp_grid_features");
    return WINO_EINVAL;
  }
  if (n_rows == 0) return WINO_OK;
  for (int q = 0; q < n_rows; ++q)
    if (row_size[q] < 0 || row_size[q] >= n_sizes) {
      set_error("row with a bad size index");
      return WINO_EINVAL;
    }
  for (int k = 0; k < n_c; ++k)
    if (!(c_grid[k] > 0.0)) {
      set_error("c values must be > 0");
      return WINO_EINVAL;
    }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t o_rows = 64 * sizeof(MlpSizeInfo);
  const size_t o_mask = o_rows + (size_t)n_rows * sizeof(int);
  const size_t o_c = (o_mask + n_rows + 15) & ~(size_t)15;
  const size_t bytes = o_c + (size_t)n_c * sizeof(double);
  void* base = nullptr;
  int rc = scratch_get(kScratchMLP, bytes, &base);
  if (rc != WINO_OK) return rc;
  MlpSizeInfo hs[64];
  for (int s = 0; s < n_sizes; ++s) hs[s] = MlpSizeInfo{sizes[s].dim, sizes[s].m, sizes[s].r, 0};
  char* b = (char*)base;
  WINO_CUDA_TRY(cudaMemcpyAsync(b, hs, n_sizes * sizeof(MlpSizeInfo), cudaMemcpyHostToDevice, st));
  WINO_CUDA_TRY(cudaMemcpyAsync(b + o_rows, row_size, n_rows * sizeof(int), cudaMemcpyHostToDevice, st));
  WINO_CUDA_TRY(cudaMemcpyAsync(b + o_mask, row_mask, n_rows, cudaMemcpyHostToDevice, st));
  WINO_CUDA_TRY(cudaMemcpyAsync(b + o_c, c_grid, n_c * sizeof(double), cudaMemcpyHostToDevice, st));
  const int64_t n = (int64_t)n_rows * n_c;
  k_mlp_grid_features<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      (const MlpSizeInfo*)b, (const int*)(b + o_rows), (const unsigned char*)(b + o_mask), n_rows,
      (const double*)(b + o_c), n_c, X);
  note_launches(1);
  WINO_CUDA_TRY(cudaGetLastError());
  WINO_CUDA_TRY(cudaStreamSynchronize(st));
  return WINO_OK;
}

int wino_topk_rows(const float* vals, int rows, int cols, int k, int* idx, void* cuda_stream) {
  if (!vals || !idx || rows < 0 || cols < 1 || cols > 8192 || k < 1 || k > cols) {
    set_error("invalid arguments to wino_topk_rows (cols <= 8192, 1 <= k <= cols)");
    return WINO_EINVAL;
  }
  if (rows == 0) return WINO_OK;
  int P = 1;
  while (P < cols) P <<= 1;
  const size_t smem = (size_t)P * 8;
  static bool attr = false;
  if (!attr) {
    WINO_CUDA_TRY(
        cudaFuncSetAttribute(k_topk_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
    attr = true;
  }
  k_topk_rows<<<rows, 512, smem, (cudaStream_t)cuda_stream>>>(vals, cols, k, idx);
  note_launches(1);
  WINO_CUDA_TRY(cudaGetLastError());
  return WINO_OK;
}

void wino_mlp_destroy(void* mlp) {
  Mlp* M = (Mlp*)mlp;
  if (!M) return;
  if (M->part) cudaFree(M->part);
  cudaFree(M->buf);
  (void)cudaGetLastError();
  delete M;
}

}  // extern "C"
