// layer.cu -- FP32 Winograd convolution layer, Eqs. (8)-(9) per tile.
//
// Pipeline (any m, r with alpha <= 12, 1D or 2D):
//   K4 filter transform   V[f][c][k] = (G g_kc G^T)[f]
//   K1 input transform    U[f][c][t] = (B^T d_tc B)[f]   (zero padding,
//                                                          ragged tiles)
//   K2 alpha^2 GEMMs      M[f][k][t] = sum_c V[f][c][k] U[f][c][t]
//   K3 output transform   y[n][k][tile] = (A^T M_tk A), cropped
// Every FP32 value is produced in the fixed order documented in wino.h's
// companion notes: transforms output by output with fmaf over the inner
// index ascending, the contraction over c ascending with fmaf, owned by one
// thread per output, so the layer is bit-reproducible.
//
// The fused kernels for the VGG-shaped F(4x4,3x3) / F(6x6,3x3) layers live in
// fused.cu; this file is the general path they fall back to.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>

#include "../../include/wino.h"
#include "common.cuh"

namespace wino {

// ---------------------------------------------------------------------------
// K4: filter transform, one thread per (c, k), k fastest (coalesced V rows).
// ---------------------------------------------------------------------------
__global__ void k_filter_transform(const float* __restrict__ w, float* __restrict__ V, int dim,
                                   int C, int K, const LayerMats M) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)C * K) return;
  const int k = (int)(idx % K), c = (int)(idx / K);
  const int taps = (dim == 1) ? M.r : M.r * M.r;
  const int64_t plane = (int64_t)C * K;
  float* out = V + (int64_t)c * K + k;
  filter_transform_one(w + ((int64_t)k * C + c) * taps, dim, M,
                       [&](int f, float v) { out[(int64_t)f * plane] = v; });
}

// ---------------------------------------------------------------------------
// K1: input transform, one thread per (c, t), t fastest (adjacent tiles read
// adjacent input columns; U rows are written coalesced).
// ---------------------------------------------------------------------------
__global__ void k_input_transform(const float* __restrict__ x, float* __restrict__ U,
                                  const LayerGeom g, const LayerMats M) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)g.C * g.T) return;
  const int64_t t = idx % g.T;
  const int c = (int)(idx / g.T);
  const int A = M.alpha, m = M.m;
  const int tpi = g.th * g.tw;
  const int n = (int)(t / tpi);
  const int ti = (int)((t / g.tw) % g.th), tj = (int)(t % g.tw);
  const int padh = (g.dim == 1) ? 0 : g.pad;
  const float* xc = x + ((int64_t)n * g.C + c) * g.H * g.W;
  const int64_t plane = (int64_t)g.C * g.T;
  float* out = U + (int64_t)c * g.T + t;
  float d[kMaxAlpha * kMaxAlpha];
  const int rows = (g.dim == 1) ? 1 : A;
  for (int i = 0; i < rows; ++i) {
    const int hh = ti * m - padh + i;
    for (int j = 0; j < A; ++j) {
      const int ww = tj * m - g.pad + j;
      float v = 0.0f;
      if (hh >= 0 && hh < g.H && ww >= 0 && ww < g.W) v = __ldg(xc + (int64_t)hh * g.W + ww);
      d[i * A + j] = v;
    }
  }
  if (g.dim == 1) {
    for (int i = 0; i < A; ++i) {
      float acc = 0.0f;
      for (int l = 0; l < A; ++l) acc = fmaf(M.BT[i * A + l], d[l], acc);
      out[i * plane] = acc;
    }
    return;
  }
  float Tm[kMaxAlpha * kMaxAlpha];
  for (int i = 0; i < A; ++i)
    for (int l = 0; l < A; ++l) {
      float acc = 0.0f;
      for (int q = 0; q < A; ++q) acc = fmaf(M.BT[i * A + q], d[q * A + l], acc);
      Tm[i * A + l] = acc;
    }
  for (int i = 0; i < A; ++i)
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
      for (int l = 0; l < A; ++l) acc = fmaf(Tm[i * A + l], M.BT[j * A + l], acc);
      out[(int64_t)(i * A + j) * plane] = acc;
    }
}

// ---------------------------------------------------------------------------
// K2: F independent GEMMs  M[f][k][t] = sum_c V[f][c][k] U[f][c][t].
// Block tile BM (k) x BN (t), BK = 8 channels per stage, 256 threads in a
// 16 x 16 grid, each owning a TM x TN register microtile and accumulating
// over c in ascending order (no split of the reduction).
// ---------------------------------------------------------------------------
template <int BM, int BN>
__global__ void __launch_bounds__(256) k_wino_gemm(const float* __restrict__ V,
                                                   const float* __restrict__ U,
                                                   float* __restrict__ Mo, int C, int K,
                                                   int64_t T) {
  constexpr int BK = 8, TM = BM / 16, TN = BN / 16;
  __shared__ float As[2][BK][BM];
  __shared__ float Bs[2][BK][BN];
  const int f = blockIdx.z;
  const int k0 = blockIdx.y * BM;
  const int64_t t0 = (int64_t)blockIdx.x * BN;
  const float* Vf = V + (int64_t)f * C * K;
  const float* Uf = U + (int64_t)f * C * T;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;

  constexpr int A_PER = BK * BM / 256, B_PER = BK * BN / 256;
  float ra[A_PER], rb[B_PER];
  auto load_regs = [&](int c0) {
#pragma unroll
    for (int q = 0; q < A_PER; ++q) {
      const int e = tid + q * 256;
      const int kk = e / BM, col = e % BM;
      const int c = c0 + kk, k = k0 + col;
      ra[q] = (c < C && k < K) ? __ldg(Vf + (int64_t)c * K + k) : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < B_PER; ++q) {
      const int e = tid + q * 256;
      const int kk = e / BN, col = e % BN;
      const int c = c0 + kk;
      const int64_t t = t0 + col;
      rb[q] = (c < C && t < T) ? __ldg(Uf + (int64_t)c * T + t) : 0.0f;
    }
  };
  auto store_smem = [&](int buf) {
#pragma unroll
    for (int q = 0; q < A_PER; ++q) {
      const int e = tid + q * 256;
      As[buf][e / BM][e % BM] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < B_PER; ++q) {
      const int e = tid + q * 256;
      Bs[buf][e / BN][e % BN] = rb[q];
    }
  };

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;

  const int nchunks = (C + BK - 1) / BK;
  load_regs(0);
  store_smem(0);
  __syncthreads();
  for (int ch = 0; ch < nchunks; ++ch) {
    const int buf = ch & 1;
    if (ch + 1 < nchunks) load_regs((ch + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (ch + 1 < nchunks) store_smem(buf ^ 1);
    __syncthreads();
  }
  float* Mf = Mo + (int64_t)f * K * T;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int k = k0 + ty * TM + i;
    if (k >= K) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t t = t0 + tx * TN + j;
      if (t < T) Mf[(int64_t)k * T + t] = acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------
// K3: output transform and write-back, one thread per (k, t), t fastest.
// ---------------------------------------------------------------------------
__global__ void k_output_transform(const float* __restrict__ Mi, float* __restrict__ y,
                                   const LayerGeom g, const LayerMats M) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)g.K * g.T) return;
  const int64_t t = idx % g.T;
  const int k = (int)(idx / g.T);
  const int A = M.alpha, m = M.m;
  const int tpi = g.th * g.tw;
  const int n = (int)(t / tpi);
  const int ti = (int)((t / g.tw) % g.th), tj = (int)(t % g.tw);
  const int64_t plane = (int64_t)g.K * g.T;
  const float* in = Mi + (int64_t)k * g.T + t;
  float Mf[kMaxAlpha * kMaxAlpha];
  for (int f = 0; f < g.F; ++f) Mf[f] = in[f * plane];
  float* yk = y + ((int64_t)n * g.K + k) * g.Ho * g.Wo;
  if (g.dim == 1) {
    for (int j = 0; j < m; ++j) {
      float acc = 0.0f;
      for (int i = 0; i < A; ++i) acc = fmaf(M.AT[j * A + i], Mf[i], acc);
      const int q = tj * m + j;
      if (q < g.Wo) yk[q] = acc;
    }
    return;
  }
  float Z[kMaxAlpha * kMaxAlpha];
  for (int a = 0; a < m; ++a)
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
      for (int i = 0; i < A; ++i) acc = fmaf(M.AT[a * A + i], Mf[i * A + j], acc);
      Z[a * A + j] = acc;
    }
  for (int a = 0; a < m; ++a) {
    const int p = ti * m + a;
    if (p >= g.Ho) break;
    for (int b = 0; b < m; ++b) {
      float acc = 0.0f;
      for (int j = 0; j < A; ++j) acc = fmaf(Z[a * A + j], M.AT[b * A + j], acc);
      const int q = tj * m + b;
      if (q < g.Wo) yk[(int64_t)p * g.Wo + q] = acc;
    }
  }
}

// Fused path (fused.cu): returns kFallback when the shape has no fused
// kernel, so the general path below runs.
int layer_forward_fused(const float* x, const float* w, float* y, const LayerGeom& g,
                        const LayerMats& M, void* ws, size_t ws_bytes, cudaStream_t st);
size_t fused_workspace_bytes(const LayerGeom& g);
size_t tc_workspace_bytes(const LayerGeom& g, int dtype);

size_t split_workspace_bytes(const LayerGeom& g);

size_t layer_workspace_bytes(const LayerGeom& g, int dtype) {
  const size_t F = (size_t)g.F;
  const size_t v = F * g.C * g.K * sizeof(float);
  const size_t u = F * g.C * (size_t)g.T * sizeof(float);
  const size_t mm = F * g.K * (size_t)g.T * sizeof(float);
  size_t general = v + u + mm + 1024;
  if (dtype != 0) return tc_workspace_bytes(g, dtype);
  const size_t split = split_workspace_bytes(g);
  return split > general ? split : general;
}

int layer_forward_general_f32(const float* x, const float* w, float* y, const LayerGeom& g,
                              const LayerMats& M, void* ws, cudaStream_t st) {
  const size_t F = (size_t)g.F;
  float* V = (float*)ws;
  float* U = V + F * g.C * g.K;
  float* Mb = U + F * g.C * (size_t)g.T;
  {
    const int64_t n = (int64_t)g.C * g.K;
    ProfScope ps(kKFilter, st);
    k_filter_transform<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, V, g.dim, g.C, g.K, M);
  }
  {
    const int64_t n = (int64_t)g.C * g.T;
    ProfScope ps(kKInput, st);
    k_input_transform<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, U, g, M);
  }
  {
    ProfScope ps(kKGemm, st);
    if (g.K > 64) {
      dim3 grid((unsigned)((g.T + 127) / 128), (unsigned)((g.K + 127) / 128), (unsigned)F);
      k_wino_gemm<128, 128><<<grid, 256, 0, st>>>(V, U, Mb, g.C, g.K, g.T);
    } else {
      dim3 grid((unsigned)((g.T + 127) / 128), (unsigned)((g.K + 63) / 64), (unsigned)F);
      k_wino_gemm<64, 128><<<grid, 256, 0, st>>>(V, U, Mb, g.C, g.K, g.T);
    }
  }
  {
    const int64_t n = (int64_t)g.K * g.T;
    ProfScope ps(kKOutput, st);
    k_output_transform<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Mb, y, g, M);
  }
  note_launches(4);
  WINO_CUDA_TRY(cudaGetLastError());
  return 0;
}

int layer_forward_split(const float* x, const float* w, float* y, const LayerGeom& g,
                        const LayerMats& M, void* ws, size_t ws_bytes, cudaStream_t st, int cfg);
int split_configs(int m);

// ---------------------------------------------------------------------------
// Variant choice for the FP32 layer (autotuner): the fully fused kernel
// (fused.cu), the split transform + GEMM/output kernels (fused.cu) in each
// of its tile shapes, and the general pipeline above compute the same bits;
// which is fastest depends on the shape.  The first call for a shape times
// the fused variant and every split tile shape on the caller's stream
// (three runs each, keeping the faster of the last two) and caches the
// fastest for the process.
// Timing synchronises the stream, so it is skipped while the stream is being
// captured into a graph (split tile shape 0 is used then) and when
// WINO_AUTOTUNE=0.  WINO_LAYER_VARIANT=fused|split|split<c>|general forces a
// variant (split<c>: split tile shape c = 1..9; a shape the layer does not
// have falls back as below).
// ---------------------------------------------------------------------------
enum LayerVariant {
  kVarUnknown = 0,
  kVarFused = 1,
  kVarSplit = 2,  // split tile shape 0
  kVarGeneral = 3,
  kVarSplitN = 16  // kVarSplitN + c: split tile shape c >= 1
};

static std::mutex g_var_mu;
static std::map<std::string, int> g_var_cache;

static std::string layer_key(const LayerGeom& g, const LayerMats& M) {
  char buf[160];
  snprintf(buf, sizeof(buf), "d%d m%d r%d N%d C%d K%d H%d W%d p%d", g.dim, M.m, M.r, g.N, g.C,
           g.K, g.H, g.W, g.pad);
  return buf;
}

static int forced_variant() {
  const char* v = getenv("WINO_LAYER_VARIANT");
  if (!v) return kVarUnknown;
  if (!strcmp(v, "fused")) return kVarFused;
  if (!strcmp(v, "split")) return kVarSplit;
  if (!strncmp(v, "split", 5) && v[5] >= '1' && v[5] <= '9' && v[6] == 0)
    return kVarSplitN + (v[5] - '0');
  if (!strcmp(v, "general")) return kVarGeneral;
  return kVarUnknown;
}

static int run_variant(int var, const float* x, const float* w, float* y, const LayerGeom& g,
                       const LayerMats& M, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (var == kVarFused) return layer_forward_fused(x, w, y, g, M, ws, ws_bytes, st);
  if (var == kVarSplit) return layer_forward_split(x, w, y, g, M, ws, ws_bytes, st, 0);
  if (var > kVarSplitN)
    return layer_forward_split(x, w, y, g, M, ws, ws_bytes, st, var - kVarSplitN);
  return layer_forward_general_f32(x, w, y, g, M, ws, st);
}

static int tune_variant(const float* x, const float* w, float* y, const LayerGeom& g,
                        const LayerMats& M, void* ws, size_t ws_bytes, cudaStream_t st,
                        int* out) {
  cudaEvent_t a, b;
  WINO_CUDA_TRY(cudaEventCreate(&a));
  WINO_CUDA_TRY(cudaEventCreate(&b));
  float best = 1e30f;
  int best_var = kVarGeneral;
  int cands[16], nc = 0;
  cands[nc++] = kVarSplit;
  for (int c = 1; c < split_configs(M.m) && nc < 15; ++c) cands[nc++] = kVarSplitN + c;
  cands[nc++] = kVarFused;
  for (int ci = 0; ci < nc; ++ci) {
    const int var = cands[ci];
    float ms = 1e30f;
    bool ok = true;
    for (int rep = 0; rep < 3 && ok; ++rep) {
      WINO_CUDA_TRY(cudaEventRecord(a, st));
      int rc = run_variant(var, x, w, y, g, M, ws, ws_bytes, st);
      if (rc == kFallback) {
        ok = false;
        break;
      }
      if (rc != WINO_OK) return rc;
      WINO_CUDA_TRY(cudaEventRecord(b, st));
      WINO_CUDA_TRY(cudaEventSynchronize(b));
      float t = 0.0f;
      WINO_CUDA_TRY(cudaEventElapsedTime(&t, a, b));
      if (rep > 0 && t < ms) ms = t;  // the first run warms up
    }
    if (ok && ms < best) {
      best = ms;
      best_var = var;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *out = best_var;
  return WINO_OK;
}

int layer_forward_f32(const float* x, const float* w, float* y, const LayerGeom& g,
                      const LayerMats& M, void* ws, size_t ws_bytes, cudaStream_t st) {
  int var = forced_variant();
  if (var == kVarUnknown) {
    const std::string key = layer_key(g, M);
    {
      std::lock_guard<std::mutex> lk(g_var_mu);
      auto it = g_var_cache.find(key);
      if (it != g_var_cache.end()) var = it->second;
    }
    if (var == kVarUnknown) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;
      }
      const char* at = getenv("WINO_AUTOTUNE");
      if (cs == cudaStreamCaptureStatusNone && !(at && !strcmp(at, "0"))) {
        int rc = tune_variant(x, w, y, g, M, ws, ws_bytes, st, &var);
        if (rc != WINO_OK) return rc;
        std::lock_guard<std::mutex> lk(g_var_mu);
        g_var_cache[key] = var;
      } else {
        var = kVarSplit;
      }
    }
  }
  int rc = run_variant(var, x, w, y, g, M, ws, ws_bytes, st);
  if (rc == kFallback && var != kVarGeneral) {
    rc = layer_forward_split(x, w, y, g, M, ws, ws_bytes, st, 0);
    if (rc == kFallback) rc = layer_forward_fused(x, w, y, g, M, ws, ws_bytes, st);
  }
  if (rc == kFallback) rc = layer_forward_general_f32(x, w, y, g, M, ws, st);
  return rc;
}

}  // namespace wino
