// reference.cu -- the FP64 steps of the method: direct correlation (Eq. (1))
// as the reference FP32 Winograd is measured against (Sec. 6), and the
// error reduction (sum and max of |yhat - y| and |y|) with FP64 warp-shuffle
// accumulators.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/wino.h"
#include "common.cuh"

namespace wino {

// K5: one thread per output position (n, p, q) and kDirKT output channels,
// positions (p, q) of a plane flattened across the blocks, q fastest
// (neighbouring threads read neighbouring input columns; a narrow plane
// still fills the block).  The
// block's filters for kDirCC channels at a time are staged in shared memory
// already widened to FP64 (read as broadcasts), and each input value is
// widened once for the kDirKT channels it feeds: per multiply-add one FP64
// FMA and an eighth of a conversion, where converting both operands at every
// use took three FP64-pipe slots.  Every output's operations are those of
// the plain loop (c, then u, then v ascending, one fma each), so the bits do
// not depend on the blocking.
constexpr int kDirKT = 8, kDirCC = 8, kDirThreads = 128;

__global__ void __launch_bounds__(kDirThreads)
    k_direct_f64(const float* __restrict__ x, const float* __restrict__ w, double* __restrict__ y,
                 int N, int C, int K, int H, int W, int pad, int rh, int r, int padh, int Ho,
                 int Wo) {
  __shared__ double ws[kDirCC][kDirKT][kMaxR * kMaxR];
  const int64_t pq = (int64_t)blockIdx.x * kDirThreads + threadIdx.x;
  const bool live = pq < (int64_t)Ho * Wo;
  const int p = live ? (int)(pq / Wo) : 0;
  const int q = live ? (int)(pq - (int64_t)p * Wo) : 0;
  const int nk = (K + kDirKT - 1) / kDirKT;
  const int n = blockIdx.y / nk, k0 = (blockIdx.y % nk) * kDirKT;
  const int taps = rh * r;
  double acc[kDirKT];
#pragma unroll
  for (int kk = 0; kk < kDirKT; ++kk) acc[kk] = 0.0;
  for (int c0 = 0; c0 < C; c0 += kDirCC) {
    const int cn = min(kDirCC, C - c0);
    __syncthreads();  // the previous chunk's filters are no longer read
    for (int e = threadIdx.x; e < cn * kDirKT * taps; e += kDirThreads) {
      const int t = e % taps, kk = (e / taps) % kDirKT, cc = e / (taps * kDirKT);
      const int k = k0 + kk;
      ws[cc][kk][t] = k < K ? (double)__ldg(w + ((int64_t)k * C + c0 + cc) * taps + t) : 0.0;
    }
    __syncthreads();
    if (live) {
      for (int cc = 0; cc < cn; ++cc) {
        const float* xc = x + ((int64_t)n * C + c0 + cc) * H * W;
        for (int u = 0; u < rh; ++u) {
          const int hh = p + u - padh;
          if (hh < 0 || hh >= H) continue;
          for (int v = 0; v < r; ++v) {
            const int ww = q + v - pad;
            if (ww < 0 || ww >= W) continue;
            const double xv = (double)__ldg(xc + (int64_t)hh * W + ww);
#pragma unroll
            for (int kk = 0; kk < kDirKT; ++kk) acc[kk] = fma(xv, ws[cc][kk][u * r + v], acc[kk]);
          }
        }
      }
    }
  }
  if (live) {
#pragma unroll
    for (int kk = 0; kk < kDirKT; ++kk) {
      const int k = k0 + kk;
      if (k < K) y[(((int64_t)n * K + k) * Ho + p) * Wo + q] = acc[kk];
    }
  }
}

int direct_conv_f64(const float* x, const float* w, double* y, int dim, int N, int C, int K,
                    int H, int W, int pad, int r, cudaStream_t st) {
  const int rh = (dim == 1) ? 1 : r;
  const int padh = (dim == 1) ? 0 : pad;
  const int Hin = (dim == 1) ? 1 : H;
  const int Ho = (dim == 1) ? 1 : H + 2 * pad - r + 1;
  const int Wo = W + 2 * pad - r + 1;
  const int64_t total = (int64_t)N * K * Ho * Wo;
  if (total == 0) return WINO_OK;
  const int64_t nz = (int64_t)N * ((K + kDirKT - 1) / kDirKT);
  const int64_t nb = ((int64_t)Ho * Wo + kDirThreads - 1) / kDirThreads;
  if (r > kMaxR || nz > 65535 || nb > 0x7fffffffLL) {
    set_error("direct reference: r <= 7, N * ceil(K / 8) <= 65535");
    return WINO_EUNSUPPORTED;
  }
  ProfScope ps(kKDirect, st);
  const dim3 grid((unsigned)nb, (unsigned)nz);
  k_direct_f64<<<grid, kDirThreads, 0, st>>>(x, w, y, N, C, K, Hin, W, pad, rh, r, padh, Ho, Wo);
  note_launches(1);
  WINO_CUDA_TRY(cudaGetLastError());
  return WINO_OK;
}

// ---------------------------------------------------------------------------
// K6: error statistics.  Pass 1: grid-stride per-thread FP64 partials,
// warp-shuffle then shared-memory reduction, one record per block.  Pass 2:
// one block reduces the records in a fixed order, so the result does not
// depend on scheduling.
// ---------------------------------------------------------------------------
struct Stats4 {
  double s_err, s_ref, m_err, m_ref;
};

// max that propagates NaN (fmax drops a NaN operand, which would let a NaN
// output hide behind the largest finite error)
__device__ __forceinline__ double nanmax(double a, double b) {
  return (a != a) ? a : (b != b) ? b : fmax(a, b);
}

__device__ __forceinline__ Stats4 warp_reduce(Stats4 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.s_err += __shfl_down_sync(0xffffffffu, v.s_err, o);
    v.s_ref += __shfl_down_sync(0xffffffffu, v.s_ref, o);
    v.m_err = nanmax(v.m_err, __shfl_down_sync(0xffffffffu, v.m_err, o));
    v.m_ref = nanmax(v.m_ref, __shfl_down_sync(0xffffffffu, v.m_ref, o));
  }
  return v;
}

__device__ __forceinline__ Stats4 block_reduce(Stats4 v) {
  __shared__ Stats4 part[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_reduce(v);
  if (lane == 0) part[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (wid == 0) {
    v = (lane < nw) ? part[lane] : Stats4{0.0, 0.0, 0.0, 0.0};
    v = warp_reduce(v);
  }
  return v;
}

__global__ void k_error_stats_pass1(const float* __restrict__ yhat, const double* __restrict__ y,
                                    int64_t n, Stats4* __restrict__ partial) {
  Stats4 v{0.0, 0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double ref = y[i];
    const double e = fabs((double)yhat[i] - ref);
    v.s_err += e;
    v.s_ref += fabs(ref);
    v.m_err = nanmax(v.m_err, e);
    v.m_ref = nanmax(v.m_ref, fabs(ref));
  }
  v = block_reduce(v);
  if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

__global__ void k_error_stats_pass2(const Stats4* __restrict__ partial, int nb,
                                    double* __restrict__ out) {
  Stats4 v{0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const Stats4 p = partial[i];
    v.s_err += p.s_err;
    v.s_ref += p.s_ref;
    v.m_err = nanmax(v.m_err, p.m_err);
    v.m_ref = nanmax(v.m_ref, p.m_ref);
  }
  v = block_reduce(v);
  if (threadIdx.x == 0) {
    out[0] = v.s_err;
    out[1] = v.s_ref;
    out[2] = v.m_err;
    out[3] = v.m_ref;
  }
}

int error_stats(const float* yhat, const double* y, int64_t n, double* out4_host,
                cudaStream_t st) {
  int sms = 0, dev = 0;
  WINO_CUDA_TRY(cudaGetDevice(&dev));
  WINO_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int64_t want = (n + 255) / 256;
  int nb = (int)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
  if (nb < 1) nb = 1;
  void* buf = nullptr;
  int rc = scratch_get(kScratchStats, sizeof(Stats4) * nb + 64, &buf);
  if (rc != WINO_OK) return rc;
  Stats4* partial = (Stats4*)buf;
  double* out = (double*)((char*)buf + sizeof(Stats4) * nb);
  k_error_stats_pass1<<<nb, 256, 0, st>>>(yhat, y, n, partial);
  k_error_stats_pass2<<<1, 256, 0, st>>>(partial, nb, out);
  note_launches(2);
  WINO_CUDA_TRY(cudaGetLastError());
  WINO_CUDA_TRY(cudaMemcpyAsync(out4_host, out, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  WINO_CUDA_TRY(cudaStreamSynchronize(st));
  return WINO_OK;
}

}  // namespace wino
