// tc_gemm.cu -- precision form of the Winograd-domain contraction on the
// 5th-generation tensor cores (tcgen05.mma, accumulators in TMEM).
//
// The transforms stay FP32 (same operation order as the FP32 layer); only the
// alpha^2 contractions M[f] = U[f] V[f] change:
//   WINO_BF16_TC       U, V rounded to BF16, FP32 accumulation
//   WINO_FP16_TC       U, V rounded to FP16, FP32 accumulation
//   WINO_SPLIT_BF16X3  a = hi + lo with hi = RN_bf16(a), lo = RN_bf16(a - hi);
//                      U V ~ Uhi Vhi + Uhi Vlo + Ulo Vhi (three MMAs into one
//                      accumulator)
// Per-frequency scaling (exact powers of two, undone before the output
// transform): U[f] by the power of two that brings |BT_i|_1 |BT_j|_1 into
// [1, 2), V[f] by the one that brings max |V[f]| into [1, 2).  This keeps FP16
// operands in range; for BF16 it only guards the subnormal range of lo.
//
// Pipeline: filter transform (FP32) -> per-frequency max |V| -> V rounded
// into [F][K][Cp] (K-major B operand); input transform (FP32) rounded into
// [F][Tp][Cp] (K-major A operand); k_tc_gemm; the general output transform.
// k_tc_gemm: one CTA = one frequency x 128 tiles (MMA M) x NB output
// channels (MMA N <= 256), contraction over Cp in chunks of 64 channels
// (one 128-byte swizzle row per operand row).  Operands are staged by
// cp.async into the SWIZZLE_128B K-major layout; one thread issues
// tcgen05.mma (K = 16 per instruction) and commits to an mbarrier; every
// wait on it is bounded and records an error instead of hanging.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "../../include/wino.h"
#include "common.cuh"

namespace wino {

__global__ void k_filter_transform(const float* __restrict__ w, float* __restrict__ V, int dim,
                                   int C, int K, const LayerMats M);
__global__ void k_output_transform(const float* __restrict__ Mi, float* __restrict__ y,
                                   const LayerGeom g, const LayerMats M);

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// 16-bit rounding of a scaled FP32 value; mode 1/3 BF16, 2 FP16.
__device__ __forceinline__ uint16_t round16(float v, int mode) {
  if (mode == 2) return __half_as_ushort(__float2half_rn(v));
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float widen16(uint16_t b, int mode) {
  if (mode == 2) return __half2float(__ushort_as_half(b));
  return __bfloat162float(__ushort_as_bfloat16(b));
}

// 2^(1-e) for m = f 2^e, f in [0.5, 1): brings m into [1, 2).
__device__ __forceinline__ float pow2_normaliser(float m) {
  if (!(m > 0.0f) || isinf(m)) return 1.0f;
  int e;
  frexpf(m, &e);
  return ldexpf(1.0f, 1 - e);
}

}  // namespace

struct TcScales {
  float sU[kMaxAlpha * kMaxAlpha];
};

// ---------------------------------------------------------------------------
// Operand preparation.
// ---------------------------------------------------------------------------
// max |V| of each frequency plane: block (x, f) reduces a grid-stride slice
// of plane f (warp shuffles, then shared memory) and issues ONE atomicMax on
// the bit pattern (non-negative floats order like their bits), so a plane of
// C K values costs gridDim.x atomics, not C K.
constexpr int kVmaxThreads = 256;
__global__ void __launch_bounds__(kVmaxThreads) k_vmax(const float* __restrict__ V, int64_t plane,
                                                       unsigned* __restrict__ vmax_bits) {
  const int f = blockIdx.y;
  const float* p = V + (int64_t)f * plane;
  float mx = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * kVmaxThreads + threadIdx.x; i < plane;
       i += (int64_t)gridDim.x * kVmaxThreads)
    mx = fmaxf(mx, fabsf(p[i]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ float wm[kVmaxThreads / 32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kVmaxThreads / 32; ++w) mx = fmaxf(mx, wm[w]);
    atomicMax(vmax_bits + f, __float_as_uint(mx));
  }
}

// V32[f][c][k] -> Vh/Vl[f][k][c] (c padded to Cp with zeros), scaled.
__global__ void k_quant_v(const float* __restrict__ V, int C, int K, int Cp, int F,
                          const unsigned* __restrict__ vmax_bits, float* __restrict__ sV,
                          uint16_t* __restrict__ Vh, uint16_t* __restrict__ Vl, int mode) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)F * K * Cp;
  if (idx >= total) return;
  const int c = (int)(idx % Cp);
  const int k = (int)((idx / Cp) % K);
  const int f = (int)(idx / ((int64_t)Cp * K));
  const float s = pow2_normaliser(__uint_as_float(vmax_bits[f]));
  if (c == 0 && k == 0) sV[f] = s;
  float v = 0.0f;
  if (c < C) v = V[((int64_t)f * C + c) * K + k] * s;
  const uint16_t h = round16(v, mode);
  Vh[idx] = h;
  if (mode == 3) Vl[idx] = round16(v - widen16(h, mode), mode);
}

// Input transform (FP32, the FP32 layer's order) -> Uh/Ul[f][t][c], scaled.
// One thread per (t, c), c fastest: each frequency row is written
// contiguously; rows t >= T and columns c >= C are zero.
template <int MM>
__global__ void __launch_bounds__(256) k_quant_input(const float* __restrict__ x, const LayerGeom g,
                                                     const LayerMats Mx, const TcScales S, int Cp,
                                                     int64_t Tp, uint16_t* __restrict__ Uh,
                                                     uint16_t* __restrict__ Ul, int mode) {
  constexpr int A = MM + 2;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Tp * Cp) return;
  const int c = (int)(idx % Cp);
  const int64_t t = idx / Cp;
  float d[A][A];
  const bool live = t < g.T && c < g.C;
  if (live) {
    const int tpi = g.th * g.tw;
    const int n = (int)(t / tpi);
    const int rem = (int)(t - (int64_t)n * tpi);
    const int ti = rem / g.tw, tj = rem - (rem / g.tw) * g.tw;
    const int h0 = ti * MM - g.pad, w0 = tj * MM - g.pad;
    const float* xc = x + ((int64_t)n * g.C + c) * g.H * g.W;
#pragma unroll
    for (int i = 0; i < A; ++i)
#pragma unroll
      for (int j = 0; j < A; ++j) {
        const int hh = h0 + i, ww = w0 + j;
        d[i][j] = ((unsigned)hh < (unsigned)g.H && (unsigned)ww < (unsigned)g.W)
                      ? __ldg(xc + (int64_t)hh * g.W + ww)
                      : 0.0f;
      }
  } else {
#pragma unroll
    for (int i = 0; i < A; ++i)
#pragma unroll
      for (int j = 0; j < A; ++j) d[i][j] = 0.0f;
  }
  float tm[A][A];
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int l = 0; l < A; ++l) {
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < A; ++q) acc = fmaf(Mx.BT[i * A + q], d[q][l], acc);
      tm[i][l] = acc;
    }
  const int64_t plane = Tp * Cp;
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
#pragma unroll
      for (int l = 0; l < A; ++l) acc = fmaf(tm[i][l], Mx.BT[j * A + l], acc);
      const int f = i * A + j;
      const float v = live ? acc * S.sU[f] : 0.0f;
      const uint16_t h = round16(v, mode);
      Uh[f * plane + idx] = h;
      if (mode == 3) Ul[f * plane + idx] = round16(v - widen16(h, mode), mode);
    }
}

// Tiled form of the same input quantisation: one block = 16 tiles x 16
// channels; a thread transforms one (tile, channel) with tiles fastest
// (neighbouring patches share input rows), the 16-bit results meet in
// shared memory and leave as 32-byte rows of 16 channels.
constexpr int kQT = 16, kQC = 16;
template <int MM>
__global__ void __launch_bounds__(kQT* kQC) k_quant_input_tiled(
    const float* __restrict__ x, const LayerGeom g, const LayerMats Mx, const TcScales S, int Cp,
    int64_t Tp, uint16_t* __restrict__ Uh, uint16_t* __restrict__ Ul, int mode) {
  constexpr int A = MM + 2, F = A * A;
  extern __shared__ __align__(16) uint16_t qs[];  // [2][F][kQT][kQC]
  const int tl = threadIdx.x % kQT, cl = threadIdx.x / kQT;
  const int64_t t = (int64_t)blockIdx.x * kQT + tl;
  const int c = blockIdx.y * kQC + cl;
  const bool live = t < g.T && c < g.C;
  float d[A][A];
  if (live) {
    const int tpi = g.th * g.tw;
    const int n = (int)(t / tpi);
    const int rem = (int)(t - (int64_t)n * tpi);
    const int ti = rem / g.tw, tj = rem - (rem / g.tw) * g.tw;
    const int h0 = ti * MM - g.pad, w0 = tj * MM - g.pad;
    const float* xc = x + ((int64_t)n * g.C + c) * g.H * g.W;
#pragma unroll
    for (int i = 0; i < A; ++i)
#pragma unroll
      for (int j = 0; j < A; ++j) {
        const int hh = h0 + i, ww = w0 + j;
        d[i][j] = ((unsigned)hh < (unsigned)g.H && (unsigned)ww < (unsigned)g.W)
                      ? __ldg(xc + (int64_t)hh * g.W + ww)
                      : 0.0f;
      }
  } else {
#pragma unroll
    for (int i = 0; i < A; ++i)
#pragma unroll
      for (int j = 0; j < A; ++j) d[i][j] = 0.0f;
  }
  float tm[A][A];
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int l = 0; l < A; ++l) {
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < A; ++q) acc = fmaf(Mx.BT[i * A + q], d[q][l], acc);
      tm[i][l] = acc;
    }
  uint16_t* sh = qs;
  uint16_t* sl = qs + F * kQT * kQC;
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
#pragma unroll
      for (int l = 0; l < A; ++l) acc = fmaf(tm[i][l], Mx.BT[j * A + l], acc);
      const int f = i * A + j;
      const float v = live ? acc * S.sU[f] : 0.0f;
      const uint16_t h = round16(v, mode);
      sh[(f * kQT + tl) * kQC + cl] = h;
      if (mode == 3) sl[(f * kQT + tl) * kQC + cl] = round16(v - widen16(h, mode), mode);
    }
  __syncthreads();
  // rows (f, tile) of 16 channels = 32 bytes = two 16-byte stores
  const int64_t plane = Tp * Cp;
  const int64_t tb = (int64_t)blockIdx.x * kQT;
  const int c0 = blockIdx.y * kQC;
  for (int e = threadIdx.x; e < F * kQT * 2; e += kQT * kQC) {
    const int half = e & 1, row = e >> 1;  // row = f * kQT + tl
    const int f = row / kQT, tr = row % kQT;
    const int64_t dst = f * plane + (tb + tr) * Cp + c0 + half * 8;
    *reinterpret_cast<uint4*>(Uh + dst) = *reinterpret_cast<const uint4*>(sh + row * kQC + half * 8);
    if (mode == 3)
      *reinterpret_cast<uint4*>(Ul + dst) =
          *reinterpret_cast<const uint4*>(sl + row * kQC + half * 8);
  }
}

// Output transform A^T M A with compile-time sizes, M [F][K][T]: one thread
// per (k, tile), tiles fastest (coalesced M reads, adjacent output segments).
template <int MM>
__global__ void __launch_bounds__(256) k_output_transform_r3(const float* __restrict__ Mi,
                                                             float* __restrict__ y,
                                                             const LayerGeom g,
                                                             const LayerMats Mx) {
  constexpr int A = MM + 2;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)g.K * g.T) return;
  const int64_t t = idx % g.T;
  const int k = (int)(idx / g.T);
  const int64_t plane = (int64_t)g.K * g.T;
  const float* in = Mi + (int64_t)k * g.T + t;
  float Mv[A * A];
#pragma unroll
  for (int f = 0; f < A * A; ++f) Mv[f] = in[f * plane];
  float Z[MM][A];
#pragma unroll
  for (int a = 0; a < MM; ++a)
#pragma unroll
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
#pragma unroll
      for (int i = 0; i < A; ++i) acc = fmaf(Mx.AT[a * A + i], Mv[i * A + j], acc);
      Z[a][j] = acc;
    }
  const int tpi = g.th * g.tw;
  const int n = (int)(t / tpi);
  const int rem = (int)(t - (int64_t)n * tpi);
  const int ti = rem / g.tw, tj = rem - (rem / g.tw) * g.tw;
  float* yk = y + ((int64_t)n * g.K + k) * g.Ho * g.Wo;
#pragma unroll
  for (int a = 0; a < MM; ++a) {
    const int p = ti * MM + a;
#pragma unroll
    for (int b = 0; b < MM; ++b) {
      float acc = 0.0f;
#pragma unroll
      for (int j = 0; j < A; ++j) acc = fmaf(Z[a][j], Mx.AT[b * A + j], acc);
      const int q = tj * MM + b;
      if (p < g.Ho && q < g.Wo) yk[(int64_t)p * g.Wo + q] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// tcgen05 contraction.
// ---------------------------------------------------------------------------
namespace {

// Shared-memory matrix descriptor, K-major operand rows of 128 bytes with
// the 128-byte swizzle: start address >> 4 (bits 0-13), leading byte offset
// (unused for this layout, 16 bytes; bits 16-29), stride byte offset between
// 8-row groups = 1024 bytes (bits 32-45), descriptor version 1 (bits 46-47),
// layout SWIZZLE_128B = 2 (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A and B format
// (bits 7-9, 10-12: 0 = F16, 1 = BF16), both K-major (bits 15, 16 = 0),
// N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ __forceinline__ uint32_t f16_idesc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
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

__device__ __forceinline__ void cp_async16_tc(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}

}  // namespace

constexpr int kTcM = 128;    // tiles per CTA (MMA M)
constexpr int kTcKc = 64;    // channels per chunk: one 128-byte row per operand row
constexpr int kTcThreads = 128;

struct TcGemmArgs {
  const uint16_t *Uh, *Ul, *Vh, *Vl;
  const float* sV;
  float* M;  // [F][K][T]
  int* err;  // set to 1 when a bounded wait gives up
  TcScales S;
  int64_t T, Tp;
  int K, Cp, NB, ncols, mode;
};

// Dynamic shared memory: per operand a 1024-byte-aligned tile: A 128 x 64 and
// B NB x 64 16-bit values (hi, and lo for the split form), then the
// mbarrier and the TMEM address.
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_gemm(const TcGemmArgs P) {
  extern __shared__ __align__(1024) unsigned char tsm_raw[];
  // the swizzled tiles must start on 1024-byte boundaries (the host asks for
  // 1 KiB of slack)
  unsigned char* tsm = tsm_raw + ((1024u - (smem_addr(tsm_raw) & 1023u)) & 1023u);
  const int f = blockIdx.z;
  const int64_t t0 = (int64_t)blockIdx.x * kTcM;
  const int n0 = blockIdx.y * P.NB;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool split = P.mode == 3;
  const uint32_t a_bytes = kTcM * 128, b_bytes = P.NB * 128;
  unsigned char* Ah = tsm;
  unsigned char* Bh = Ah + a_bytes;
  unsigned char* Al = Bh + b_bytes;
  unsigned char* Bl = Al + (split ? a_bytes : 0);
  unsigned char* tail = Bl + (split ? b_bytes : 0);
  uint64_t* bar = reinterpret_cast<uint64_t*>(tail);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tail + 8);
  const uint32_t bar_a = smem_addr(bar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_addr(tmem_holder)),
                 "r"(P.ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_holder;

  const int fmt = (P.mode == 2) ? 0 : 1;
  const uint32_t idesc = f16_idesc(fmt, kTcM, P.NB);
  const int nchunks = P.Cp / kTcKc;
  const int64_t aplane = P.Tp * P.Cp;
  const int64_t bplane = (int64_t)P.K * P.Cp;
  bool ok = true;
  for (int ch = 0; ch < nchunks && ok; ++ch) {
    const int c0 = ch * kTcKc;
    // stage A (128 rows) and B (NB rows), 8 x 16-byte chunks per row, with
    // the 128-byte swizzle: chunk j of row r goes to position j ^ (r & 7)
    for (int e = tid; e < kTcM * 8; e += kTcThreads) {
      const int r = e >> 3, j = e & 7;
      const uint32_t off = r * 128 + ((j ^ (r & 7)) << 4);
      const int64_t g = f * aplane + (t0 + r) * P.Cp + c0 + j * 8;
      cp_async16_tc(smem_addr(Ah + off), P.Uh + g);
      if (split) cp_async16_tc(smem_addr(Al + off), P.Ul + g);
    }
    for (int e = tid; e < P.NB * 8; e += kTcThreads) {
      const int r = e >> 3, j = e & 7;
      const uint32_t off = r * 128 + ((j ^ (r & 7)) << 4);
      const int64_t g = f * bplane + (int64_t)(n0 + r) * P.Cp + c0 + j * 8;
      cp_async16_tc(smem_addr(Bh + off), P.Vh + g);
      if (split) cp_async16_tc(smem_addr(Bl + off), P.Vl + g);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kTcKc / 16; ++kk) {
        const uint32_t acc = (ch > 0 || kk > 0) ? 1u : 0u;
        const uint64_t ah = sw128_desc(smem_addr(Ah) + kk * 32);
        const uint64_t bh = sw128_desc(smem_addr(Bh) + kk * 32);
        mma_f16(tmem, ah, bh, idesc, acc);
        if (split) {
          const uint64_t al = sw128_desc(smem_addr(Al) + kk * 32);
          const uint64_t bl = sw128_desc(smem_addr(Bl) + kk * 32);
          mma_f16(tmem, ah, bl, idesc, 1u);
          mma_f16(tmem, al, bh, idesc, 1u);
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              bar_a)
          : "memory");
    }
    // every thread waits for this chunk's MMAs before the tiles are reused
    if (!mbar_wait(bar_a, (uint32_t)(ch & 1))) {
      ok = false;
      if (lane == 0) atomicExch(P.err, 1);
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  if (ok) {
    // epilogue: warp w reads TMEM lanes 32w..32w+31 (tiles), 16 columns per load
    const float inv = 1.0f / (P.S.sU[f] * P.sV[f]);  // exact: powers of two
    const int64_t t = t0 + warp * 32 + lane;
    for (int col = 0; col < P.NB; col += 16) {
      uint32_t v[16];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)col;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (t < P.T) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          P.M[((int64_t)f * P.K + n0 + col + j) * P.T + t] = __uint_as_float(v[j]) * inv;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(P.ncols));
  }
}

static size_t tc_smem_bytes(int NB, bool split) {
  const size_t a = (size_t)kTcM * 128, b = (size_t)NB * 128;
  size_t s = (a + b) * (split ? 2 : 1) + 64 + 1024;
  // at most two CTAs per SM, so their TMEM columns (NB <= 256 each) fit
  return s < 80 * 1024 ? 80 * 1024 : s;
}

// Workspace layout of the precision form (bytes), all 1024-aligned.
struct TcLayout {
  size_t V32, vmax, sV, err, Vh, Vl, Uh, Ul, M, total;
};

static TcLayout tc_layout(const LayerGeom& g, int dtype) {
  auto al = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
  const int64_t Tp = (g.T + kTcM - 1) / kTcM * kTcM;
  const int Cp = (g.C + kTcKc - 1) / kTcKc * kTcKc;
  const bool split = dtype == WINO_SPLIT_BF16X3;
  TcLayout L;
  size_t o = 0;
  L.V32 = o;
  o = al(o + (size_t)g.F * g.C * g.K * 4);
  L.vmax = o;
  o = al(o + (size_t)g.F * 4);
  L.sV = o;
  o = al(o + (size_t)g.F * 4);
  L.err = o;
  o = al(o + 64);
  L.Vh = o;
  o = al(o + (size_t)g.F * g.K * Cp * 2);
  L.Vl = o;
  o = al(o + (split ? (size_t)g.F * g.K * Cp * 2 : 0));
  L.Uh = o;
  o = al(o + (size_t)g.F * Tp * Cp * 2);
  L.Ul = o;
  o = al(o + (split ? (size_t)g.F * Tp * Cp * 2 : 0));
  L.M = o;
  o = al(o + (size_t)g.F * g.K * g.T * 4);
  L.total = o;
  return L;
}

size_t tc_workspace_bytes(const LayerGeom& g, int dtype) { return tc_layout(g, dtype).total; }

static int tc_nb(int K) {
  const int cands[5] = {256, 128, 64, 32, 16};
  for (int nb : cands)
    if (K % nb == 0) return nb;
  return 0;
}

int layer_forward_tc(const float* x, const float* w, float* y, const LayerGeom& g,
                     const LayerMats& M, int dtype, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (g.dim != 2 || M.r != 3 || (M.m != 2 && M.m != 4 && M.m != 6)) {
    set_error("tensor-core forms support 2D F(m x m, 3 x 3), m in {2, 4, 6}");
    return WINO_EUNSUPPORTED;
  }
  const int NB = tc_nb(g.K);
  if (NB == 0) {
    set_error("tensor-core forms need K a multiple of 16");
    return WINO_EUNSUPPORTED;
  }
  const TcLayout L = tc_layout(g, dtype);
  if (ws_bytes < L.total) {
    set_error("workspace too small for the tensor-core form");
    return WINO_ENOMEM;
  }
  const int mode = dtype;  // 1 bf16, 2 fp16, 3 split bf16
  char* b = (char*)ws;
  float* V32 = (float*)(b + L.V32);
  unsigned* vmax = (unsigned*)(b + L.vmax);
  float* sV = (float*)(b + L.sV);
  int* err = (int*)(b + L.err);
  uint16_t* Vh = (uint16_t*)(b + L.Vh);
  uint16_t* Vl = (uint16_t*)(b + L.Vl);
  uint16_t* Uh = (uint16_t*)(b + L.Uh);
  uint16_t* Ul = (uint16_t*)(b + L.Ul);
  float* Mb = (float*)(b + L.M);
  const int64_t Tp = (g.T + kTcM - 1) / kTcM * kTcM;
  const int Cp = (g.C + kTcKc - 1) / kTcKc * kTcKc;
  const bool split = dtype == WINO_SPLIT_BF16X3;

  // per-frequency scale of U from the transform's row norms (host, exact)
  TcScales S;
  {
    const int A = M.alpha;
    double rown[kMaxAlpha];
    for (int i = 0; i < A; ++i) {
      double s = 0.0;
      for (int l = 0; l < A; ++l) s += fabs((double)M.BT[i * A + l]);
      rown[i] = s;
    }
    for (int f = 0; f < g.F; ++f) {
      const double gain = rown[f / A] * rown[f % A];
      int e = 0;
      frexp(gain, &e);
      S.sU[f] = (gain > 0.0) ? (float)ldexp(1.0, 1 - e) : 1.0f;
    }
  }
  WINO_CUDA_TRY(cudaMemsetAsync(vmax, 0, (size_t)g.F * 4, st));
  WINO_CUDA_TRY(cudaMemsetAsync(err, 0, 4, st));
  {
    ProfScope ps(kKTcTransform, st);
    const int64_t n = (int64_t)g.C * g.K;
    k_filter_transform<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, V32, g.dim, g.C, g.K, M);
    const int64_t plane = (int64_t)g.C * g.K;
    const unsigned bx = (unsigned)std::min<int64_t>(256, (plane + 8 * kVmaxThreads - 1) /
                                                            (8 * kVmaxThreads));
    k_vmax<<<dim3(bx, (unsigned)g.F), kVmaxThreads, 0, st>>>(V32, plane, vmax);
    const int64_t nq = (int64_t)g.F * g.K * Cp;
    k_quant_v<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(V32, g.C, g.K, Cp, g.F, vmax, sV, Vh,
                                                            Vl, mode);
    const dim3 gq((unsigned)(Tp / kQT), (unsigned)(Cp / kQC));
    const size_t qsm = (size_t)2 * g.F * kQT * kQC * sizeof(uint16_t);
    static bool qattr[16] = {false};
    int qdev = 0;
    WINO_CUDA_TRY(cudaGetDevice(&qdev));
    if (qdev < 16 && !qattr[qdev]) {
      WINO_CUDA_TRY(cudaFuncSetAttribute(k_quant_input_tiled<2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
      WINO_CUDA_TRY(cudaFuncSetAttribute(k_quant_input_tiled<4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
      WINO_CUDA_TRY(cudaFuncSetAttribute(k_quant_input_tiled<6>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
      qattr[qdev] = true;
    }
    if (M.m == 2)
      k_quant_input_tiled<2><<<gq, kQT * kQC, qsm, st>>>(x, g, M, S, Cp, Tp, Uh, Ul, mode);
    else if (M.m == 4)
      k_quant_input_tiled<4><<<gq, kQT * kQC, qsm, st>>>(x, g, M, S, Cp, Tp, Uh, Ul, mode);
    else
      k_quant_input_tiled<6><<<gq, kQT * kQC, qsm, st>>>(x, g, M, S, Cp, Tp, Uh, Ul, mode);
    note_launches(4);
  }
  TcGemmArgs P;
  P.Uh = Uh;
  P.Ul = Ul;
  P.Vh = Vh;
  P.Vl = Vl;
  P.sV = sV;
  P.M = Mb;
  P.err = err;
  P.S = S;
  P.T = g.T;
  P.Tp = Tp;
  P.K = g.K;
  P.Cp = Cp;
  P.NB = NB;
  P.ncols = NB < 32 ? 32 : NB;
  P.mode = mode;
  const size_t smem = tc_smem_bytes(NB, split);
  static bool attr_set[16] = {false};
  int dev = 0;
  WINO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 16 && !attr_set[dev]) {
    WINO_CUDA_TRY(
        cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set[dev] = true;
  }
  {
    ProfScope ps(kKTcGemm, st);
    dim3 grid((unsigned)(Tp / kTcM), (unsigned)(g.K / NB), (unsigned)g.F);
    k_tc_gemm<<<grid, kTcThreads, smem, st>>>(P);
    note_launches(1);
  }
  {
    ProfScope ps(kKOutput, st);
    const int64_t n = (int64_t)g.K * g.T;
    const unsigned go = (unsigned)((n + 255) / 256);
    if (M.m == 2)
      k_output_transform_r3<2><<<go, 256, 0, st>>>(Mb, y, g, M);
    else if (M.m == 4)
      k_output_transform_r3<4><<<go, 256, 0, st>>>(Mb, y, g, M);
    else
      k_output_transform_r3<6><<<go, 256, 0, st>>>(Mb, y, g, M);
    note_launches(1);
  }
  WINO_CUDA_TRY(cudaGetLastError());
  return WINO_OK;
}

// Reads (and clears) the error flag of the last precision-form layer run in
// workspace `ws`: 1 when a bounded wait on the tensor cores gave up.
int tc_error_flag(void* ws, const LayerGeom& g, int dtype, cudaStream_t st, int* flag) {
  const TcLayout L = tc_layout(g, dtype);
  int* err = (int*)((char*)ws + L.err);
  WINO_CUDA_TRY(cudaMemcpyAsync(flag, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  WINO_CUDA_TRY(cudaStreamSynchronize(st));
  return WINO_OK;
}

}  // namespace wino
