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
//   WINO_SPLIT_BF16X6  a = hi + mid + lo with mid = RN_bf16(a - hi),
//                      lo = RN_bf16(a - hi - mid) (the differences are exact in
//                      FP32, so the three parts hold every bit of the FP32
//                      operand); U V ~ hh + hm + mh + hl + lh + mm (six MMAs;
//                      the dropped terms are below 2^-23 of hh).  hh goes to
//                      one TMEM accumulator and the five small products to a
//                      second (their rounding is 2^-7 smaller), added in the
//                      epilogue: the error falls below the FP32 SIMT layer's
// The operand parts are stored in order (hi, then lo or mid, then lo), one
// [F][rows][Cp] 16-bit array each.
// Per-frequency scaling (exact powers of two, undone before the output
// transform): U[f] by the power of two that brings |BT_i|_1 |BT_j|_1 into
// [1, 2), V[f] by the one that brings max |V[f]| into [1, 2).  This keeps FP16
// operands in range; for BF16 it only guards the subnormal range of lo.
//
// Pipeline: filter transform (FP32) -> per-frequency max |V| -> V rounded
// into the blocked image of [F][K][Cp] (K-major B operand); input transform
// (FP32) rounded into the blocked image of [F][Tp][Cp] (K-major A operand);
// k_tc_gemm; the general output transform.
// k_tc_gemm: one CTA = one frequency x 128 tiles (MMA M) x NB output
// channels (MMA N <= 256), contraction over Cp in chunks of 64 channels
// (one 128-byte swizzle row per operand row).  The quantising kernels write
// the operands as the SWIZZLE_128B K-major shared-memory images of these
// chunks, so one thread moves each chunk with one bulk copy per operand
// part (mbarrier-counted), issues tcgen05.mma (K = 16 per instruction) and
// commits to a second mbarrier; every wait is bounded and records an error
// instead of hanging.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "../../include/wino.h"
#include "async_copy.cuh"
#include "common.cuh"

namespace wino {

constexpr int kTcM = 128;    // tiles per CTA (MMA M)
constexpr int kTcKc = 64;    // channels per chunk: one 128-byte row per operand row

// Operand parts in HBM are the shared-memory images the contraction copies
// whole (one bulk copy per operand part and chunk): U per (frequency,
// 128-tile block, 64-channel chunk) one 16 KB block, V per (frequency,
// NB-channel k block, chunk) one NB x 128-byte block.  Row r of a block (a
// tile, an output channel) is 128 bytes at r x 128, its 16-byte piece j (8
// channels) at position j ^ (r & 7): the 128-byte swizzle the MMA's K-major
// operand descriptors name.  Element index of (f, tile t, channel c) in a U
// part, and of (f, output channel k, c) in a V part:
__host__ __device__ __forceinline__ int64_t tc_u_index(int f, int64_t t, int c, int64_t ntb,
                                                       int nch) {
  const int64_t blk = ((int64_t)f * ntb + t / kTcM) * nch + c / kTcKc;
  const int r = (int)(t % kTcM), j = (c % kTcKc) / 8;
  return blk * (kTcM * kTcKc) + r * kTcKc + ((j ^ (r & 7)) * 8) + (c % 8);
}
__host__ __device__ __forceinline__ int64_t tc_v_index(int f, int k, int c, int NB, int nkb,
                                                       int nch) {
  const int64_t blk = ((int64_t)f * nkb + k / NB) * nch + c / kTcKc;
  const int r = k % NB, j = (c % kTcKc) / 8;
  return blk * ((int64_t)NB * kTcKc) + r * kTcKc + ((j ^ (r & 7)) * 8) + (c % 8);
}


__global__ void k_output_transform(const float* __restrict__ Mi, float* __restrict__ y,
                                   const LayerGeom g, const LayerMats M);

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// 16-bit rounding of a scaled FP32 value; mode 2 FP16, every other mode BF16.
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

// Number of 16-bit parts an operand is split into.
__host__ __device__ __forceinline__ int tc_parts(int mode) {
  return mode == 3 ? 2 : (mode == 4 ? 3 : 1);
}

// The parts of a (scaled) FP32 value, hi first.
__device__ __forceinline__ void split_parts(float v, int mode, uint16_t out[3]) {
  out[0] = round16(v, mode);
  if (mode == 3) {
    out[1] = round16(v - widen16(out[0], mode), mode);
  } else if (mode == 4) {
    const float r1 = v - widen16(out[0], mode);  // exact
    out[1] = round16(r1, mode);
    out[2] = round16(r1 - widen16(out[1], mode), mode);  // exact difference
  }
}

}  // namespace

struct TcScales {
  float sU[kMaxAlpha * kMaxAlpha];
};

// ---------------------------------------------------------------------------
// Operand preparation.
// ---------------------------------------------------------------------------
// max |V[f]| over every (c, k): a grid-stride loop over kernels (channels
// fastest, so neighbouring threads read neighbouring weights), per-thread
// maxima, then per block one warp-shuffle and shared-memory reduction and
// ONE atomicMax per frequency on the bit pattern (non-negative floats order
// like their bits).
constexpr int kFvThreads = 256;
template <int MM>
__global__ void __launch_bounds__(kFvThreads) k_filter_vmax(const float* __restrict__ w, int C,
                                                           int K, const LayerMats M,
                                                           unsigned* __restrict__ vmax_bits) {
  constexpr int F = (MM + 2) * (MM + 2);
  float mx[F];
#pragma unroll
  for (int f = 0; f < F; ++f) mx[f] = 0.0f;
  const int64_t n = (int64_t)C * K;
  for (int64_t idx = (int64_t)blockIdx.x * kFvThreads + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * kFvThreads) {
    const int c = (int)(idx % C), k = (int)(idx / C);
    float v[F];
    filter_fixed<MM>(w + ((int64_t)k * C + c) * 9, M, v);
#pragma unroll
    for (int f = 0; f < F; ++f) mx[f] = fmaxf(mx[f], fabsf(v[f]));
  }
  __shared__ float wm[kFvThreads / 32][F];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int f = 0; f < F; ++f) {
    float m = mx[f];
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) wm[warp][f] = m;
  }
  __syncthreads();
  if (threadIdx.x < F) {
    float m = wm[0][threadIdx.x];
    for (int q = 1; q < kFvThreads / 32; ++q) m = fmaxf(m, wm[q][threadIdx.x]);
    atomicMax(vmax_bits + threadIdx.x, __float_as_uint(m));
  }
}

// Filter transform recomputed, scaled by sV[f] = 2^(1 - e) for max |V[f]| =
// m 2^e, m in [0.5, 1), and split into the operand parts V0/V1/V2 (the
// blocked image of tc_v_index for k blocks of NB; channels c >= C zero).
// One thread per (k, c), channels fastest (each 64-channel row is one
// 128-byte line, its pieces permuted).  Block 0 also records sV for the
// epilogue.
template <int MM>
__global__ void __launch_bounds__(256) k_filter_quant(const float* __restrict__ w, int C, int K,
                                                      int Cp, const LayerMats M,
                                                      const unsigned* __restrict__ vmax_bits,
                                                      float* __restrict__ sV,
                                                      uint16_t* __restrict__ V0,
                                                      uint16_t* __restrict__ V1,
                                                      uint16_t* __restrict__ V2, int mode,
                                                      int NB) {
  constexpr int F = (MM + 2) * (MM + 2);
  __shared__ float ss[F];
  if (threadIdx.x < F) {
    ss[threadIdx.x] = pow2_normaliser(__uint_as_float(vmax_bits[threadIdx.x]));
    if (blockIdx.x == 0) sV[threadIdx.x] = ss[threadIdx.x];
  }
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)K * Cp) return;
  const int c = (int)(idx % Cp), k = (int)(idx / Cp);
  float v[F];
  if (c < C) {
    filter_fixed<MM>(w + ((int64_t)k * C + c) * 9, M, v);
  } else {
#pragma unroll
    for (int f = 0; f < F; ++f) v[f] = 0.0f;
  }
  const int parts = tc_parts(mode);
#pragma unroll
  for (int f = 0; f < F; ++f) {
    uint16_t q[3];
    split_parts(v[f] * ss[f], mode, q);
    const int64_t o = tc_v_index(f, k, c, NB, K / NB, Cp / kTcKc);
    V0[o] = q[0];
    if (parts > 1) V1[o] = q[1];
    if (parts > 2) V2[o] = q[2];
  }
}

// Input transform (FP32, the FP32 layer's order) -> operand parts
// U0/U1/U2 [f][t][c], scaled; rows t >= T and columns c >= C are zero.
// One block = kQT = 4 tiles x 64 channels; a thread transforms two adjacent
// channels of one tile (tiles fastest: neighbouring patches share input
// rows).  The 16-bit results are staged in shared memory as 32-bit channel
// pairs -- rows of kQRow = 32 pairs, pair p of tile tl's row at word
// p ^ 8 tl, so the 32 stores of a warp (4 tiles x 8 pairs) hit 32 distinct
// banks with no padding -- and leave as whole 128-byte rows of 64 channels
// (one cache line per (f, tile) and part).  (Rows padded to 40 words
// instead held one F(6x6) split-BF16x6 block per SM, not two.)
// (Splitting the transform's rows over 2-4 blocks, for staging within 36 KB
// and five blocks per SM, measured 8-15% slower per stack: every block
// loads the whole patch, and the patch loads are what this kernel waits on.
// Issuing both channels' patch loads before either transform measured the
// same for the split forms and 3% slower for BF16: 122 registers instead
// of 80.)
constexpr int kQT = 4, kQC = 64, kQP = kQC / 2, kQRow = kQP;
// staging word of channel pair p in tile tl's row (bank-conflict swizzle)
__device__ __forceinline__ int qswz(int p, int tl) { return p ^ (tl << 3); }
constexpr int kQuantThreads = kQT * kQP;
// largest staging: three parts of F = 64 frequencies (m = 6)
constexpr int kQuantSmemMax = 3 * 64 * kQT * kQRow * 4;

// B^T d B of the tile patch of channel c (zeros when the tile or the channel
// is out of range), rows i in [I0, I1) of the result only: frequency f =
// i alpha + j at out(f, v).  Each value is computed exactly as by the whole
// transform (the row restriction only skips rows).
template <int MM, int I0, int I1, class Out>
__device__ __forceinline__ void quant_patch(const float* __restrict__ x, const LayerGeom& g,
                                            const LayerMats& Mx, int64_t t, int c, Out out) {
  constexpr int A = MM + 2;
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
  float tm[I1 - I0][A];
#pragma unroll
  for (int i = I0; i < I1; ++i)
#pragma unroll
    for (int l = 0; l < A; ++l) {
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < A; ++q) acc = fmaf(Mx.BT[i * A + q], d[q][l], acc);
      tm[i - I0][l] = acc;
    }
#pragma unroll
  for (int i = I0; i < I1; ++i)
#pragma unroll
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
#pragma unroll
      for (int l = 0; l < A; ++l) acc = fmaf(tm[i - I0][l], Mx.BT[j * A + l], acc);
      out(i * A + j, live ? acc : 0.0f);
    }
}

// Rows [I0, I1) of two adjacent channels' transforms, scaled, split and
// staged as 32-bit channel pairs (channel c in the low half).
template <int MM, int I0, int I1>
__device__ __forceinline__ void quant_pair_rows(const float* __restrict__ x, const LayerGeom& g,
                                                const LayerMats& Mx, const TcScales& S,
                                                int64_t t, int c, int tl, int cp, int mode,
                                                int parts, uint32_t* qs, int kPart) {
  constexpr int A = MM + 2, NR = (I1 - I0) * A;
  float ua[NR];
  quant_patch<MM, I0, I1>(x, g, Mx, t, c, [&](int f, float v) { ua[f - I0 * A] = v; });
  quant_patch<MM, I0, I1>(x, g, Mx, t, c + 1, [&](int f, float v) {
    uint16_t qa[3], qb[3];
    split_parts(ua[f - I0 * A] * S.sU[f], mode, qa);
    split_parts(v * S.sU[f], mode, qb);
    const int o = (f * kQT + tl) * kQRow + qswz(cp, tl);
    qs[o] = (uint32_t)qa[0] | ((uint32_t)qb[0] << 16);
    if (parts > 1) qs[kPart + o] = (uint32_t)qa[1] | ((uint32_t)qb[1] << 16);
    if (parts > 2) qs[2 * kPart + o] = (uint32_t)qa[2] | ((uint32_t)qb[2] << 16);
  });
}

template <int MM>
__global__ void __launch_bounds__(kQuantThreads) k_quant_input_tiled(
    const float* __restrict__ x, const LayerGeom g, const LayerMats Mx, const TcScales S, int Cp,
    int64_t Tp, uint16_t* __restrict__ U0, uint16_t* __restrict__ U1, uint16_t* __restrict__ U2,
    int mode) {
  constexpr int A = MM + 2, F = A * A;
  extern __shared__ __align__(16) uint32_t qs[];  // [parts][F][kQT][kQRow] channel pairs
  constexpr int kPart = F * kQT * kQRow;          // one part's staging, in words
  const int tl = threadIdx.x % kQT, cp = threadIdx.x / kQT;
  const int64_t t = (int64_t)blockIdx.x * kQT + tl;
  const int c = blockIdx.y * kQC + 2 * cp;
  const int parts = tc_parts(mode);
  if constexpr (A <= 6) {
    // both channels' values of a frequency meet in registers: one 32-bit
    // store per (f, part)
    quant_pair_rows<MM, 0, A>(x, g, Mx, S, t, c, tl, cp, mode, parts, qs, kPart);
  } else {
    // alpha = 8: holding one channel's 64 values while transforming the
    // other costs too many registers (and transforming in row halves costs
    // a second pass over the patches), so each channel goes straight to its
    // 16-bit half of the same words
    uint16_t* qh = reinterpret_cast<uint16_t*>(qs);
    for (int h = 0; h < 2; ++h)
      quant_patch<MM, 0, A>(x, g, Mx, t, c + h, [&](int f, float v) {
        uint16_t q[3];
        split_parts(v * S.sU[f], mode, q);
        const int o = 2 * ((f * kQT + tl) * kQRow + qswz(cp, tl)) + h;
        qh[o] = q[0];
        if (parts > 1) qh[2 * kPart + o] = q[1];
        if (parts > 2) qh[4 * kPart + o] = q[2];
      });
  }
  __syncthreads();
  // rows (f, tile) of 64 channels = 8 x 16-byte stores, consecutive threads
  // on consecutive segments of a row (one 128-byte line of the blocked image)
  const int64_t tb = (int64_t)blockIdx.x * kQT;
  const int c0 = blockIdx.y * kQC;
  uint16_t* const dsts[3] = {U0, U1, U2};
  for (int e = threadIdx.x; e < F * kQT * 8; e += kQuantThreads) {
    const int seg = e % 8, row = e / 8;  // row = f * kQT + tile
    const int f = row / kQT, tr = row % kQT;
    const int64_t dst = tc_u_index(f, tb + tr, c0 + seg * 8, Tp / kTcM, Cp / kTcKc);
    for (int pp = 0; pp < parts; ++pp)
      *reinterpret_cast<uint4*>(dsts[pp] + dst) =
          *reinterpret_cast<const uint4*>(qs + pp * kPart + row * kQRow + qswz(seg * 4, tr));
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
  const int cols = min(MM, g.Wo - tj * MM);
#pragma unroll
  for (int a = 0; a < MM; ++a) {
    const int p = ti * MM + a;
    float yr[MM];
#pragma unroll
    for (int b = 0; b < MM; ++b) {
      float acc = 0.0f;
#pragma unroll
      for (int j = 0; j < A; ++j) acc = fmaf(Z[a][j], Mx.AT[b * A + j], acc);
      yr[b] = acc;
    }
    if (p >= g.Ho) continue;
    float* yrow = yk + (int64_t)p * g.Wo + tj * MM;
    // whole rows as vector stores when aligned (adjacent lanes hold adjacent
    // tiles, so a warp writes one contiguous run)
    if (MM % 4 == 0 && cols == MM && (((uintptr_t)yrow) & 15) == 0) {
#pragma unroll
      for (int b = 0; b < MM; b += 4)
        *reinterpret_cast<float4*>(yrow + b) = make_float4(yr[b], yr[b + 1], yr[b + 2], yr[b + 3]);
    } else if (MM % 2 == 0 && cols == MM && (((uintptr_t)yrow) & 7) == 0) {
#pragma unroll
      for (int b = 0; b < MM; b += 2)
        *reinterpret_cast<float2*>(yrow + b) = make_float2(yr[b], yr[b + 1]);
    } else {
#pragma unroll
      for (int b = 0; b < MM; ++b)
        if (b < cols) yrow[b] = yr[b];
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

// 32 lanes x 16 consecutive FP32 columns of TMEM, one row per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}


}  // namespace

constexpr int kTcThreads = 128;

struct TcGemmArgs {
  const uint16_t* U[3];  // operand parts (hi first), blocked images (tc_u_index)
  const uint16_t* V[3];  // blocked images (tc_v_index, k blocks of NB)
  const float* sV;
  float* M;  // [F][K][T]
  int* err;  // the device's wait-error flag: set to 1 when a bounded wait gives up
  TcScales S;
  int64_t T, Tp;
  int K, Cp, NB, ncols, mode;
};

// Dynamic shared memory: per operand part a 1024-byte-aligned tile: A parts
// 128 x 64, then B parts NB x 64 16-bit values, then the two mbarriers and
// the TMEM address.  Products per 16-channel step, as (A part, B part):
//   1 part  (BF16, FP16): (0,0)
//   2 parts (split x3):   (0,0) (0,1) (1,0)
//   3 parts (split x6):   (0,0) into accumulator D, then (0,1) (1,0) (0,2)
//                         (2,0) (1,1) into a second accumulator D' (TMEM
//                         columns NB..2NB-1); the epilogue adds D + D'
// One stage: two CTAs per SM already overlap one's loads with the other's
// MMAs and epilogue.  With the per-thread copies this kernel used before the
// bulk copies, a two-stage ring at two CTAs per SM (one-part forms, NB =
// 256) measured the same within 2% on the VGG-16 stages and a two-to-four-
// stage ring at one CTA per SM 15-35% slower; with the bulk copies a
// two-stage ring of the one-part forms measured 1.5% faster (within run-to-
// run spread), so the single stage stays.
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_gemm(const TcGemmArgs P) {
  extern __shared__ __align__(1024) unsigned char tsm_raw[];
  // the swizzled tiles must start on 1024-byte boundaries (the host asks for
  // 1 KiB of slack)
  unsigned char* tsm = tsm_raw + ((1024u - (smem_addr(tsm_raw) & 1023u)) & 1023u);
  const int f = blockIdx.z;
  const int64_t t0 = (int64_t)blockIdx.x * kTcM;
  const int n0 = blockIdx.y * P.NB;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int parts = tc_parts(P.mode);
  const uint32_t a_bytes = kTcM * 128, b_bytes = P.NB * 128;
  unsigned char* As = tsm;                        // part p at As + p * a_bytes
  unsigned char* Bs = As + parts * a_bytes;       // part p at Bs + p * b_bytes
  unsigned char* tail = Bs + parts * b_bytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tail);  // [0] copies landed, [1] MMAs done
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tail + 16);
  const uint32_t bar_ld = smem_addr(bar), bar_mma = smem_addr(bar + 1);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_addr(tmem_holder)),
                 "r"(P.ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  if (tid == 0) {
    mbar_init1(bar_ld);
    mbar_init1(bar_mma);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_holder;

  const int fmt = (P.mode == 2) ? 0 : 1;
  const uint32_t idesc = f16_idesc(fmt, kTcM, P.NB);
  const int nchunks = P.Cp / kTcKc;
  // this CTA's operand blocks (blocked images, see tc_u_index / tc_v_index):
  // chunk ch of A part p at U[p] + a0 + ch * 8192, of B part p at V[p] + b0
  // + ch * NB * 64 (16-bit elements)
  const int64_t a0 = ((int64_t)f * gridDim.x + blockIdx.x) * nchunks * (kTcM * kTcKc);
  const int64_t b0 = ((int64_t)f * gridDim.y + blockIdx.y) * nchunks * ((int64_t)P.NB * kTcKc);
  // Thread 0 runs the chunk loop: two bulk copies per operand part into the
  // stage, then the MMAs, committed to bar_mma; the stage is refilled once
  // they completed.  The other threads wait at the barrier below.
  bool ok = true;
  if (tid == 0) {
    for (int ch = 0; ch < nchunks; ++ch) {
      if (ch > 0 && !mbar_wait_bounded(bar_mma, (uint32_t)((ch - 1) & 1))) {
        ok = false;
        break;
      }
      mbar_expect_tx(bar_ld, (uint32_t)parts * (a_bytes + b_bytes));
      for (int pp = 0; pp < parts; ++pp) {
        bulk_g2s(smem_addr(As + pp * a_bytes), P.U[pp] + a0 + (int64_t)ch * (kTcM * kTcKc), a_bytes,
                 bar_ld);
        bulk_g2s(smem_addr(Bs + pp * b_bytes), P.V[pp] + b0 + (int64_t)ch * P.NB * kTcKc, b_bytes,
                 bar_ld);
      }
      if (!mbar_wait_bounded(bar_ld, (uint32_t)(ch & 1))) {
        ok = false;
        // the copies may still land: wait for them (bounded) before the
        // stage is given up
        (void)mbar_wait_bounded(bar_ld, (uint32_t)(ch & 1));
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kTcKc / 16; ++kk) {
        const uint32_t acc = (ch > 0 || kk > 0) ? 1u : 0u;
        uint64_t ad[3], bd[3];
        for (int pp = 0; pp < parts; ++pp) {
          ad[pp] = sw128_desc(smem_addr(As + pp * a_bytes) + kk * 32);
          bd[pp] = sw128_desc(smem_addr(Bs + pp * b_bytes) + kk * 32);
        }
        mma_f16(tmem, ad[0], bd[0], idesc, acc);
        if (parts == 2) {
          mma_f16(tmem, ad[0], bd[1], idesc, 1u);
          mma_f16(tmem, ad[1], bd[0], idesc, 1u);
        } else if (parts == 3) {
          const uint32_t tlo = tmem + (uint32_t)P.NB;  // second accumulator
          mma_f16(tlo, ad[0], bd[1], idesc, acc);
          mma_f16(tlo, ad[1], bd[0], idesc, 1u);
          mma_f16(tlo, ad[0], bd[2], idesc, 1u);
          mma_f16(tlo, ad[2], bd[0], idesc, 1u);
          mma_f16(tlo, ad[1], bd[1], idesc, 1u);
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              bar_mma)
          : "memory");
    }
    // the last chunk's MMAs (and so every earlier one) completed
    if (ok && !mbar_wait_bounded(bar_mma, (uint32_t)((nchunks - 1) & 1))) ok = false;
    if (!ok) atomicExch(P.err, 1);
  }
  ok = __syncthreads_and(tid == 0 ? (ok ? 1 : 0) : 1) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  if (ok) {
    // epilogue: warp w reads TMEM lanes 32w..32w+31 (tiles), 16 columns per load
    const float inv = 1.0f / (P.S.sU[f] * P.sV[f]);  // exact: powers of two
    const int64_t t = t0 + warp * 32 + lane;
    for (int col = 0; col < P.NB; col += 16) {
      uint32_t v[16], w[16];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)col;
      tmem_ld16(ta, v);
      if (parts == 3) {
        tmem_ld16(ta + (uint32_t)P.NB, w);
#pragma unroll
        for (int j = 0; j < 16; ++j)
          v[j] = __float_as_uint(__fadd_rn(__uint_as_float(v[j]), __uint_as_float(w[j])));
      }
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

// TMEM columns of one CTA: NB FP32 accumulator columns (two accumulators for
// the split x6 form), at least 32.
static int tc_ncols(int NB, int parts) {
  const int c = parts == 3 ? 2 * NB : NB;
  return c < 32 ? 32 : c;
}

// Dynamic shared memory of one CTA: its stage, raised so that the CTAs an
// SM holds at once fit TMEM's 512 columns together -- at most 512 / ncols
// of them, given the SM's shared memory (smem_sm) and the part reserved per
// CTA (reserved).
static size_t tc_smem_bytes(int NB, int parts, size_t smem_sm, size_t reserved) {
  const size_t a = (size_t)kTcM * 128, b = (size_t)NB * 128;
  const size_t s = (a + b) * parts + 64 + 1024;
  const int fit = 512 / tc_ncols(NB, parts);
  const size_t floor_b = smem_sm / (fit + 1) + 1 - reserved;
  return s < floor_b ? floor_b : s;
}

// Workspace layout of the precision form (bytes), all 1024-aligned.
struct TcLayout {
  size_t vmax, sV, V[3], U[3], M, total;
};

static TcLayout tc_layout(const LayerGeom& g, int dtype) {
  auto al = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
  const int64_t Tp = (g.T + kTcM - 1) / kTcM * kTcM;
  const int Cp = (g.C + kTcKc - 1) / kTcKc * kTcKc;
  const int parts = tc_parts(dtype);
  TcLayout L;
  size_t o = 0;
  L.vmax = o;
  o = al(o + (size_t)g.F * 4);
  L.sV = o;
  o = al(o + (size_t)g.F * 4);
  for (int pp = 0; pp < 3; ++pp) {
    L.V[pp] = o;
    o = al(o + (pp < parts ? (size_t)g.F * g.K * Cp * 2 : 0));
  }
  for (int pp = 0; pp < 3; ++pp) {
    L.U[pp] = o;
    o = al(o + (pp < parts ? (size_t)g.F * Tp * Cp * 2 : 0));
  }
  L.M = o;
  o = al(o + (size_t)g.F * g.K * g.T * 4);
  L.total = o;
  return L;
}

size_t tc_workspace_bytes(const LayerGeom& g, int dtype) { return tc_layout(g, dtype).total; }

// Output channels per CTA (MMA N): the largest of 256..16 dividing K; at most
// 128 for the three-part form, whose 256-wide tiles would need 148 KB of
// shared memory and so leave one CTA per SM, with nothing to overlap its
// single-stage load / MMA loop.
static int tc_nb(int K, int parts) {
  const int cands[5] = {256, 128, 64, 32, 16};
  for (int nb : cands)
    if (K % nb == 0 && !(parts == 3 && nb > 128)) return nb;
  return 0;
}

int layer_forward_tc(const float* x, const float* w, float* y, const LayerGeom& g,
                     const LayerMats& M, int dtype, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (g.dim != 2 || M.r != 3 || (M.m != 2 && M.m != 4 && M.m != 6)) {
    set_error("tensor-core forms support 2D F(m x m, 3 x 3), m in {2, 4, 6}");
    return WINO_EUNSUPPORTED;
  }
  const int NB = tc_nb(g.K, tc_parts(dtype));
  if (NB == 0) {
    set_error("tensor-core forms need K a multiple of 16");
    return WINO_EUNSUPPORTED;
  }
  const TcLayout L = tc_layout(g, dtype);
  if (ws_bytes < L.total) {
    set_error("workspace too small for the tensor-core form");
    return WINO_ENOMEM;
  }
  const int mode = dtype;  // 1 bf16, 2 fp16, 3 split bf16 x3, 4 split bf16 x6
  const int parts = tc_parts(mode);
  char* b = (char*)ws;
  unsigned* vmax = (unsigned*)(b + L.vmax);
  float* sV = (float*)(b + L.sV);
  int* err = nullptr;
  {
    int rc = wait_error_flag(&err);
    if (rc != WINO_OK) return rc;
  }
  uint16_t *Vp[3], *Up[3];
  for (int pp = 0; pp < 3; ++pp) {
    Vp[pp] = (uint16_t*)(b + L.V[pp]);
    Up[pp] = (uint16_t*)(b + L.U[pp]);
  }
  float* Mb = (float*)(b + L.M);
  const int64_t Tp = (g.T + kTcM - 1) / kTcM * kTcM;
  const int Cp = (g.C + kTcKc - 1) / kTcKc * kTcKc;

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
  {
    ProfScope ps(kKTcTransform, st);
    // per-frequency maxima of V (each block reduces up to 8 kernels per
    // thread), then V recomputed, scaled and split
    const int64_t nck = (int64_t)g.C * g.K;
    const unsigned bf = (unsigned)std::max<int64_t>(1, std::min<int64_t>(
                                                           (nck + 8 * kFvThreads - 1) /
                                                           (8 * kFvThreads), 1 << 16));
    const unsigned bq = (unsigned)(((int64_t)g.K * Cp + 255) / 256);
    if (M.m == 2) {
      k_filter_vmax<2><<<bf, kFvThreads, 0, st>>>(w, g.C, g.K, M, vmax);
      k_filter_quant<2><<<bq, 256, 0, st>>>(w, g.C, g.K, Cp, M, vmax, sV, Vp[0], Vp[1], Vp[2], mode,
                                            NB);
    } else if (M.m == 4) {
      k_filter_vmax<4><<<bf, kFvThreads, 0, st>>>(w, g.C, g.K, M, vmax);
      k_filter_quant<4><<<bq, 256, 0, st>>>(w, g.C, g.K, Cp, M, vmax, sV, Vp[0], Vp[1], Vp[2], mode,
                                            NB);
    } else {
      k_filter_vmax<6><<<bf, kFvThreads, 0, st>>>(w, g.C, g.K, M, vmax);
      k_filter_quant<6><<<bq, 256, 0, st>>>(w, g.C, g.K, Cp, M, vmax, sV, Vp[0], Vp[1], Vp[2], mode,
                                            NB);
    }
    const dim3 gq((unsigned)(Tp / kQT), (unsigned)(Cp / kQC));
    size_t qsm = (size_t)parts * g.F * kQT * kQRow * sizeof(uint32_t);
    // the patch loads reuse overlapping input rows through L1, which shares
    // the SM's storage with these blocks' staging: the two-part F(4x4) form
    // (37 KB) runs best at four blocks per SM (six measured 4% slower)
    if (parts == 2 && M.m == 4 && qsm < 46 * 1024) qsm = 46 * 1024;
    static bool qattr[16] = {false};
    int qdev = 0;
    WINO_CUDA_TRY(cudaGetDevice(&qdev));
    if (qdev < 16 && !qattr[qdev]) {
      WINO_CUDA_TRY(cudaFuncSetAttribute(k_quant_input_tiled<2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kQuantSmemMax));
      WINO_CUDA_TRY(cudaFuncSetAttribute(k_quant_input_tiled<4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kQuantSmemMax));
      WINO_CUDA_TRY(cudaFuncSetAttribute(k_quant_input_tiled<6>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kQuantSmemMax));
      qattr[qdev] = true;
    }
    if (M.m == 2)
      k_quant_input_tiled<2><<<gq, kQuantThreads, qsm, st>>>(x, g, M, S, Cp, Tp, Up[0], Up[1], Up[2],
                                                         mode);
    else if (M.m == 4)
      k_quant_input_tiled<4><<<gq, kQuantThreads, qsm, st>>>(x, g, M, S, Cp, Tp, Up[0], Up[1], Up[2],
                                                         mode);
    else
      k_quant_input_tiled<6><<<gq, kQuantThreads, qsm, st>>>(x, g, M, S, Cp, Tp, Up[0], Up[1], Up[2],
                                                         mode);
    note_launches(3);
  }
  TcGemmArgs P;
  for (int pp = 0; pp < 3; ++pp) {
    P.U[pp] = Up[pp];
    P.V[pp] = Vp[pp];
  }
  P.sV = sV;
  P.M = Mb;
  P.err = err;
  P.S = S;
  P.T = g.T;
  P.Tp = Tp;
  P.K = g.K;
  P.Cp = Cp;
  P.NB = NB;
  P.ncols = tc_ncols(NB, parts);
  P.mode = mode;
  static size_t smem_sm[16] = {0}, reserved[16] = {0};
  int sdev = 0;
  WINO_CUDA_TRY(cudaGetDevice(&sdev));
  if (sdev >= 16) return WINO_EUNSUPPORTED;
  if (smem_sm[sdev] == 0) {
    int v = 0, r = 0;
    WINO_CUDA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, sdev));
    WINO_CUDA_TRY(cudaDeviceGetAttribute(&r, cudaDevAttrReservedSharedMemoryPerBlock, sdev));
    reserved[sdev] = (size_t)r;
    smem_sm[sdev] = (size_t)v;
  }
  const size_t smem = tc_smem_bytes(NB, parts, smem_sm[sdev], reserved[sdev]);
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

}  // namespace wino
