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

// V32[f][c][k] -> parts V0/V1/V2 [f][k][c] (c padded to Cp with zeros), scaled.
__global__ void k_quant_v(const float* __restrict__ V, int C, int K, int Cp, int F,
                          const unsigned* __restrict__ vmax_bits, float* __restrict__ sV,
                          uint16_t* __restrict__ V0, uint16_t* __restrict__ V1,
                          uint16_t* __restrict__ V2, int mode) {
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
  uint16_t q[3];
  split_parts(v, mode, q);
  V0[idx] = q[0];
  if (mode == 3 || mode == 4) V1[idx] = q[1];
  if (mode == 4) V2[idx] = q[2];
}

// Input transform (FP32, the FP32 layer's order) -> operand parts
// U0/U1/U2 [f][t][c], scaled; rows t >= T and columns c >= C are zero.
// One block = 16 tiles x 16 channels; a thread transforms one (tile,
// channel) with tiles fastest (neighbouring patches share input rows), the
// 16-bit results meet in shared memory and leave as 32-byte rows of 16
// channels.
constexpr int kQT = 16, kQC = 16;
// largest staging: three parts of F = 64 frequencies (m = 6)
constexpr int kQuantSmemMax = 3 * 64 * kQT * kQC * 2;
template <int MM>
__global__ void __launch_bounds__(kQT* kQC) k_quant_input_tiled(
    const float* __restrict__ x, const LayerGeom g, const LayerMats Mx, const TcScales S, int Cp,
    int64_t Tp, uint16_t* __restrict__ U0, uint16_t* __restrict__ U1, uint16_t* __restrict__ U2,
    int mode) {
  constexpr int A = MM + 2, F = A * A;
  extern __shared__ __align__(16) uint16_t qs[];  // [parts][F][kQT][kQC]
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
  const int parts = tc_parts(mode);
  constexpr int kPart = F * kQT * kQC;  // one part's staging, in 16-bit values
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
#pragma unroll
      for (int l = 0; l < A; ++l) acc = fmaf(tm[i][l], Mx.BT[j * A + l], acc);
      const int f = i * A + j;
      const float v = live ? acc * S.sU[f] : 0.0f;
      uint16_t q[3];
      split_parts(v, mode, q);
      const int o = (f * kQT + tl) * kQC + cl;
      qs[o] = q[0];
      if (parts > 1) qs[kPart + o] = q[1];
      if (parts > 2) qs[2 * kPart + o] = q[2];
    }
  __syncthreads();
  // rows (f, tile) of 16 channels = 32 bytes = two 16-byte stores per part
  const int64_t plane = Tp * Cp;
  const int64_t tb = (int64_t)blockIdx.x * kQT;
  const int c0 = blockIdx.y * kQC;
  uint16_t* const dsts[3] = {U0, U1, U2};
  for (int e = threadIdx.x; e < F * kQT * 2; e += kQT * kQC) {
    const int half = e & 1, row = e >> 1;  // row = f * kQT + tl
    const int f = row / kQT, tr = row % kQT;
    const int64_t dst = f * plane + (tb + tr) * Cp + c0 + half * 8;
    for (int pp = 0; pp < parts; ++pp)
      *reinterpret_cast<uint4*>(dsts[pp] + dst) =
          *reinterpret_cast<const uint4*>(qs + pp * kPart + row * kQC + half * 8);
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

__device__ __forceinline__ void cp_async16_tc(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}

}  // namespace

constexpr int kTcM = 128;    // tiles per CTA (MMA M)
constexpr int kTcKc = 64;    // channels per chunk: one 128-byte row per operand row
constexpr int kTcThreads = 128;

struct TcGemmArgs {
  const uint16_t* U[3];  // operand parts (hi first), [F][Tp][Cp]
  const uint16_t* V[3];  // [F][K][Cp]
  const float* sV;
  float* M;  // [F][K][T]
  int* err;  // the device's wait-error flag: set to 1 when a bounded wait gives up
  TcScales S;
  int64_t T, Tp;
  int K, Cp, NB, ncols, mode;
};

// Dynamic shared memory: per operand part a 1024-byte-aligned tile: A parts
// 128 x 64, then B parts NB x 64 16-bit values, then the mbarrier and the
// TMEM address.  Products per 16-channel step, as (A part, B part):
//   1 part  (BF16, FP16): (0,0)
//   2 parts (split x3):   (0,0) (0,1) (1,0)
//   3 parts (split x6):   (0,0) into accumulator D, then (0,1) (1,0) (0,2)
//                         (2,0) (1,1) into a second accumulator D' (TMEM
//                         columns NB..2NB-1); the epilogue adds D + D'
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
      for (int pp = 0; pp < parts; ++pp)
        cp_async16_tc(smem_addr(As + pp * a_bytes + off), P.U[pp] + g);
    }
    for (int e = tid; e < P.NB * 8; e += kTcThreads) {
      const int r = e >> 3, j = e & 7;
      const uint32_t off = r * 128 + ((j ^ (r & 7)) << 4);
      const int64_t g = f * bplane + (int64_t)(n0 + r) * P.Cp + c0 + j * 8;
      for (int pp = 0; pp < parts; ++pp)
        cp_async16_tc(smem_addr(Bs + pp * b_bytes + off), P.V[pp] + g);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
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

static size_t tc_smem_bytes(int NB, int parts) {
  const size_t a = (size_t)kTcM * 128, b = (size_t)NB * 128;
  size_t s = (a + b) * parts + 64 + 1024;
  // a CTA holding more than half of TMEM (512 columns) must be alone on its
  // SM: ask for more than half of the shared memory
  if (tc_ncols(NB, parts) > 256 && s < 120 * 1024) s = 120 * 1024;
  // at most two CTAs per SM, so their TMEM columns (NB <= 256 each) fit
  return s < 80 * 1024 ? 80 * 1024 : s;
}

// Workspace layout of the precision form (bytes), all 1024-aligned.
struct TcLayout {
  size_t V32, vmax, sV, V[3], U[3], M, total;
};

static TcLayout tc_layout(const LayerGeom& g, int dtype) {
  auto al = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
  const int64_t Tp = (g.T + kTcM - 1) / kTcM * kTcM;
  const int Cp = (g.C + kTcKc - 1) / kTcKc * kTcKc;
  const int parts = tc_parts(dtype);
  TcLayout L;
  size_t o = 0;
  L.V32 = o;
  o = al(o + (size_t)g.F * g.C * g.K * 4);
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
  const int mode = dtype;  // 1 bf16, 2 fp16, 3 split bf16 x3, 4 split bf16 x6
  const int parts = tc_parts(mode);
  char* b = (char*)ws;
  float* V32 = (float*)(b + L.V32);
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
    const int64_t n = (int64_t)g.C * g.K;
    k_filter_transform<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, V32, g.dim, g.C, g.K, M);
    const int64_t plane = (int64_t)g.C * g.K;
    const unsigned bx = (unsigned)std::min<int64_t>(256, (plane + 8 * kVmaxThreads - 1) /
                                                            (8 * kVmaxThreads));
    k_vmax<<<dim3(bx, (unsigned)g.F), kVmaxThreads, 0, st>>>(V32, plane, vmax);
    const int64_t nq = (int64_t)g.F * g.K * Cp;
    k_quant_v<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(V32, g.C, g.K, Cp, g.F, vmax, sV,
                                                            Vp[0], Vp[1], Vp[2], mode);
    const dim3 gq((unsigned)(Tp / kQT), (unsigned)(Cp / kQC));
    const size_t qsm = (size_t)parts * g.F * kQT * kQC * sizeof(uint16_t);
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
      k_quant_input_tiled<2><<<gq, kQT * kQC, qsm, st>>>(x, g, M, S, Cp, Tp, Up[0], Up[1], Up[2],
                                                         mode);
    else if (M.m == 4)
      k_quant_input_tiled<4><<<gq, kQT * kQC, qsm, st>>>(x, g, M, S, Cp, Tp, Up[0], Up[1], Up[2],
                                                         mode);
    else
      k_quant_input_tiled<6><<<gq, kQT * kQC, qsm, st>>>(x, g, M, S, Cp, Tp, Up[0], Up[1], Up[2],
                                                         mode);
    note_launches(4);
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
  const size_t smem = tc_smem_bytes(NB, parts);
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
