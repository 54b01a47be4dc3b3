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
// (FP32) rounded into the blocked image of [F][Tp][Cp] (MN-major A operand);
// k_tc_gemm; the general output transform.
// k_tc_gemm: one CTA = one frequency x 128 tiles (MMA M) x NB output
// channels (MMA N <= 256), contraction over Cp in chunks of 64 channels
// (one 128-byte swizzle row per operand row).  The quantising kernels write
// the operands as the SWIZZLE_128B shared-memory images of these chunks (A
// MN-major, B K-major), so one thread moves each chunk with one bulk copy
// per operand part (mbarrier-counted), issues tcgen05.mma (K = 16 per
// instruction) and commits to a second mbarrier; every wait is bounded and
// records an error instead of hanging.  k_tc_gemm_ws, the warp-specialised
// persistent form (a producer, an MMA issuer and epilogue warps over a ring
// of stages and two TMEM accumulator buffers), takes the split x6 layers and
// the others whose contraction has four or more chunks.
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
#include "packed.cuh"

namespace wino {

constexpr int kTcM = 128;    // tiles per CTA (MMA M)
constexpr int kTcKc = 64;    // channels per chunk: one 128-byte row per operand row

// Operand parts in HBM are the shared-memory images the contraction copies
// whole (one bulk copy per operand part and chunk): U per (frequency,
// 128-tile block, 64-channel chunk) one 16 KB block, V per (frequency,
// NB-channel k block, chunk) one NB x 128-byte block.
// U is the MMA's A operand in MN-major form (tiles contiguous): the block is
// 16 atoms of 1024 bytes, atom (g, a) at (2 g + a) x 1024 holding channels
// 8 g .. 8 g + 7 (rows r = c % 8, 128 bytes each) of tiles 64 a .. 64 a + 63;
// the 16-byte piece j (8 tiles) of row r sits at position j ^ r (the
// 128-byte swizzle).  Atoms along the tiles are 1024 bytes apart (the
// descriptor's leading byte offset), groups of 8 channels 2048 bytes (its
// stride byte offset).  V is the B operand in K-major form: row r of a block
// (an output channel) is 128 bytes at r x 128, its piece j (8 channels) at
// position j ^ (r & 7).  Element index of (f, tile t, channel c) in a U part,
// and of (f, output channel k, c) in a V part:
__host__ __device__ __forceinline__ int64_t tc_u_index(int f, int64_t t, int c, int64_t ntb,
                                                       int nch) {
  const int64_t blk = ((int64_t)f * ntb + t / kTcM) * nch + c / kTcKc;
  const int tl = (int)(t % kTcM), cl = c % kTcKc;
  const int r = cl % 8, j = (tl % 64) / 8;
  return blk * (kTcM * kTcKc) + (((cl / 8) * 2 + tl / 64) * 8 + r) * 64 + ((j ^ r) * 8) + (tl % 8);
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
// U0/U1/U2, scaled, in the MN-major image of tc_u_index; rows t >= T and
// channels c >= C are zero.  A warp takes one channel of 64 consecutive
// tiles (F(2x2), F(4x4): two adjacent tiles per lane) or 32 (F(6x6): one per
// lane), so that its patch loads run along the input rows (F(4x4): a lane's
// two patches are one run of ten columns per row, loaded as one 32-byte
// vector with the two edge columns from the neighbouring lanes, or as two
// 16-byte vectors and two scalars) and its results for one frequency and
// part are one contiguous run of the image: 128 bytes (a whole line, two
// tiles' 16-bit values in each 32-bit store) or 64 bytes.  Nothing is
// staged in shared memory.  Launch: grid (Tp / 64, Cp / 8) blocks of 256
// threads for F(2x2) and F(4x4), (Tp / 64, Cp / 4) for F(6x6).
constexpr int kQuantThreads = 256;

// B^T d B of one patch, FP32 in the layer's order (column transforms B^T d,
// then the rows times B; every sum from zero with fmaf, inner index
// ascending), frequency f = i alpha + j at out(f, v).  The column
// transforms overwrite d, one column at a time.
template <int A, class Out>
__device__ __forceinline__ void bt_d_b(float (&d)[A][A], const LayerMats& Mx, Out out) {
#pragma unroll
  for (int l = 0; l < A; ++l) {
    float col[A];
#pragma unroll
    for (int i = 0; i < A; ++i) {
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < A; ++q) acc = fmaf(Mx.BT[i * A + q], d[q][l], acc);
      col[i] = acc;
    }
#pragma unroll
    for (int i = 0; i < A; ++i) d[i][l] = col[i];
  }
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
#pragma unroll
      for (int l = 0; l < A; ++l) acc = fmaf(d[i][l], Mx.BT[j * A + l], acc);
      out(i * A + j, acc);
    }
}

// The alpha x alpha input patch of tile t, channel c: zero outside the
// image, and all zero for t >= T or c >= C.
template <int MM>
__device__ __forceinline__ void load_patch(const float* __restrict__ x, const LayerGeom& g,
                                           int64_t t, int c, float (&d)[MM + 2][MM + 2]) {
  constexpr int A = MM + 2;
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int j = 0; j < A; ++j) d[i][j] = 0.0f;
  if (t >= g.T || c >= g.C) return;
  const int tpi = g.th * g.tw;
  const int n = (int)(t / tpi);
  const int rem = (int)(t - (int64_t)n * tpi);
  const int ti = rem / g.tw, tj = rem - ti * g.tw;
  const int h0 = ti * MM - g.pad, w0 = tj * MM - g.pad;
  const float* xc = x + ((int64_t)n * g.C + c) * g.H * g.W;
  // F(6x6) inside the row (pad 1, even W, 8-byte aligned rows): three
  // 8-byte vectors and two scalars per row
  const bool vec2 = MM == 6 && g.pad == 1 && (g.W & 1) == 0 && (((uintptr_t)x) & 7) == 0 &&
                    w0 + A - 2 < g.W;
#pragma unroll
  for (int i = 0; i < A; ++i) {
    const int hh = h0 + i;
    if ((unsigned)hh >= (unsigned)g.H) continue;
    const float* row = xc + (int64_t)hh * g.W;
    if (vec2) {
      const float2* r2 = reinterpret_cast<const float2*>(row + w0 + 1);
#pragma unroll
      for (int v = 0; v < (A - 2) / 2; ++v) {
        const float2 p = __ldg(r2 + v);
        d[i][1 + 2 * v] = p.x;
        d[i][2 + 2 * v] = p.y;
      }
      if (w0 >= 0) d[i][0] = __ldg(row + w0);
      if (w0 + A - 1 < g.W) d[i][A - 1] = __ldg(row + w0 + A - 1);
    } else {
#pragma unroll
      for (int j = 0; j < A; ++j) {
        const int ww = w0 + j;
        if ((unsigned)ww < (unsigned)g.W) d[i][j] = __ldg(row + ww);
      }
    }
  }
}

// 32 bytes of x (8 floats, 32-byte aligned) in one load.
__device__ __forceinline__ void ldg8(const float* p, float (&v)[8]) {
  asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                 "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}

// F(4x4) tile pairs, W a multiple of 8 and x 32-byte aligned: a tile row
// has an even number of tiles (and T is even), so the lane's two tiles t, t
// + 1 (t even) share a tile row and start at an even tj.  Per input row the
// lane loads columns 4 tj .. 4 tj + 7 as one 32-byte vector (the warp: one
// contiguous run); column 4 tj - 1 is column 7 of lane q - 1 and column
// 4 tj + 8 column 0 of lane q + 1 whenever those columns are inside the row
// (the neighbours hold the adjacent tiles of the same tile row), else zero
// padding, and the warp's first and last lanes load them.  All six rows'
// loads are issued before the first shuffle, which waits on them, so that
// they are in flight together.  Called by every lane of the warp, lane q
// with t = t_w + 2q.
__device__ __forceinline__ void load_pair_f4_v8(const float* __restrict__ x, const LayerGeom& g,
                                                int64_t t, int c, int lane,
                                                unsigned long long (&d)[6][6]) {
  const bool live = t < g.T && c < g.C;
  int n = 0, ti = 0, tj = 0;
  if (live) {
    const int tpi = g.th * g.tw;
    n = (int)(t / tpi);
    const int rem = (int)(t - (int64_t)n * tpi);
    ti = rem / g.tw;
    tj = rem - ti * g.tw;
  }
  const int h0 = ti * 4 - 1, c0 = tj * 4;
  const float* xc = x + ((int64_t)n * g.C + c) * g.H * g.W;
  const bool has_l = live && c0 > 0, has_r = live && c0 + 8 < g.W;
  float v[6][8], el[6], er[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const int hh = h0 + i;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[i][k] = 0.0f;
    el[i] = 0.0f;
    er[i] = 0.0f;
    if (live && (unsigned)hh < (unsigned)g.H) {
      const float* row = xc + (int64_t)hh * g.W + c0;
      ldg8(row, v[i]);
      if (lane == 0 && has_l) el[i] = __ldg(row - 1);
      if (lane == 31 && has_r) er[i] = __ldg(row + 8);
    }
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const bool in = live && (unsigned)(h0 + i) < (unsigned)g.H;
    float e0 = __shfl_up_sync(0xffffffffu, v[i][7], 1);
    float e9 = __shfl_down_sync(0xffffffffu, v[i][0], 1);
    if (!(in && has_l))
      e0 = 0.0f;
    else if (lane == 0)
      e0 = el[i];
    if (!(in && has_r))
      e9 = 0.0f;
    else if (lane == 31)
      e9 = er[i];
    d[i][0] = pack2(e0, v[i][3]);
    d[i][1] = pack2(v[i][0], v[i][4]);
    d[i][2] = pack2(v[i][1], v[i][5]);
    d[i][3] = pack2(v[i][2], v[i][6]);
    d[i][4] = pack2(v[i][3], v[i][7]);
    d[i][5] = pack2(v[i][4], e9);
  }
}

// F(4x4) tile pairs in one tile row, W a multiple of 4 and x 16-byte
// aligned: columns 4 tj - 1 .. 4 tj + 8 per row (tile t takes 0-5, tile t + 1
// takes 4-9) as two 16-byte vectors and two scalars; 4 tj .. 4 tj + 7 lie
// inside the row (tile tj + 1 exists).  False (nothing loaded) when the
// pair does not qualify.
__device__ __forceinline__ bool load_pair_f4_v4(const float* __restrict__ x, const LayerGeom& g,
                                                int64_t t, int c,
                                                unsigned long long (&d)[6][6]) {
  if (!(t + 1 < g.T && c < g.C && g.pad == 1 && (g.W & 3) == 0 && (((uintptr_t)x) & 15) == 0))
    return false;
  const int tpi = g.th * g.tw;
  const int n = (int)(t / tpi);
  const int rem = (int)(t - (int64_t)n * tpi);
  const int ti = rem / g.tw, tj = rem - ti * g.tw;
  if (tj + 1 >= g.tw) return false;  // the pair spans two tile rows
  const int h0 = ti * 4 - 1, c0 = tj * 4;
  const float* xc = x + ((int64_t)n * g.C + c) * g.H * g.W;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const int hh = h0 + i;
    float e0 = 0.0f, e9 = 0.0f;
    float4 v0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), v1 = v0;
    if ((unsigned)hh < (unsigned)g.H) {
      const float* row = xc + (int64_t)hh * g.W + c0;
      v0 = __ldg(reinterpret_cast<const float4*>(row));
      v1 = __ldg(reinterpret_cast<const float4*>(row + 4));
      if (c0 > 0) e0 = __ldg(row - 1);
      if (c0 + 8 < g.W) e9 = __ldg(row + 8);
    }
    d[i][0] = pack2(e0, v0.w);
    d[i][1] = pack2(v0.x, v1.x);
    d[i][2] = pack2(v0.y, v1.y);
    d[i][3] = pack2(v0.z, v1.z);
    d[i][4] = pack2(v0.w, v1.w);
    d[i][5] = pack2(v1.x, e9);
  }
  return true;
}

// The patches of tiles t and t + 1 (channel c) as FP32 pairs, tile t in the
// low half.  Called by every lane of the warp, lane q with t = t_w + 2q.
template <int MM>
__device__ __forceinline__ void load_patch_pair(const float* __restrict__ x, const LayerGeom& g,
                                                int64_t t, int c, int lane,
                                                unsigned long long (&d)[MM + 2][MM + 2]) {
  constexpr int A = MM + 2;
  if constexpr (MM == 4) {
    if (g.pad == 1 && (g.W & 7) == 0 && (((uintptr_t)x) & 31) == 0) {
      load_pair_f4_v8(x, g, t, c, lane, d);
      return;
    }
    if (load_pair_f4_v4(x, g, t, c, d)) return;
  }
  float p0[A][A], p1[A][A];
  load_patch<MM>(x, g, t, c, p0);
  load_patch<MM>(x, g, t + 1, c, p1);
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int j = 0; j < A; ++j) d[i][j] = pack2(p0[i][j], p1[i][j]);
}

// MODE 1-4 fixes the form at compile time (its parts, stores and pointer
// updates only); MODE 0 takes it from `mode_rt`.
template <int MM, int MODE>
__global__ void __launch_bounds__(kQuantThreads) k_quant_input_mn(
    const float* __restrict__ x, const LayerGeom g, const LayerMats Mx, const TcScales S, int Cp,
    int64_t Tp, uint16_t* __restrict__ U0, uint16_t* __restrict__ U1, uint16_t* __restrict__ U2,
    int mode_rt) {
  const int mode = MODE != 0 ? MODE : mode_rt;
  constexpr int A = MM + 2, F = A * A;
  constexpr int TPL = A <= 6 ? 2 : 1;    // tiles per lane
  constexpr int WT = 64 / (32 * TPL);    // warps per 64 tiles
  constexpr int WC = (kQuantThreads / 32) / WT;  // channels per block
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * 64 + (warp % WT) * (32 * TPL) + lane * TPL;
  const int c = blockIdx.y * WC + warp / WT;
  const int64_t ntb = Tp / kTcM;
  const int nch = Cp / kTcKc;
  // element index of (f, t, c) = base + f * fstride
  const int64_t base = tc_u_index(0, t, c, ntb, nch);
  const int64_t fstride = ntb * nch * (int64_t)(kTcM * kTcKc);
  const bool fp16 = mode == 2;
  if constexpr (TPL == 2) {
    // two tiles per lane as FP32 pairs: B^T d B in fma.rn.f32x2 (each half
    // the scalar transform's fmaf sequence, so the same bits), the scale in
    // mul.rn.f32x2, the split in paired conversions; each 32-bit store
    // holds both tiles' 16-bit values (tile t, even, at the lower address)
    unsigned long long d[A][A];
    load_patch_pair<MM>(x, g, t, c, lane, d);
#pragma unroll
    for (int l = 0; l < A; ++l) {
      unsigned long long col[A];
#pragma unroll
      for (int i = 0; i < A; ++i) {
        unsigned long long acc = 0ull;
#pragma unroll
        for (int q = 0; q < A; ++q) acc = fma2(pack_dup(Mx.BT[i * A + q]), d[q][l], acc);
        col[i] = acc;
      }
#pragma unroll
      for (int i = 0; i < A; ++i) d[i][l] = col[i];
    }
    // running pointers to frequency f (f ascending below)
    uint32_t* W0 = reinterpret_cast<uint32_t*>(U0 + base);
    uint32_t* W1 = reinterpret_cast<uint32_t*>(U1 + base);
    uint32_t* W2 = reinterpret_cast<uint32_t*>(U2 + base);
    const int64_t fs = fstride / 2;
#pragma unroll
    for (int i = 0; i < A; ++i)
#pragma unroll
      for (int j = 0; j < A; ++j) {
        unsigned long long acc = 0ull;
#pragma unroll
        for (int l = 0; l < A; ++l) acc = fma2(d[i][l], pack_dup(Mx.BT[j * A + l]), acc);
        const int f = i * A + j;
        const unsigned long long v = mul2(acc, pack_dup(S.sU[f]));
        const uint32_t hi = cvt16x2(v, fp16);
        *W0 = hi;
        if (mode == 3 || mode == 4) {
          const unsigned long long r1 = sub2(v, widen16x2(hi, fp16));  // exact
          const uint32_t mid = cvt16x2(r1, fp16);
          *W1 = mid;
          if (mode == 4) *W2 = cvt16x2(sub2(r1, widen16x2(mid, fp16)), fp16);
        }
        W0 += fs;
        W1 += fs;
        W2 += fs;
      }
  } else {
    float d[A][A];
    load_patch<MM>(x, g, t, c, d);
    // running pointers to frequency f (bt_d_b emits f ascending)
    uint16_t* D0 = U0 + base;
    uint16_t* D1 = U1 + base;
    uint16_t* D2 = U2 + base;
    const int parts = tc_parts(mode);
    bt_d_b<A>(d, Mx, [&](int f, float v) {
      uint16_t q[3];
      split_parts(v * S.sU[f], mode, q);
      *D0 = q[0];
      if (parts > 1) *D1 = q[1];
      if (parts > 2) *D2 = q[2];
      D0 += fstride;
      D1 += fstride;
      D2 += fstride;
    });
  }
  (void)F;
}

// k_quant_input_mn with the form (1 BF16, 2 FP16, 3 split-BF16x3, 4
// split-BF16x6) as a template argument.
template <int MM>
static void launch_quant_input(dim3 gq, cudaStream_t st, const float* x, const LayerGeom& g,
                               const LayerMats& M, const TcScales& S, int Cp, int64_t Tp,
                               uint16_t* U0, uint16_t* U1, uint16_t* U2, int mode) {
  if (mode == 1)
    k_quant_input_mn<MM, 1><<<gq, kQuantThreads, 0, st>>>(x, g, M, S, Cp, Tp, U0, U1, U2, mode);
  else if (mode == 2)
    k_quant_input_mn<MM, 2><<<gq, kQuantThreads, 0, st>>>(x, g, M, S, Cp, Tp, U0, U1, U2, mode);
  else if (mode == 3)
    k_quant_input_mn<MM, 3><<<gq, kQuantThreads, 0, st>>>(x, g, M, S, Cp, Tp, U0, U1, U2, mode);
  else
    k_quant_input_mn<MM, 4><<<gq, kQuantThreads, 0, st>>>(x, g, M, S, Cp, Tp, U0, U1, U2, mode);
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

// The same for an MN-major operand (the A images, tc_u_index): 1024-byte
// atoms of 8 rows (channels) x 128 bytes (64 tiles), leading byte offset =
// 1024 bytes between the atoms along M, stride byte offset = 2048 bytes
// between groups of 8 rows along K.
__device__ __forceinline__ uint64_t sw128_desc_mn(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(1024u >> 4) << 16;
  d |= (uint64_t)(2048u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A and B format
// (bits 7-9, 10-12: 0 = F16, 1 = BF16), A MN-major (bit 15 = 1), B K-major
// (bit 16 = 0), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ __forceinline__ uint32_t f16_idesc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | (1u << 15) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
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
          ad[pp] = sw128_desc_mn(smem_addr(As + pp * a_bytes) + kk * 4096);
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

// ---------------------------------------------------------------------------
// Warp-specialised persistent form of the contraction.
// ---------------------------------------------------------------------------
// One CTA per SM loops over work units (frequency f, 128-tile block, NB-
// channel k block), the k blocks of one (f, tile block) adjacent so that
// its U blocks are re-read from L2.  Roles:
//   warp 0, lane 0  producer: per (unit, 64-channel chunk) one bulk copy per
//                   operand part of A and of B into an NS-stage ring, each
//                   fill counted in bytes on full[s];
//   warp 1, lane 0  MMA issuer: per unit, waits until the epilogue has
//                   drained the unit's TMEM accumulator buffer (two
//                   buffers, alternating), then per chunk waits full[s],
//                   issues the MMAs and commits to empty[s]; after the
//                   unit's last chunk it commits to tfull[buffer];
//   warps 2-5       epilogue: wait tfull[buffer], read their 32 TMEM lanes
//                   (tiles) of the buffer, write M = (D (+ D')) / (sU sV)
//                   and arrive on tempty[buffer].
// So the epilogue of unit i overlaps the MMAs of unit i + 1 and the copies
// of the chunks after it.  The products per 16-channel step and their
// accumulators are those of k_tc_gemm, so M is the same.  Every wait is
// bounded; a role whose wait gave up records the error and stops, and the
// CTA drains its copies and MMAs before TMEM is freed.  Launch: one CTA of
// 192 threads per SM (shared memory and TMEM keep it alone), NS ring stages.
constexpr int kTwsThreads = 192;
constexpr int kTwsMaxNS = 8;
// The layer uses this form for the split x6 form, and for the others when
// the contraction has at least this many 64-channel chunks (C >= 256): on
// the VGG16 stages it took stages 3-5 from 134 / 99 / 34 to 117 / 77 / 32 us
// (BF16 F(4x4), with the output transform), while with one or two chunks per
// unit the one- and two-part forms ran 2-8% behind k_tc_gemm (also with
// eight epilogue warps instead of four); the split x6 stacks are fastest
// with this form on every stage.
constexpr int kTwsMinChunks = 4;

__device__ __forceinline__ void mbar_init_n(uint32_t bar, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(n));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(kTwsThreads, 1) k_tc_gemm_ws(const TcGemmArgs P, int NS,
                                                              int F) {
  extern __shared__ __align__(1024) unsigned char wsm_raw[];
  unsigned char* wsm = wsm_raw + ((1024u - (smem_addr(wsm_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t full[kTwsMaxNS], empty[kTwsMaxNS], tfull[2], tempty[2], done;
  __shared__ uint32_t tmem_holder;
  __shared__ int s_issued, s_consumed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int parts = tc_parts(P.mode);
  const int NB = P.NB;
  const int nch = P.Cp / kTcKc, nkb = P.K / NB;
  const int64_t ntb = P.Tp / kTcM;
  const int64_t n_units = (int64_t)F * ntb * nkb;
  const uint32_t a_bytes = kTcM * 128, b_bytes = (uint32_t)NB * 128;
  const uint32_t stage_bytes = (uint32_t)parts * (a_bytes + b_bytes);
  const uint32_t ncols = (uint32_t)max(32, parts == 3 ? 2 * NB : NB);  // one buffer
  const uint32_t ring = smem_addr(wsm);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_addr(&tmem_holder)),
                 "r"(2 * ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init1(smem_addr(&full[s]));
      mbar_init1(smem_addr(&empty[s]));
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init1(smem_addr(&tfull[b]));
      mbar_init_n(smem_addr(&tempty[b]), 4);
    }
    mbar_init1(smem_addr(&done));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_issued = 0;
    s_consumed = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_holder;

  bool ok = true;
  if (warp == 0 && lane == 0) {
    // producer
    int it = 0;
    for (int64_t u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const int kb = (int)(u % nkb);
      const int64_t r = u / nkb;
      const int64_t tb = r % ntb;
      const int f = (int)(r / ntb);
      for (int ch = 0; ch < nch; ++ch, ++it) {
        const int s = it % NS;
        if (it >= NS && !mbar_wait_bounded(smem_addr(&empty[s]), (uint32_t)((it / NS - 1) & 1))) {
          ok = false;
          break;
        }
        const uint32_t dst = ring + (uint32_t)s * stage_bytes, bar = smem_addr(&full[s]);
        mbar_expect_tx(bar, stage_bytes);
        const int64_t ua = (((int64_t)f * ntb + tb) * nch + ch) * (int64_t)(kTcM * kTcKc);
        const int64_t vb = (((int64_t)f * nkb + kb) * nch + ch) * ((int64_t)NB * kTcKc);
        for (int pp = 0; pp < parts; ++pp) {
          bulk_g2s(dst + pp * a_bytes, P.U[pp] + ua, a_bytes, bar);
          bulk_g2s(dst + parts * a_bytes + pp * b_bytes, P.V[pp] + vb, b_bytes, bar);
        }
      }
    }
    s_issued = it;
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = f16_idesc(P.mode == 2 ? 0 : 1, kTcM, NB);
    int it = 0, lu = 0;
    for (int64_t u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++lu) {
      const int b = lu & 1;
      if (lu >= 2 && !mbar_wait_bounded(smem_addr(&tempty[b]), (uint32_t)((lu / 2 - 1) & 1))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t td = tmem + (uint32_t)b * ncols, td2 = td + (uint32_t)NB;
      for (int ch = 0; ch < nch; ++ch, ++it) {
        const int s = it % NS;
        if (!mbar_wait_bounded(smem_addr(&full[s]), (uint32_t)((it / NS) & 1))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t As = ring + (uint32_t)s * stage_bytes, Bs = As + parts * a_bytes;
#pragma unroll
        for (int kk = 0; kk < kTcKc / 16; ++kk) {
          const uint32_t acc = (ch > 0 || kk > 0) ? 1u : 0u;
          uint64_t ad[3], bd[3];
          for (int pp = 0; pp < parts; ++pp) {
            ad[pp] = sw128_desc_mn(As + pp * a_bytes + kk * 4096);
            bd[pp] = sw128_desc(Bs + pp * b_bytes + kk * 32);
          }
          mma_f16(td, ad[0], bd[0], idesc, acc);
          if (parts == 2) {
            mma_f16(td, ad[0], bd[1], idesc, 1u);
            mma_f16(td, ad[1], bd[0], idesc, 1u);
          } else if (parts == 3) {
            mma_f16(td2, ad[0], bd[1], idesc, acc);
            mma_f16(td2, ad[1], bd[0], idesc, 1u);
            mma_f16(td2, ad[0], bd[2], idesc, 1u);
            mma_f16(td2, ad[2], bd[0], idesc, 1u);
            mma_f16(td2, ad[1], bd[1], idesc, 1u);
          }
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_addr(&empty[s]))
            : "memory");
      }
      if (!ok) break;
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_addr(&tfull[b]))
          : "memory");
    }
    s_consumed = it;
    // arrives once every MMA issued above has completed
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_addr(&done))
        : "memory");
  } else if (warp >= 2) {
    // epilogue: TMEM lanes 32 (warp % 4) .. are this warp's tiles
    const int lg = warp & 3;
    int lu = 0;
    for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x, ++lu) {
      const int b = lu & 1;
      const bool got = mbar_wait_bounded(smem_addr(&tfull[b]), (uint32_t)((lu / 2) & 1));
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const int kb = (int)(u % nkb);
      const int64_t r = u / nkb;
      const int64_t tb = r % ntb;
      const int f = (int)(r / ntb);
      const float inv = 1.0f / (P.S.sU[f] * P.sV[f]);  // exact: powers of two
      const int64_t t = tb * kTcM + lg * 32 + lane;
      const uint32_t base = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)b * ncols;
      for (int col = 0; col < NB; col += 16) {
        uint32_t v[16], w[16];
        tmem_ld16(base + (uint32_t)col, v);
        if (parts == 3) {
          tmem_ld16(base + (uint32_t)(NB + col), w);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            v[j] = __float_as_uint(__fadd_rn(__uint_as_float(v[j]), __uint_as_float(w[j])));
        }
        if (t < P.T) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            P.M[((int64_t)f * P.K + kb * NB + col + j) * P.T + t] = __uint_as_float(v[j]) * inv;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&tempty[b]));
    }
  }
  const bool cta_ok = __syncthreads_and(ok ? 1 : 0) != 0;
  if (tid == 0) {
    // every MMA completed (the issuer's last commit), then, after a failed
    // wait, the fills that were issued but not consumed
    const bool fin = mbar_wait_bounded(smem_addr(&done), 0u);
    if (!cta_ok || !fin) {
      atomicExch(P.err, 1);
      for (int it = s_consumed; it < s_issued; ++it)
        (void)mbar_wait_bounded(smem_addr(&full[it % NS]), (uint32_t)((it / NS) & 1));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(2 * ncols));
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
  // the filter side (max |V|, V rounded and split) does not depend on x: it
  // runs on the side stream, beside the quantising input transform, and the
  // caller's stream waits for it before the contraction
  cudaStream_t aux = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  {
    int rc = side_stream(&aux, &fork, &join);
    if (rc != WINO_OK) return rc;
  }
  {
    // profiled as one phase on the caller's stream, fork to join (the two
    // sides overlap, so per-kernel events would count the overlap twice)
    ProfScope ps(kKTcTransform, st);
    WINO_CUDA_TRY(cudaEventRecord(fork, st));
    WINO_CUDA_TRY(cudaStreamWaitEvent(aux, fork, 0));
    WINO_CUDA_TRY(cudaMemsetAsync(vmax, 0, (size_t)g.F * 4, aux));
    {
      // per-frequency maxima of V (each block reduces up to 8 kernels per
      // thread), then V recomputed, scaled and split
      const int64_t nck = (int64_t)g.C * g.K;
      const unsigned bf = (unsigned)std::max<int64_t>(1, std::min<int64_t>(
                                                             (nck + 8 * kFvThreads - 1) /
                                                             (8 * kFvThreads), 1 << 16));
      const unsigned bq = (unsigned)(((int64_t)g.K * Cp + 255) / 256);
      if (M.m == 2) {
        k_filter_vmax<2><<<bf, kFvThreads, 0, aux>>>(w, g.C, g.K, M, vmax);
        k_filter_quant<2><<<bq, 256, 0, aux>>>(w, g.C, g.K, Cp, M, vmax, sV, Vp[0], Vp[1], Vp[2], mode,
                                              NB);
      } else if (M.m == 4) {
        k_filter_vmax<4><<<bf, kFvThreads, 0, aux>>>(w, g.C, g.K, M, vmax);
        k_filter_quant<4><<<bq, 256, 0, aux>>>(w, g.C, g.K, Cp, M, vmax, sV, Vp[0], Vp[1], Vp[2], mode,
                                              NB);
      } else {
        k_filter_vmax<6><<<bf, kFvThreads, 0, aux>>>(w, g.C, g.K, M, vmax);
        k_filter_quant<6><<<bq, 256, 0, aux>>>(w, g.C, g.K, Cp, M, vmax, sV, Vp[0], Vp[1], Vp[2], mode,
                                              NB);
      }
      note_launches(2);
    }
    WINO_CUDA_TRY(cudaEventRecord(join, aux));
    {
      const dim3 gq((unsigned)(Tp / 64), (unsigned)(Cp / (M.m == 6 ? 4 : 8)));
      if (M.m == 2)
        k_quant_input_mn<2, 0><<<gq, kQuantThreads, 0, st>>>(x, g, M, S, Cp, Tp, Up[0], Up[1],
                                                             Up[2], mode);
      else if (M.m == 4)
        launch_quant_input<4>(gq, st, x, g, M, S, Cp, Tp, Up[0], Up[1], Up[2], mode);
      else
        launch_quant_input<6>(gq, st, x, g, M, S, Cp, Tp, Up[0], Up[1], Up[2], mode);
      note_launches(1);
    }
    WINO_CUDA_TRY(cudaStreamWaitEvent(st, join, 0));
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
  if (parts < 3 && Cp / kTcKc < kTwsMinChunks) {
    ProfScope ps(kKTcGemm, st);
    dim3 grid((unsigned)(Tp / kTcM), (unsigned)(g.K / NB), (unsigned)g.F);
    k_tc_gemm<<<grid, kTcThreads, smem, st>>>(P);
    note_launches(1);
  } else {
    // warp-specialised persistent form: one CTA per SM, as many ring stages
    // as fit in 200 KB
    ProfScope ps(kKTcGemm, st);
    const size_t stage = (size_t)parts * ((size_t)kTcM * 128 + (size_t)NB * 128);
    int ns = (int)((200 * 1024) / stage);
    ns = ns < 2 ? 2 : (ns > kTwsMaxNS ? kTwsMaxNS : ns);
    const size_t smem_ws = (size_t)ns * stage + 1024;
    static bool ws_attr[16] = {false};
    if (!ws_attr[dev]) {
      WINO_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm_ws, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         210 * 1024));
      ws_attr[dev] = true;
    }
    int sms = 0;
    WINO_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t units = (int64_t)g.F * (Tp / kTcM) * (g.K / NB);
    const unsigned grid = (unsigned)std::min<int64_t>(units, sms);
    k_tc_gemm_ws<<<grid, kTwsThreads, smem_ws, st>>>(P, ns, g.F);
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
