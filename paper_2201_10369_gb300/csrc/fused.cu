// fused.cu -- fused FP32 Winograd layer F(m x m, 3 x 3), m in {2, 4, 6}.
//
// One CTA owns TB consecutive tiles x KB output channels and ALL alpha^2
// frequencies, so neither the transformed input U nor the Winograd-domain
// products M ever leave the SM (the unfused pipeline in layer.cu writes and
// re-reads both through HBM).  Per chunk of CC input channels:
//   1. cp.async (zero-filled outside the image: padding and ragged tiles)
//      brings the alpha x alpha input patches and the V[f][c][k0..k0+KB)
//      filter rows into shared memory, double-buffered so chunk i+1 loads
//      while chunk i is contracted;
//   2. B^T d B (Eq. (9)) in two passes, column transforms then row
//      transforms, into U_s[f][c][t];
//   3. each thread owns one frequency f and an 8 (tiles) x 16 (channels)
//      register microtile and accumulates sum_c U_s[f][c][t] V_s[f][c][k]
//      with fmaf, c ascending (the same order as the general path, so the
//      layer stays bit-identical to it).
// Epilogue: the alpha^2 accumulators of each (tile, k) meet in shared
// memory; A^T M A and the cropped write-back follow.
// The filter transform V = G g G^T (layer.cu, K4) runs first; it is O(C K)
// and amortised over all tiles (Sec. 4.1).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wino.h"
#include "common.cuh"

namespace wino {

__global__ void k_filter_transform(const float* __restrict__ w, float* __restrict__ V, int dim,
                                   int C, int K, const LayerMats M);

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src),
               "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
               "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

}  // namespace

// Thread mapping: a warp owns LX * FPL frequencies; its 32 lanes split into
// LX (frequency) x LT (tiles) x LK (channels); each lane accumulates FPL
// frequencies x MT tiles x MK channels.  Its MK channels are MK/4 groups of
// 4 consecutive channels, group s at s * 4 * LK + lane_k * 4, so the LK lanes
// of a frequency read one contiguous run of V_s per group.
template <int MM, int LX, int LT, int LK, int FPL, int MT, int MK, int CC>
struct FusedCfg {
  static constexpr int A = MM + 2;            // alpha for r = 3
  static constexpr int F = A * A;             // frequencies
  static constexpr int TB = LT * MT;          // tiles per CTA
  static constexpr int KB = LK * MK;          // output channels per CTA
  static constexpr int NW = F / (LX * FPL);   // warps per CTA
  static constexpr int NT = NW * 32;          // threads per CTA
  static constexpr int VPL = CC * KB + 16;    // V_s frequency plane (padded)
  static constexpr int UPL = CC * TB + 4;     // U_s frequency plane (padded)
  static constexpr int D_FL = CC * TB * A * A;  // raw patches per buffer
  static constexpr int V_FL = F * VPL;          // filter rows per buffer
  static constexpr int T_FL = CC * TB * A * A;  // column-pass result
  static constexpr int U_FL = F * UPL;          // transformed input
  static constexpr int MAIN_FL = 2 * D_FL + 2 * V_FL + T_FL + U_FL;
  static constexpr int EKB = KB + 4;            // epilogue row (padded)
  static constexpr int EPI_FL = F * TB * EKB;   // accumulators in the epilogue
  static constexpr int SMEM_FL = MAIN_FL > EPI_FL ? MAIN_FL : EPI_FL;
  static constexpr size_t SMEM = (size_t)SMEM_FL * sizeof(float);
  static_assert(LX * LT * LK == 32, "a warp is 32 lanes");
  static_assert(F % (LX * FPL) == 0 && NW % 4 == 0, "whole warps, 4 per SM sub-partition");
  static_assert(MT % 4 == 0 && MK % 4 == 0, "float4 operand loads");
};

#define FUSED_TPARAMS int MM, int LX, int LT, int LK, int FPL, int MT, int MK, int CC
#define FUSED_TARGS MM, LX, LT, LK, FPL, MT, MK, CC

template <FUSED_TPARAMS>
__global__ void __launch_bounds__(FusedCfg<FUSED_TARGS>::NT, 1)
    k_fused_layer(const float* __restrict__ x, const float* __restrict__ V, float* __restrict__ y,
                  const LayerGeom g, const LayerMats Mx) {
  using Cfg = FusedCfg<FUSED_TARGS>;
  constexpr int A = Cfg::A, F = Cfg::F, NT = Cfg::NT, TB = Cfg::TB, KB = Cfg::KB;
  extern __shared__ __align__(16) float sm[];
  float* Dr = sm;                         // [2][CC][A][A][TB]
  float* Vs = Dr + 2 * Cfg::D_FL;         // [2][F][VPL]
  float* Tm = Vs + 2 * Cfg::V_FL;         // [CC][A][A][TB]
  float* Us = Tm + Cfg::T_FL;             // [F][UPL]  (c-major inside a plane)

  const int tid = threadIdx.x;
  // k-blocks of one tile block are adjacent in launch order, so the CTAs
  // that re-read the same input patches run together (L2 reuse).
  const int nkb = g.K / KB;
  const int k0 = (int)(blockIdx.x % nkb) * KB;
  const int64_t t0 = (int64_t)(blockIdx.x / nkb) * TB;
  const int tpi = g.th * g.tw;
  const int nchunks = (g.C + CC - 1) / CC;
  // ---- per-tile coordinates of this CTA, computed once ----
  __shared__ int64_t s_base[TB];   // element offset of image n, channel 0
  __shared__ int s_h0[TB], s_w0[TB];  // top-left input coordinate (with padding)
  if (tid < TB) {
    const int64_t tg = t0 + tid;
    if (tg < g.T) {
      const int n = (int)(tg / tpi);
      const int rem = (int)(tg - (int64_t)n * tpi);
      const int ti = rem / g.tw, tj = rem - (rem / g.tw) * g.tw;
      s_base[tid] = (int64_t)n * g.C * g.H * g.W;
      s_h0[tid] = ti * MM - g.pad;
      s_w0[tid] = tj * MM - g.pad;
    } else {  // past the last tile: every load fails the bounds test
      s_base[tid] = 0;
      s_h0[tid] = -(1 << 29);
      s_w0[tid] = -(1 << 29);
    }
  }
  __syncthreads();
  const int64_t HW = (int64_t)g.H * g.W;

  // ---- chunk loader (cp.async, zero fill outside the image / beyond C) ----
  auto load_chunk = [&](int ch, int buf) {
    const int c0 = ch * CC;
    float* dbuf = Dr + buf * Cfg::D_FL;
    constexpr int NEL = CC * TB * A * A;
    for (int e = tid; e < NEL; e += NT) {  // Dr[cc][i][j][t], t fastest
      const int t = e % TB;
      const int j = (e / TB) % A;
      const int i = (e / (TB * A)) % A;
      const int cc = e / (TB * A * A);
      const int c = c0 + cc;
      const int hh = s_h0[t] + i, ww = s_w0[t] + j;
      const bool ok = c < g.C && (unsigned)hh < (unsigned)g.H && (unsigned)ww < (unsigned)g.W;
      const float* src = ok ? x + s_base[t] + c * HW + (int64_t)hh * g.W + ww : x;
      cp_async4(smem_u32(dbuf + e), src, ok);
    }
    float* vbuf = Vs + buf * Cfg::V_FL;
    constexpr int NV4 = F * CC * KB / 4;
    for (int e = tid; e < NV4; e += NT) {
      const int kk = (e % (KB / 4)) * 4;
      const int cc = (e / (KB / 4)) % CC;
      const int f = e / (KB / 4 * CC);
      const int c = c0 + cc;
      const bool ok = c < g.C;
      const float* src = ok ? V + ((int64_t)f * g.C + c) * g.K + k0 + kk : V;
      cp_async16(smem_u32(vbuf + f * Cfg::VPL + cc * KB + kk), src, ok);
    }
    cp_async_commit();
  };

  // ---- B^T d B of one chunk: column pass into Tm, row pass into Us ----
  auto transform_chunk = [&](int buf) {
    // column pass: Tm[cc][i][l][t] = sum_q BT[i][q] D[cc][q][l][t]
    const float* dbuf = Dr + buf * Cfg::D_FL;
    for (int e = tid; e < CC * A * TB; e += NT) {  // (cc, column l, t), t fastest
      const int t = e % TB;
      const int l = (e / TB) % A;
      const int cc = e / (TB * A);
      const float* dcol = dbuf + (cc * A * A + l) * TB + t;
      float dv[A];
#pragma unroll
      for (int q = 0; q < A; ++q) dv[q] = dcol[q * A * TB];
      float* tcol = Tm + (cc * A * A + l) * TB + t;
#pragma unroll
      for (int i = 0; i < A; ++i) {
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < A; ++q) acc = fmaf(Mx.BT[i * A + q], dv[q], acc);
        tcol[i * A * TB] = acc;
      }
    }
    __syncthreads();
    // row pass: U[i*A+j][cc][t] = sum_l Tm[cc][i][l][t] BT[j][l]
    for (int e = tid; e < CC * A * TB; e += NT) {  // (cc, row i, t), t fastest
      const int t = e % TB;
      const int i = (e / TB) % A;
      const int cc = e / (TB * A);
      const float* trow = Tm + (cc * A * A + i * A) * TB + t;
      float tv[A];
#pragma unroll
      for (int l = 0; l < A; ++l) tv[l] = trow[l * TB];
#pragma unroll
      for (int j = 0; j < A; ++j) {
        float acc = 0.0f;
#pragma unroll
        for (int l = 0; l < A; ++l) acc = fmaf(tv[l], Mx.BT[j * A + l], acc);
        Us[(i * A + j) * Cfg::UPL + cc * TB + t] = acc;
      }
    }
  };

  // ---- lane's frequencies and microtile ----
  const int warp = tid >> 5, lane = tid & 31;
  const int lx = lane / (LT * LK);
  const int lt = (lane / LK) % LT;
  const int lk = lane % LK;
  const int f0 = (warp * LX + lx) * FPL;  // first of this lane's FPL frequencies
  float acc[FPL][MT][MK];
#pragma unroll
  for (int q = 0; q < FPL; ++q)
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int j = 0; j < MK; ++j) acc[q][i][j] = 0.0f;

  load_chunk(0, 0);
  cp_async_wait_all();
  __syncthreads();
  transform_chunk(0);
  __syncthreads();

  for (int ch = 0; ch < nchunks; ++ch) {
    const int buf = ch & 1;
    if (ch + 1 < nchunks) load_chunk(ch + 1, buf ^ 1);
    const float* vbase = Vs + buf * Cfg::V_FL + lk * 4;
#pragma unroll
    for (int cc = 0; cc < CC; ++cc) {
#pragma unroll
      for (int q = 0; q < FPL; ++q) {
        const float* up = Us + (f0 + q) * Cfg::UPL + cc * TB + lt * MT;
        const float* vp = vbase + (f0 + q) * Cfg::VPL + cc * KB;
        float a[MT], b[MK];
#pragma unroll
        for (int i = 0; i < MT; i += 4) {
          const float4 v = *reinterpret_cast<const float4*>(up + i);
          a[i] = v.x;
          a[i + 1] = v.y;
          a[i + 2] = v.z;
          a[i + 3] = v.w;
        }
#pragma unroll
        for (int s4 = 0; s4 < MK / 4; ++s4) {
          const float4 v = *reinterpret_cast<const float4*>(vp + s4 * 4 * LK);
          b[4 * s4] = v.x;
          b[4 * s4 + 1] = v.y;
          b[4 * s4 + 2] = v.z;
          b[4 * s4 + 3] = v.w;
        }
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
          for (int j = 0; j < MK; ++j) acc[q][i][j] = fmaf(a[i], b[j], acc[q][i][j]);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    if (ch + 1 < nchunks) {
      transform_chunk(buf ^ 1);
      __syncthreads();
    }
  }

  // ---- epilogue: accumulators to Es[f][k][t], then A^T M A per (t, k) ----
  float* Es = sm;
  // Es[f][t][k] with rows of KB + 4 floats: the float4 stores of a warp
  // spread evenly over the banks, and the epilogue's reads (k fastest) are
  // conflict-free.
#pragma unroll
  for (int q = 0; q < FPL; ++q)
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int s4 = 0; s4 < MK / 4; ++s4) {
        float* dst = Es + ((size_t)(f0 + q) * TB + lt * MT + i) * Cfg::EKB + s4 * 4 * LK + lk * 4;
        *reinterpret_cast<float4*>(dst) =
            make_float4(acc[q][i][4 * s4], acc[q][i][4 * s4 + 1], acc[q][i][4 * s4 + 2],
                        acc[q][i][4 * s4 + 3]);
      }
  __syncthreads();
  for (int p = tid; p < TB * KB; p += NT) {
    const int kl = p % KB, t = p / KB;
    const int64_t tg = t0 + t;
    const int k = k0 + kl;
    if (tg >= g.T || k >= g.K) continue;
    float Mv[F];
#pragma unroll
    for (int q = 0; q < F; ++q) Mv[q] = Es[((size_t)q * TB + t) * Cfg::EKB + kl];
    float Z[MM * A];
#pragma unroll
    for (int a = 0; a < MM; ++a)
#pragma unroll
      for (int j = 0; j < A; ++j) {
        float z = 0.0f;
#pragma unroll
        for (int i = 0; i < A; ++i) z = fmaf(Mx.AT[a * A + i], Mv[i * A + j], z);
        Z[a * A + j] = z;
      }
    const int n = (int)(s_base[t] / (g.C * HW));
    const int ti = (s_h0[t] + g.pad) / MM, tj = (s_w0[t] + g.pad) / MM;
    float* yk = y + ((int64_t)n * g.K + k) * g.Ho * g.Wo;
#pragma unroll
    for (int a = 0; a < MM; ++a) {
      const int pr = ti * MM + a;
      float yr[MM];
#pragma unroll
      for (int b = 0; b < MM; ++b) {
        float v = 0.0f;
#pragma unroll
        for (int j = 0; j < A; ++j) v = fmaf(Z[a * A + j], Mx.AT[b * A + j], v);
        yr[b] = v;
      }
      if (pr >= g.Ho) continue;
      float* yrow = yk + (int64_t)pr * g.Wo + tj * MM;
#pragma unroll
      for (int b = 0; b < MM; ++b)
        if (tj * MM + b < g.Wo) yrow[b] = yr[b];
    }
  }
}

template <FUSED_TPARAMS>
static int launch_fused(const float* x, const float* V, float* y, const LayerGeom& g,
                        const LayerMats& M, cudaStream_t st) {
  using Cfg = FusedCfg<FUSED_TARGS>;
  if (g.K % Cfg::KB != 0) return kFallback;
  static bool attr_set[16] = {false};
  int dev = 0;
  WINO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 16 && !attr_set[dev]) {
    WINO_CUDA_TRY(cudaFuncSetAttribute(k_fused_layer<FUSED_TARGS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Cfg::SMEM));
    attr_set[dev] = true;
  }
  const int64_t nblk = (int64_t)(g.K / Cfg::KB) * ((g.T + Cfg::TB - 1) / Cfg::TB);
  if (nblk > 0x7fffffffLL) return kFallback;
  ProfScope ps(kKFused, st);
  k_fused_layer<FUSED_TARGS><<<(unsigned)nblk, Cfg::NT, Cfg::SMEM, st>>>(x, V, y, g, M);
  note_launches(1);
  WINO_CUDA_TRY(cudaGetLastError());
  return WINO_OK;
}

size_t fused_workspace_bytes(const LayerGeom& g) {
  return (size_t)g.F * g.C * g.K * sizeof(float);
}

int layer_forward_fused(const float* x, const float* w, float* y, const LayerGeom& g,
                        const LayerMats& M, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (g.dim != 2 || M.r != 3 || (M.m != 2 && M.m != 4 && M.m != 6) || g.K % 64 != 0)
    return kFallback;
  if (ws_bytes < fused_workspace_bytes(g)) return kFallback;
  float* V = (float*)ws;
  {
    const int64_t n = (int64_t)g.C * g.K;
    ProfScope ps(kKFilter, st);
    k_filter_transform<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, V, g.dim, g.C, g.K, M);
    note_launches(1);
  }
  //                       MM LX LT LK FPL MT MK CC
  switch (M.m) {
    case 2:
      return launch_fused<2, 2, 4, 4, 1, 8, 16, 8>(x, V, y, g, M, st);
    case 4:
      return launch_fused<4, 1, 4, 8, 3, 4, 8, 8>(x, V, y, g, M, st);
    default:
      return launch_fused<6, 8, 1, 4, 1, 8, 16, 4>(x, V, y, g, M, st);
  }
}

// ===========================================================================
// Split variant: a memory-bound input-transform kernel writes U once, then a
// compute-bound kernel runs the alpha^2 contractions with the output
// transform fused into its epilogue (M never leaves the SM).  The main loop
// only streams contiguous U / V rows (16-byte cp.async, double-buffered) and
// issues FFMAs.  Same operation order as the fused kernel, bit for bit.
// U is stored [F][C][Tp], Tp = T rounded up to a multiple of 4.
// ===========================================================================

// One thread per (c, tile), tile fastest: coalesced U rows; the input patch
// loads of neighbouring tiles overlap and hit L1.
template <int MM>
__global__ void __launch_bounds__(256) k_input_transform_r3(const float* __restrict__ x,
                                                            float* __restrict__ U,
                                                            const LayerGeom g, const LayerMats Mx,
                                                            int64_t Tp) {
  constexpr int A = MM + 2;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)g.C * Tp) return;
  const int64_t t = idx % Tp;
  const int c = (int)(idx / Tp);
  if (t >= g.T) return;
  const int tpi = g.th * g.tw;
  const int n = (int)(t / tpi);
  const int rem = (int)(t - (int64_t)n * tpi);
  const int ti = rem / g.tw, tj = rem - (rem / g.tw) * g.tw;
  const int h0 = ti * MM - g.pad, w0 = tj * MM - g.pad;
  const float* xc = x + ((int64_t)n * g.C + c) * g.H * g.W;
  float d[A][A];
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int j = 0; j < A; ++j) {
      const int hh = h0 + i, ww = w0 + j;
      d[i][j] = ((unsigned)hh < (unsigned)g.H && (unsigned)ww < (unsigned)g.W)
                    ? __ldg(xc + (int64_t)hh * g.W + ww)
                    : 0.0f;
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
  const int64_t plane = (int64_t)g.C * Tp;
  float* out = U + (int64_t)c * Tp + t;
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
#pragma unroll
      for (int l = 0; l < A; ++l) acc = fmaf(tm[i][l], Mx.BT[j * A + l], acc);
      out[(i * A + j) * plane] = acc;
    }
}

template <FUSED_TPARAMS>
struct SplitCfg {
  using Base = FusedCfg<FUSED_TARGS>;
  static constexpr int STAGE = Base::F * Base::UPL + Base::F * Base::VPL;
  static constexpr int MAIN_FL = 2 * STAGE;
  static constexpr int SMEM_FL = MAIN_FL > Base::EPI_FL ? MAIN_FL : Base::EPI_FL;
  static constexpr size_t SMEM = (size_t)SMEM_FL * sizeof(float);
};

template <FUSED_TPARAMS>
__global__ void __launch_bounds__(FusedCfg<FUSED_TARGS>::NT, 1)
    k_gemm_otx(const float* __restrict__ U, const float* __restrict__ V, float* __restrict__ y,
               const LayerGeom g, const LayerMats Mx, int64_t Tp) {
  using Cfg = FusedCfg<FUSED_TARGS>;
  using SC = SplitCfg<FUSED_TARGS>;
  constexpr int A = Cfg::A, F = Cfg::F, NT = Cfg::NT, TB = Cfg::TB, KB = Cfg::KB;
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x;
  const int nkb = g.K / KB;
  const int k0 = (int)(blockIdx.x % nkb) * KB;
  const int64_t t0 = (int64_t)(blockIdx.x / nkb) * TB;
  const int nchunks = (g.C + CC - 1) / CC;

  auto load_chunk = [&](int ch, int buf) {
    const int c0 = ch * CC;
    float* us = sm + buf * SC::STAGE;
    float* vs = us + F * Cfg::UPL;
    constexpr int NU4 = F * CC * (TB / 4);
    for (int e = tid; e < NU4; e += NT) {
      const int q = e % (TB / 4);
      const int cc = (e / (TB / 4)) % CC;
      const int f = e / ((TB / 4) * CC);
      const int c = c0 + cc;
      const bool ok = c < g.C && t0 + 4 * q < Tp;
      const float* src = ok ? U + ((int64_t)f * g.C + c) * Tp + t0 + 4 * q : U;
      cp_async16(smem_u32(us + f * Cfg::UPL + cc * TB + 4 * q), src, ok);
    }
    constexpr int NV4 = F * CC * (KB / 4);
    for (int e = tid; e < NV4; e += NT) {
      const int q = e % (KB / 4);
      const int cc = (e / (KB / 4)) % CC;
      const int f = e / ((KB / 4) * CC);
      const int c = c0 + cc;
      const bool ok = c < g.C;
      const float* src = ok ? V + ((int64_t)f * g.C + c) * g.K + k0 + 4 * q : V;
      cp_async16(smem_u32(vs + f * Cfg::VPL + cc * KB + 4 * q), src, ok);
    }
    cp_async_commit();
  };

  const int warp = tid >> 5, lane = tid & 31;
  const int lx = lane / (LT * LK);
  const int lt = (lane / LK) % LT;
  const int lk = lane % LK;
  const int f0 = (warp * LX + lx) * FPL;
  float acc[FPL][MT][MK];
#pragma unroll
  for (int q = 0; q < FPL; ++q)
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int j = 0; j < MK; ++j) acc[q][i][j] = 0.0f;

  load_chunk(0, 0);
  for (int ch = 0; ch < nchunks; ++ch) {
    const int buf = ch & 1;
    if (ch + 1 < nchunks) {
      load_chunk(ch + 1, buf ^ 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    const float* us = sm + buf * SC::STAGE;
    const float* vbase = us + F * Cfg::UPL + lk * 4;
#pragma unroll
    for (int cc = 0; cc < CC; ++cc) {
#pragma unroll
      for (int q = 0; q < FPL; ++q) {
        const float* up = us + (f0 + q) * Cfg::UPL + cc * TB + lt * MT;
        const float* vp = vbase + (f0 + q) * Cfg::VPL + cc * KB;
        float a[MT], b[MK];
#pragma unroll
        for (int i = 0; i < MT; i += 4) {
          const float4 v = *reinterpret_cast<const float4*>(up + i);
          a[i] = v.x;
          a[i + 1] = v.y;
          a[i + 2] = v.z;
          a[i + 3] = v.w;
        }
#pragma unroll
        for (int s4 = 0; s4 < MK / 4; ++s4) {
          const float4 v = *reinterpret_cast<const float4*>(vp + s4 * 4 * LK);
          b[4 * s4] = v.x;
          b[4 * s4 + 1] = v.y;
          b[4 * s4 + 2] = v.z;
          b[4 * s4 + 3] = v.w;
        }
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
          for (int j = 0; j < MK; ++j) acc[q][i][j] = fmaf(a[i], b[j], acc[q][i][j]);
      }
    }
    __syncthreads();
  }

  // epilogue: accumulators to Es[f][k][t], then A^T M A per (t, k)
  float* Es = sm;
  // Es[f][t][k] with rows of KB + 4 floats: the float4 stores of a warp
  // spread evenly over the banks, and the epilogue's reads (k fastest) are
  // conflict-free.
#pragma unroll
  for (int q = 0; q < FPL; ++q)
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int s4 = 0; s4 < MK / 4; ++s4) {
        float* dst = Es + ((size_t)(f0 + q) * TB + lt * MT + i) * Cfg::EKB + s4 * 4 * LK + lk * 4;
        *reinterpret_cast<float4*>(dst) =
            make_float4(acc[q][i][4 * s4], acc[q][i][4 * s4 + 1], acc[q][i][4 * s4 + 2],
                        acc[q][i][4 * s4 + 3]);
      }
  __syncthreads();
  const int tpi = g.th * g.tw;
  for (int p = tid; p < TB * KB; p += NT) {
    const int kl = p % KB, t = p / KB;
    const int64_t tg = t0 + t;
    const int k = k0 + kl;
    if (tg >= g.T || k >= g.K) continue;
    float Mv[F];
#pragma unroll
    for (int q = 0; q < F; ++q) Mv[q] = Es[((size_t)q * TB + t) * Cfg::EKB + kl];
    float Z[MM * A];
#pragma unroll
    for (int a = 0; a < MM; ++a)
#pragma unroll
      for (int j = 0; j < A; ++j) {
        float z = 0.0f;
#pragma unroll
        for (int i = 0; i < A; ++i) z = fmaf(Mx.AT[a * A + i], Mv[i * A + j], z);
        Z[a * A + j] = z;
      }
    const int n = (int)(tg / tpi);
    const int rem = (int)(tg - (int64_t)n * tpi);
    const int ti = rem / g.tw, tj = rem - (rem / g.tw) * g.tw;
    float* yk = y + ((int64_t)n * g.K + k) * g.Ho * g.Wo;
#pragma unroll
    for (int a = 0; a < MM; ++a) {
      const int pr = ti * MM + a;
      float yr[MM];
#pragma unroll
      for (int b = 0; b < MM; ++b) {
        float v = 0.0f;
#pragma unroll
        for (int j = 0; j < A; ++j) v = fmaf(Z[a * A + j], Mx.AT[b * A + j], v);
        yr[b] = v;
      }
      if (pr >= g.Ho) continue;
      float* yrow = yk + (int64_t)pr * g.Wo + tj * MM;
#pragma unroll
      for (int b = 0; b < MM; ++b)
        if (tj * MM + b < g.Wo) yrow[b] = yr[b];
    }
  }
}

template <FUSED_TPARAMS>
static int launch_split(const float* x, const float* V, float* U, float* y, const LayerGeom& g,
                        const LayerMats& M, cudaStream_t st) {
  using Cfg = FusedCfg<FUSED_TARGS>;
  using SC = SplitCfg<FUSED_TARGS>;
  if (g.K % Cfg::KB != 0) return kFallback;
  const int64_t Tp = (g.T + 3) & ~(int64_t)3;
  static bool attr_set[16] = {false};
  int dev = 0;
  WINO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 16 && !attr_set[dev]) {
    WINO_CUDA_TRY(cudaFuncSetAttribute(k_gemm_otx<FUSED_TARGS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SC::SMEM));
    attr_set[dev] = true;
  }
  const int64_t nblk = (int64_t)(g.K / Cfg::KB) * ((g.T + Cfg::TB - 1) / Cfg::TB);
  const int64_t nin = (int64_t)g.C * Tp;
  if (nblk > 0x7fffffffLL || (nin + 255) / 256 > 0x7fffffffLL) return kFallback;
  {
    ProfScope ps(kKInput, st);
    k_input_transform_r3<MM><<<(unsigned)((nin + 255) / 256), 256, 0, st>>>(x, U, g, M, Tp);
  }
  {
    ProfScope ps(kKFused, st);
    k_gemm_otx<FUSED_TARGS><<<(unsigned)nblk, Cfg::NT, SC::SMEM, st>>>(U, V, y, g, M, Tp);
  }
  note_launches(2);
  WINO_CUDA_TRY(cudaGetLastError());
  return WINO_OK;
}

size_t split_workspace_bytes(const LayerGeom& g) {
  const int64_t Tp = (g.T + 3) & ~(int64_t)3;
  return (size_t)g.F * g.C * g.K * sizeof(float) + (size_t)g.F * g.C * Tp * sizeof(float) + 256;
}

// Two-kernel variant (needs V and U in the workspace).
int layer_forward_split(const float* x, const float* w, float* y, const LayerGeom& g,
                        const LayerMats& M, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (g.dim != 2 || M.r != 3 || (M.m != 2 && M.m != 4 && M.m != 6) || g.K % 64 != 0)
    return kFallback;
  if (ws_bytes < split_workspace_bytes(g)) return kFallback;
  float* V = (float*)ws;
  float* U = V + (((size_t)g.F * g.C * g.K + 63) & ~(size_t)63);
  {
    const int64_t n = (int64_t)g.C * g.K;
    ProfScope ps(kKFilter, st);
    k_filter_transform<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, V, g.dim, g.C, g.K, M);
    note_launches(1);
  }
  switch (M.m) {
    case 2:
      return launch_split<2, 2, 4, 4, 1, 8, 16, 8>(x, V, U, y, g, M, st);
    case 4:
      return launch_split<4, 1, 4, 8, 3, 4, 8, 8>(x, V, U, y, g, M, st);
    default:
      return launch_split<6, 8, 1, 4, 1, 8, 16, 4>(x, V, U, y, g, M, st);
  }
}

}  // namespace wino
