// fused.cu -- fused FP32 Winograd layer F(m x m, 3 x 3), m in {2, 4, 6}.
//
// Three forms of the layer, bit-identical to one another and to the general
// path in layer.cu (the layer autotuner there picks one per shape):
//   - k_fused_layer (below): input transform, contraction and output
//     transform in one kernel;
//   - the split variant: k_input_transform_blk writes U once in a blocked
//     layout, k_gemm_otx contracts and fuses the output transform;
//   - its cluster form, k_gemm_otx_cl: a tile block's alpha^2 frequencies
//     spread over the CTAs of a thread-block cluster.
//
// k_fused_layer: one CTA owns TB consecutive tiles x KB output channels and ALL alpha^2
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
#include "async_copy.cuh"
#include "common.cuh"
#include "packed.cuh"
#include "patch.cuh"

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
  static_assert(F % (LX * FPL) == 0, "whole warps");
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
  // acc[q][i][j2] holds output channels (2 j2, 2 j2 + 1) of tile i
  unsigned long long acc[FPL][MT][MK / 2];
#pragma unroll
  for (int q = 0; q < FPL; ++q)
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int j = 0; j < MK / 2; ++j) acc[q][i][j] = 0ull;

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
        float a[MT];
        unsigned long long b2[MK / 2];  // channel pairs
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
          const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(vp + s4 * 4 * LK);
          b2[2 * s4] = v.x;
          b2[2 * s4 + 1] = v.y;
        }
#pragma unroll
        for (int i = 0; i < MT; ++i) {
          const unsigned long long ai = pack_dup(a[i]);
#pragma unroll
          for (int j = 0; j < MK / 2; ++j) acc[q][i][j] = fma2(ai, b2[j], acc[q][i][j]);
        }
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
        const float2 lo = unpack2(acc[q][i][2 * s4]), hi = unpack2(acc[q][i][2 * s4 + 1]);
        *reinterpret_cast<float4*>(dst) = make_float4(lo.x, lo.y, hi.x, hi.y);
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
// transform fused into its epilogue (M never leaves the SM).
//
// U and V are written in a blocked layout, so that everything one CTA needs
// for one chunk of CC input channels is ONE contiguous run per operand:
//   Ub[tile block][chunk][f][UPL]   UPL = CC TB + 4 (row cc at cc TB)
//   Vb[k block][chunk][f][VPL]      VPL = CC KB + 16 (row cc at cc KB)
// (channels past C are zero; the padding words are never read).  The GEMM
// kernel streams chunks with two bulk copies (cp.async.bulk, the TMA's 1D
// form) per chunk into an NS-stage ring of shared-memory stages whose
// mbarriers count the bytes: no per-thread copy instructions, and NS - 1
// chunks in flight.  The inner product order is that of the fused kernel
// (c ascending, fused multiply-add), bit for bit.
// ===========================================================================

namespace {

// The give-up path of the layer kernels' bounded waits (mbar_wait_bounded),
// run on purpose: one warp waits on an mbarrier that nothing arrives at,
// gives up after `polls` polls, sets the device's wait-error flag as a layer
// kernel would and returns; ns[0] = the device time the polls took.
__global__ void k_wait_probe(int polls, int* err, long long* ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init1((uint32_t)__cvta_generic_to_shared(&bar));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  long long t0, t1;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t0));
  const bool got = mbar_wait_bounded((uint32_t)__cvta_generic_to_shared(&bar), 0u, polls);
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t1));
  if (threadIdx.x == 0) {
    if (!got) atomicExch(err, 1);
    ns[0] = t1 - t0;
  }
}

}  // namespace

int wait_probe(int polls, long long* elapsed_ns, cudaStream_t st) {
  int* err = nullptr;
  int rc = wait_error_flag(&err);
  if (rc != WINO_OK) return rc;
  long long* d_ns = nullptr;
  WINO_CUDA_TRY(cudaMalloc(&d_ns, sizeof(long long)));
  k_wait_probe<<<1, 32, 0, st>>>(polls, err, d_ns);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(elapsed_ns, d_ns, sizeof(long long), cudaMemcpyDeviceToHost);
  (void)cudaFree(d_ns);
  WINO_CUDA_TRY(e);
  return WINO_OK;
}

// Blocked layout geometry of one split tile shape.
struct SplitGeom {
  int TB, KB, CC, UPL, VPL, nch, ntb, nkb;
  int64_t ub_floats() const { return (int64_t)ntb * nch * F_ * UPL; }
  int64_t vb_floats() const { return (int64_t)nkb * nch * F_ * VPL; }
  int F_;
};

static SplitGeom split_geom(const LayerGeom& g, int TB, int KB, int CC) {
  SplitGeom s;
  s.TB = TB;
  s.KB = KB;
  s.CC = CC;
  s.UPL = CC * TB + 4;
  s.VPL = CC * KB + 16;
  s.nch = (g.C + CC - 1) / CC;
  s.ntb = (int)((g.T + TB - 1) / TB);
  s.nkb = g.K / KB;
  s.F_ = g.F;
  return s;
}

// Input transform into Ub: one CTA per (tile block, chunk), one thread per
// (channel, tile) of it (tiles fastest: with padding 1 and W even a lane
// loads its patch's interior columns as vectors and takes the halo columns
// from the neighbouring lanes, patch.cuh; otherwise neighbouring tiles
// share input rows in L1).  The chunk's F x UPL floats are staged in shared memory and leave
// as one contiguous run of 16-byte stores (the chunk's rows are UPL floats
// apart, not a multiple of the 128-byte line, so per-row stores would split
// lines).  (Unpadded planes for the cluster shapes, UPL = CC TB, stored
// straight from registers as whole lines, measured the same layer times.)
// Launch: grid (ntb, nch), blockDim = CC x TB, dynamic shared memory
// F x UPL floats.
template <int MM>
__global__ void __launch_bounds__(256) k_input_transform_blk(const float* __restrict__ x,
                                                             float* __restrict__ Ub,
                                                             const LayerGeom g,
                                                             const LayerMats Mx,
                                                             const SplitGeom sg) {
  constexpr int A = MM + 2, F = A * A;
  extern __shared__ __align__(16) float cs[];  // [F][UPL]
  const int tb = blockIdx.x, ch = blockIdx.y;
  const int tl = threadIdx.x % sg.TB, cc = threadIdx.x / sg.TB;
  const int64_t t = (int64_t)tb * sg.TB + tl;
  const int c = ch * sg.CC + cc;
  float d[A][A];
  const bool live = t < g.T && c < g.C;
  if (patch_rowvec_ok(x, g) && (blockDim.x & 31) == 0) {
    // a lane's neighbours hold tiles t -+ 1 of channel c unless it is at
    // an end of the warp or of the block's tile range
    const int lane = threadIdx.x & 31;
    load_patch_rowvec<MM>(x, g, t, c, live, lane == 0 || tl == 0,
                          lane == 31 || tl == sg.TB - 1, d);
  } else if (live) {
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
  float* row = cs + cc * sg.TB + tl;
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
#pragma unroll
      for (int l = 0; l < A; ++l) acc = fmaf(tm[i][l], Mx.BT[j * A + l], acc);
      row[(i * A + j) * sg.UPL] = live ? acc : 0.0f;
    }
  __syncthreads();
  // the chunk, padding words included, as 16-byte stores (F UPL is a
  // multiple of 4 floats and the chunk starts 16-byte aligned)
  const int n4 = F * sg.UPL / 4;
  float4* dst = reinterpret_cast<float4*>(Ub + ((int64_t)tb * sg.nch + ch) * F * sg.UPL);
  const float4* src = reinterpret_cast<const float4*>(cs);
  for (int e = threadIdx.x; e < n4; e += blockDim.x) dst[e] = src[e];
}

// Filter transform into Vb.  One CTA per 32 output channels x 32 input
// channels (of the padded range): the 32 x 32 kernels are staged in shared
// memory first -- for each output channel its 32 input channels' taps are
// 288 contiguous floats of w, read coalesced -- with rows padded to 289
// floats, so that the compute pass, one thread per (input, output channel)
// with output channels across the lanes, reads them without bank conflicts
// and writes each frequency's 32 outputs as one contiguous run of Vb.
// (Reading w straight from global memory with output channels across the
// lanes touched 32 lines per load.)  Launch: grid (ceil(K / 32),
// ceil(nch CC / 32)), 256 threads.
constexpr int kFtK = 32, kFtC = 32, kFtRow = kFtC * 9 + 1;
template <int MM>
__global__ void __launch_bounds__(256) k_filter_transform_blk(const float* __restrict__ w,
                                                              float* __restrict__ Vb, int C,
                                                              int K, const LayerMats M,
                                                              const SplitGeom sg) {
  constexpr int F = (MM + 2) * (MM + 2);
  __shared__ float ws[kFtK * kFtRow];
  const int k0 = blockIdx.x * kFtK, c0 = blockIdx.y * kFtC;
  const int cpad = sg.nch * sg.CC;
  for (int e = threadIdx.x; e < kFtK * kFtC * 9; e += blockDim.x) {
    const int kk = e / (kFtC * 9), r = e - kk * (kFtC * 9);
    const int k = k0 + kk, c = c0 + r / 9;
    ws[kk * kFtRow + r] = (k < K && c < C) ? __ldg(w + ((int64_t)k * C + c0) * 9 + r) : 0.0f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kFtK * kFtC; e += blockDim.x) {
    const int kk = e % kFtK, cl = e / kFtK;
    const int k = k0 + kk, c = c0 + cl;
    if (k >= K || c >= cpad) continue;
    const int kb = k / sg.KB, kl = k - kb * sg.KB;
    const int ch = c / sg.CC, cc = c - ch * sg.CC;
    float* out = Vb + ((int64_t)kb * sg.nch + ch) * F * sg.VPL + cc * sg.KB + kl;
    float v[F];
    if (c < C) {
      filter_fixed<MM>(ws + kk * kFtRow + cl * 9, M, v);
    } else {
#pragma unroll
      for (int f = 0; f < F; ++f) v[f] = 0.0f;
    }
#pragma unroll
    for (int f = 0; f < F; ++f) out[(int64_t)f * sg.VPL] = v[f];
  }
}

// NS stages of (U chunk, V chunk) in shared memory; MINB CTAs per SM.
template <FUSED_TPARAMS, int NS, int MINB>
struct SplitCfg {
  using Base = FusedCfg<FUSED_TARGS>;
  static constexpr int SU = Base::F * Base::UPL;  // U chunk (floats)
  static constexpr int SV = Base::F * Base::VPL;  // V chunk (floats)
  static constexpr int STAGE = SU + SV;
  static constexpr int MAIN_FL = NS * STAGE;
  static constexpr int ETB = Base::TB + 4;                  // epilogue row: TB tiles (padded)
  static constexpr int EPI_FL = Base::F * Base::KB * ETB;   // Es[f][k][t]
  static constexpr int SMEM_FL = MAIN_FL > EPI_FL ? MAIN_FL : EPI_FL;
  static constexpr size_t SMEM = (size_t)SMEM_FL * sizeof(float);
  static_assert(NS >= 2, "at least double buffering");
  static_assert((SU * 4) % 16 == 0 && (SV * 4) % 16 == 0, "bulk copies move 16-byte multiples");
};

#define SPLIT_TPARAMS FUSED_TPARAMS, int NS, int MINB
#define SPLIT_TARGS FUSED_TARGS, NS, MINB

// Output coordinates of tile t for an epilogue: ybase = offset of
// y[n][0][ti m][tj m], rows / cols = the tile's valid output rows and
// columns (all 0 for t past the last tile).
template <int MM>
__device__ __forceinline__ void tile_out_coords(const LayerGeom& g, int64_t t, int64_t& ybase,
                                                int& rows, int& cols) {
  if (t < g.T) {
    const int tpi = g.th * g.tw;
    const int n = (int)(t / tpi);
    const int rem = (int)(t - (int64_t)n * tpi);
    const int ti = rem / g.tw, tj = rem - (rem / g.tw) * g.tw;
    ybase = (int64_t)n * g.K * g.Ho * g.Wo + (int64_t)ti * MM * g.Wo + tj * MM;
    rows = min(MM, g.Ho - ti * MM);
    cols = min(MM, g.Wo - tj * MM);
  } else {
    ybase = 0;
    rows = 0;
    cols = 0;
  }
}

// Output transform Y = A^T M A of one (tile, output channel): M[q] (q = i A
// + j, frequencies row-major) from `ld(q)`, Y's valid rows x cols written
// to y_t (row stride Wo).  Z = A^T M, then Y = Z A, sums over i and j
// ascending; the pairs (j, j + 1) of Z and (b, b + 1) of Y run as one
// fma.rn.f32x2 each (two IEEE fused multiply-adds, the same bits).
template <int MM, typename LdM>
__device__ __forceinline__ void otx_tile(LdM ld, const LayerMats& Mx, float* yt, int rows,
                                         int cols, int Wo) {
  constexpr int A = MM + 2, F = A * A;
  unsigned long long Mp[F / 2];  // (M[i][j], M[i][j + 1]), j even
#pragma unroll
  for (int q = 0; q < F; q += 2) Mp[q / 2] = pack2(ld(q), ld(q + 1));
  float Z[MM * A];
#pragma unroll
  for (int a = 0; a < MM; ++a)
#pragma unroll
    for (int j = 0; j < A; j += 2) {
      unsigned long long z = 0ull;
#pragma unroll
      for (int i = 0; i < A; ++i) z = fma2(pack_dup(Mx.AT[a * A + i]), Mp[(i * A + j) / 2], z);
      const float2 zz = unpack2(z);
      Z[a * A + j] = zz.x;
      Z[a * A + j + 1] = zz.y;
    }
#pragma unroll
  for (int a = 0; a < MM; ++a) {
    float yr[MM];
#pragma unroll
    for (int b = 0; b < MM; b += 2) {
      unsigned long long v = 0ull;
#pragma unroll
      for (int j = 0; j < A; ++j)
        v = fma2(pack_dup(Z[a * A + j]), pack2(Mx.AT[b * A + j], Mx.AT[(b + 1) * A + j]), v);
      const float2 vv = unpack2(v);
      yr[b] = vv.x;
      yr[b + 1] = vv.y;
    }
    if (a >= rows) continue;
    float* yrow = yt + (int64_t)a * Wo;
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

template <SPLIT_TPARAMS>
__global__ void __launch_bounds__(FusedCfg<FUSED_TARGS>::NT, MINB)
    k_gemm_otx(const float* __restrict__ Ub, const float* __restrict__ Vb, float* __restrict__ y,
               const LayerGeom g, const LayerMats Mx, const SplitGeom sg, int* err) {
  using Cfg = FusedCfg<FUSED_TARGS>;
  using SC = SplitCfg<SPLIT_TARGS>;
  constexpr int NT = Cfg::NT, TB = Cfg::TB, KB = Cfg::KB;
  extern __shared__ __align__(128) float gsm_[];
  float* sm = gsm_;
  __shared__ __align__(8) uint64_t full[NS];
  const int tid = threadIdx.x;
  const int nkb = g.K / KB;
  const int kb = (int)(blockIdx.x % nkb);
  const int tb = (int)(blockIdx.x / nkb);
  const int k0 = kb * KB;
  const int64_t t0 = (int64_t)tb * TB;
  const int nchunks = sg.nch;
  const float* ublk = Ub + (int64_t)tb * nchunks * SC::SU;
  const float* vblk = Vb + (int64_t)kb * nchunks * SC::SV;

  // per-tile output coordinates for the epilogue, computed once
  __shared__ int64_t s_ybase[TB];  // offset of y[n][0][ti m][tj m]
  __shared__ int s_rows[TB], s_cols[TB];  // valid output rows / columns (0: no tile)
  if (tid < TB) tile_out_coords<MM>(g, t0 + tid, s_ybase[tid], s_rows[tid], s_cols[tid]);
  if (tid == 0) {
#pragma unroll
    for (int st = 0; st < NS; ++st) mbar_init1((uint32_t)__cvta_generic_to_shared(&full[st]));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // thread 0 refills stage `st` with chunk `ch`
  auto issue = [&](int ch, int st) {
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&full[st]);
    const uint32_t dst = smem_u32(sm + st * SC::STAGE);
    mbar_expect_tx(bar, (uint32_t)(SC::STAGE * 4));
    bulk_g2s(dst, ublk + (int64_t)ch * SC::SU, (uint32_t)(SC::SU * 4), bar);
    bulk_g2s(dst + SC::SU * 4, vblk + (int64_t)ch * SC::SV, (uint32_t)(SC::SV * 4), bar);
  };
  // chunks [0, issued) are in flight or landed
  int issued = nchunks < NS - 1 ? nchunks : NS - 1;
  if (tid == 0) {
    for (int st = 0; st < issued; ++st) issue(st, st);
  }

  const int warp = tid >> 5, lane = tid & 31;
  const int lx = lane / (LT * LK);
  const int lt = (lane / LK) % LT;
  const int lk = lane % LK;
  const int f0 = (warp * LX + lx) * FPL;
  // acc[q][i][j2] holds output channels (2 j2, 2 j2 + 1) of tile i
  unsigned long long acc[FPL][MT][MK / 2];
#pragma unroll
  for (int q = 0; q < FPL; ++q)
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int j = 0; j < MK / 2; ++j) acc[q][i][j] = 0ull;

  bool ok = true;
  for (int ch = 0; ch < nchunks; ++ch) {
    const int st = ch % NS;
    const bool got =
        mbar_wait_bounded((uint32_t)__cvta_generic_to_shared(&full[st]), (uint32_t)((ch / NS) & 1));
    // chunk ch landed for everyone (or someone gave up); every thread is done
    // with chunk ch - 1, whose stage the refill below overwrites
    ok = __syncthreads_and(got ? 1 : 0) != 0;
    if (!ok) {
      // drain the copies still in flight (bounded), then abandon the tile
      if (tid == 0) {
        atomicExch(err, 1);
        for (int c2 = ch; c2 < issued; ++c2)
          (void)mbar_wait_bounded((uint32_t)__cvta_generic_to_shared(&full[c2 % NS]),
                                  (uint32_t)((c2 / NS) & 1));
      }
      return;
    }
    if (ch + NS - 1 < nchunks) {
      if (tid == 0) {
        // the stage's previous contents were read through the generic proxy
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        issue(ch + NS - 1, (ch + NS - 1) % NS);
      }
      ++issued;
    }
    const float* us = sm + st * SC::STAGE;
    const float* vbase = us + SC::SU + lk * 4;
    // operand fragments of step (cc, q); the next step's are loaded before
    // this step's FMAs are issued
    auto load_frag = [&](int cc, int q, float (&a)[MT], unsigned long long (&b2)[MK / 2]) {
      const float* up = us + (f0 + q) * Cfg::UPL + cc * TB + lt * MT;
      const float* vp = vbase + (f0 + q) * Cfg::VPL + cc * KB;
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
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(vp + s4 * 4 * LK);
        b2[2 * s4] = v.x;
        b2[2 * s4 + 1] = v.y;
      }
    };
    float a[2][MT];
    unsigned long long b2[2][MK / 2];
    load_frag(0, 0, a[0], b2[0]);
#pragma unroll
    for (int step = 0; step < CC * FPL; ++step) {
      const int cur = step & 1;
      if (step + 1 < CC * FPL)
        load_frag((step + 1) / FPL, (step + 1) % FPL, a[cur ^ 1], b2[cur ^ 1]);
      const int q = step % FPL;
#pragma unroll
      for (int i = 0; i < MT; ++i) {
        const unsigned long long ai = pack_dup(a[cur][i]);
#pragma unroll
        for (int j = 0; j < MK / 2; ++j) acc[q][i][j] = fma2(ai, b2[cur][j], acc[q][i][j]);
      }
    }
  }
  __syncthreads();  // every thread done with the stages the epilogue reuses

  // epilogue: accumulators to Es[f][k][t] (rows of TB + 4 floats, tiles
  // contiguous), then A^T M A per (t, k) with consecutive lanes on
  // consecutive tiles of one output channel, so that a warp's output rows
  // land in adjacent 16-byte segments of y.
  constexpr int ETB = SC::ETB;
  float* Es = sm;
#pragma unroll
  for (int q = 0; q < FPL; ++q)
#pragma unroll
    for (int s4 = 0; s4 < MK / 4; ++s4)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int kl = s4 * 4 * LK + lk * 4 + jj;
        float* dst = Es + ((size_t)(f0 + q) * KB + kl) * ETB + lt * MT;
#pragma unroll
        for (int i = 0; i < MT; i += 4) {
          float v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 pr = unpack2(acc[q][i + u][2 * s4 + jj / 2]);
            v[u] = (jj & 1) ? pr.y : pr.x;
          }
          *reinterpret_cast<float4*>(dst + i) = make_float4(v[0], v[1], v[2], v[3]);
        }
      }
  __syncthreads();
  // A^T M A per (t, k), the same order as the fused kernel's epilogue
  const int64_t plane = (int64_t)g.Ho * g.Wo;
  for (int p = tid; p < TB * KB; p += NT) {
    const int t = p % TB, kl = p / TB;
    const int rows = s_rows[t];
    if (rows == 0) continue;
    otx_tile<MM>([&](int q) { return Es[((size_t)q * KB + kl) * ETB + t]; }, Mx,
                 y + s_ybase[t] + (int64_t)(k0 + kl) * plane, rows, s_cols[t], g.Wo);
  }
}

// ===========================================================================
// Cluster form of the GEMM + output-transform kernel.  The alpha^2
// frequencies of a (TB tiles x KB output channels) block are split over a
// cluster of NCL CTAs, FC = alpha^2 / NCL each.  A CTA holds the
// accumulators of its FC frequencies only, which leaves registers for 8 x 8
// outputs per thread: 16 operand floats per 64 FMAs, the ratio at which
// the shared-memory operand path (one float per lane per 4 FMA lanes of the
// SM) keeps the FMA pipe busy.  Each CTA streams its frequencies' slice of
// every chunk (one contiguous run of the blocked U and V layouts, so the
// transform kernels are shared with the single-CTA form) and stores its
// accumulators to its own shared memory; after a cluster barrier the CTAs
// split the block's (tile, channel) pairs and read the other frequencies
// from their peers' shared memory (distributed shared memory).  Inner
// products (c ascending, fused multiply-add) and output transform are those
// of the single-CTA form, bit for bit.
// ===========================================================================
template <int MM, int NCL, int LX, int LT, int LK, int MT, int MK, int CC, int NS, int MINB>
struct ClCfg {
  static constexpr int A = MM + 2, F = A * A, FC = F / NCL;
  static constexpr int TB = LT * MT, KB = LK * MK;
  static constexpr int NW = FC / LX, NT = NW * 32;
  static constexpr int UPL = CC * TB + 4, VPL = CC * KB + 16;  // the blocked layouts' planes
  static constexpr int SU = FC * UPL, SV = FC * VPL, STAGE = SU + SV;
  static constexpr int MAIN_FL = NS * STAGE;
  static constexpr int ETB = TB + 4;               // epilogue row: TB tiles (padded)
  static constexpr int EPI_FL = FC * KB * ETB;     // Es[fl][k][t]
  static constexpr int SMEM_FL = MAIN_FL > EPI_FL ? MAIN_FL : EPI_FL;
  static constexpr size_t SMEM = (size_t)SMEM_FL * sizeof(float);
  static_assert(F % NCL == 0 && FC % LX == 0, "whole frequency slices and warps");
  static_assert(LX * LT * LK == 32, "a warp is 32 lanes");
  static_assert(MT % 4 == 0 && MK % 4 == 0, "float4 operand loads");
  static_assert(NS >= 2 && NCL >= 2 && NCL <= 8, "double buffering; portable cluster size");
  static_assert((SU * 4) % 16 == 0 && (SV * 4) % 16 == 0 && (UPL * 4) % 16 == 0 &&
                    (VPL * 4) % 16 == 0,
                "bulk copies move 16-byte multiples from 16-byte boundaries");
};

#define CL_TPARAMS int MM, int NCL, int LX, int LT, int LK, int MT, int MK, int CC, int NS, int MINB
#define CL_TARGS MM, NCL, LX, LT, LK, MT, MK, CC, NS, MINB

namespace {
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// The address of shared-memory word `a` (this CTA's) in CTA `rank` of the
// cluster.
__device__ __forceinline__ uint32_t cluster_map(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ float ld_dsmem(uint32_t a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];\n" : "=f"(v) : "r"(a) : "memory");
  return v;
}
}  // namespace

// Launch: grid NCL x (K / KB) x ceil(T / TB) CTAs (cluster NCL x 1 x 1, the
// NCL CTAs of one block adjacent), NT threads, ClCfg::SMEM bytes of dynamic
// shared memory.
template <CL_TPARAMS>
__global__ void __cluster_dims__(NCL, 1, 1) __launch_bounds__(ClCfg<CL_TARGS>::NT, MINB)
    k_gemm_otx_cl(const float* __restrict__ Ub, const float* __restrict__ Vb,
                  float* __restrict__ y, const LayerGeom g, const LayerMats Mx,
                  const SplitGeom sg, int* err) {
  using Cfg = ClCfg<CL_TARGS>;
  constexpr int F = Cfg::F, FC = Cfg::FC, NT = Cfg::NT, TB = Cfg::TB, KB = Cfg::KB;
  constexpr int ETB = Cfg::ETB;
  extern __shared__ __align__(128) float csm_[];
  float* sm = csm_;
  __shared__ __align__(8) uint64_t full[NS];
  __shared__ uint32_t s_done[NS];  // warps done with stage s, counted over its chunks
  __shared__ int s_issued;         // chunks 0 .. s_issued - 1 issued
  __shared__ int64_t s_ybase[TB];
  __shared__ int s_rows[TB], s_cols[TB];
  const int tid = threadIdx.x;
  uint32_t rank;
  asm("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(rank));
  const int64_t blk = blockIdx.x / NCL;
  const int nkb = g.K / KB;
  const int kb = (int)(blk % nkb);
  const int64_t tb = blk / nkb;
  const int k0 = kb * KB;
  const int64_t t0 = tb * TB;
  const int nchunks = sg.nch;
  // chunk ch of this CTA's frequency slice at ublk + ch F UPL (vblk alike)
  const float* ublk = Ub + tb * nchunks * F * Cfg::UPL + (int64_t)rank * Cfg::SU;
  const float* vblk = Vb + (int64_t)kb * nchunks * F * Cfg::VPL + (int64_t)rank * Cfg::SV;

  if (tid < TB) tile_out_coords<MM>(g, t0 + tid, s_ybase[tid], s_rows[tid], s_cols[tid]);
  auto issue = [&](int ch, int st) {
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&full[st]);
    const uint32_t dst = smem_u32(sm + st * Cfg::STAGE);
    mbar_expect_tx(bar, (uint32_t)(Cfg::STAGE * 4));
    bulk_g2s(dst, ublk + (int64_t)ch * F * Cfg::UPL, (uint32_t)(Cfg::SU * 4), bar);
    bulk_g2s(dst + Cfg::SU * 4, vblk + (int64_t)ch * F * Cfg::VPL, (uint32_t)(Cfg::SV * 4), bar);
  };
  // every stage starts filled: chunks 0 .. NS - 1 in flight
  if (tid == 0) {
#pragma unroll
    for (int st = 0; st < NS; ++st) {
      mbar_init1((uint32_t)__cvta_generic_to_shared(&full[st]));
      s_done[st] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    const int n0 = nchunks < NS ? nchunks : NS;
    for (int st = 0; st < n0; ++st) issue(st, st);
    s_issued = n0;
  }
  __syncthreads();

  const int warp = tid >> 5, lane = tid & 31;
  const int lx = lane / (LT * LK);
  const int lt = (lane / LK) % LT;
  const int lk = lane % LK;
  const int fl = warp * LX + lx;  // this lane's frequency within the slice
  // acc[i][j2] holds output channels (2 j2, 2 j2 + 1) of tile i
  unsigned long long acc[MT][MK / 2];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < MK / 2; ++j) acc[i][j] = 0ull;

  // No CTA-wide barrier per chunk: each warp waits for the chunk's bytes
  // and, when done with it, counts itself out of the stage; the last warp
  // out refills the stage with chunk ch + NS.
  bool ok = true;
  for (int ch = 0; ch < nchunks; ++ch) {
    const int st = ch % NS;
    const bool got =
        mbar_wait_bounded((uint32_t)__cvta_generic_to_shared(&full[st]), (uint32_t)((ch / NS) & 1));
    if (!__all_sync(0xffffffffu, got)) {
      ok = false;  // the warp leaves the loop; its peers' waits run out in turn
      break;
    }
    const float* up0 = sm + st * Cfg::STAGE + fl * Cfg::UPL + lt * MT;
    const float* vp0 = sm + st * Cfg::STAGE + Cfg::SU + fl * Cfg::VPL + lk * 4;
    auto load_frag = [&](int cc, float (&a)[MT], unsigned long long (&b2)[MK / 2]) {
      const float* up = up0 + cc * TB;
      const float* vp = vp0 + cc * KB;
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
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(vp + s4 * 4 * LK);
        b2[2 * s4] = v.x;
        b2[2 * s4 + 1] = v.y;
      }
    };
    float a[2][MT];
    unsigned long long b2[2][MK / 2];
    load_frag(0, a[0], b2[0]);
#pragma unroll
    for (int cc = 0; cc < CC; ++cc) {
      const int cur = cc & 1;
      if (cc + 1 < CC) load_frag(cc + 1, a[cur ^ 1], b2[cur ^ 1]);
#pragma unroll
      for (int i = 0; i < MT; ++i) {
        const unsigned long long ai = pack_dup(a[cur][i]);
#pragma unroll
        for (int j = 0; j < MK / 2; ++j) acc[i][j] = fma2(ai, b2[cur][j], acc[i][j]);
      }
    }
    // every lane's reads of the stage are done (their values are in the
    // accumulators); lane 0 counts the warp out with release semantics, and
    // the warp that completes the count acquires the others' releases,
    // orders them before the async proxy's writes and refills the stage
    __syncwarp();
    if (lane == 0) {
      uint32_t prev;
      asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;\n"
                   : "=r"(prev)
                   : "r"((uint32_t)__cvta_generic_to_shared(&s_done[st]))
                   : "memory");
      if (prev + 1 == (uint32_t)(Cfg::NW * (ch / NS + 1)) && ch + NS < nchunks) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        issue(ch + NS, st);
        atomicMax(&s_issued, ch + NS + 1);
      }
    }
  }
  // every thread done with the stages the epilogue reuses
  const bool cta_ok = __syncthreads_and(ok ? 1 : 0) != 0;
  if (!cta_ok && tid == 0) {
    // a wait gave up: wait (bounded) for the copies that may still be in
    // flight -- at most the last chunk issued to each stage -- before the
    // shared memory is given up; the CTA still takes part in the cluster
    // barriers below, so that no peer waits forever
    atomicExch(err, 1);
    const int iss = s_issued;
    for (int s2 = 0; s2 < NS && s2 < iss; ++s2) {
      const int c_last = s2 + ((iss - 1 - s2) / NS) * NS;
      (void)mbar_wait_bounded((uint32_t)__cvta_generic_to_shared(&full[s2]),
                              (uint32_t)((c_last / NS) & 1));
    }
  }

  float* Es = sm;
  if (cta_ok) {
#pragma unroll
    for (int s4 = 0; s4 < MK / 4; ++s4)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int kl = s4 * 4 * LK + lk * 4 + jj;
        float* dst = Es + ((size_t)fl * KB + kl) * ETB + lt * MT;
#pragma unroll
        for (int i = 0; i < MT; i += 4) {
          float v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 pr = unpack2(acc[i + u][2 * s4 + jj / 2]);
            v[u] = (jj & 1) ? pr.y : pr.x;
          }
          *reinterpret_cast<float4*>(dst + i) = make_float4(v[0], v[1], v[2], v[3]);
        }
      }
  }
  // every CTA's accumulators are in its shared memory
  cluster_sync_all();
  if (cta_ok) {
    uint32_t es[NCL];  // Es of each CTA of the cluster
#pragma unroll
    for (int r = 0; r < NCL; ++r) es[r] = cluster_map(smem_u32(Es), (uint32_t)r);
    const int64_t plane = (int64_t)g.Ho * g.Wo;
    const int p_lo = (int)((int64_t)TB * KB * rank / NCL);
    const int p_hi = (int)((int64_t)TB * KB * (rank + 1) / NCL);
    for (int p = p_lo + tid; p < p_hi; p += NT) {
      const int t = p % TB, kl = p / TB;
      const int rows = s_rows[t];
      if (rows == 0) continue;
      otx_tile<MM>(
          [&](int q) {
            return ld_dsmem(es[q / FC] + (uint32_t)((((q % FC) * KB + kl) * ETB + t) * 4));
          },
          Mx, y + s_ybase[t] + (int64_t)(k0 + kl) * plane, rows, s_cols[t], g.Wo);
    }
  }
  // no CTA leaves while a peer may still read its shared memory.  Relaxed:
  // the values of every peer read were consumed before its thread arrives,
  // and the output stores need no ordering here (a release would wait for
  // them).
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory");
}

// Blocked workspace of a tile shape: Vb, then Ub (256-byte aligned).
static size_t split_ws_bytes(const SplitGeom& sg) {
  const size_t v = ((size_t)sg.vb_floats() * 4 + 255) & ~(size_t)255;
  return v + (size_t)sg.ub_floats() * 4 + 256;
}

template <SPLIT_TPARAMS>
static size_t split_ws_for(const LayerGeom& g) {
  using Cfg = FusedCfg<FUSED_TARGS>;
  if (g.K % Cfg::KB != 0) return 0;
  return split_ws_bytes(split_geom(g, Cfg::TB, Cfg::KB, CC));
}

// Filter and input transforms into the blocked layouts of `sg`; false when
// a launch dimension would overflow.
template <int MM>
static bool launch_split_transforms(const float* x, const float* w, const LayerGeom& g,
                                    const LayerMats& M, const SplitGeom& sg, float* Ub, float* Vb,
                                    cudaStream_t st) {
  const int fy = (sg.nch * sg.CC + kFtC - 1) / kFtC;
  const size_t csm = (size_t)g.F * sg.UPL * sizeof(float);
  constexpr int kMaxCsm = 96 * 1024;
  if (sg.nch > 65535 || fy > 65535 || csm > (size_t)kMaxCsm) return false;
  static bool attr_set[16] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (dev < 16 && !attr_set[dev]) {
    if (cudaFuncSetAttribute(k_input_transform_blk<MM>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxCsm) != cudaSuccess)
      return false;
    attr_set[dev] = true;
  }
  // the filter transform does not depend on x: it runs on the side stream,
  // beside the input transform, and the caller's stream waits for it
  // before the contraction
  cudaStream_t aux = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  if (side_stream(&aux, &fork, &join) != WINO_OK) return false;
  if (cudaEventRecord(fork, st) != cudaSuccess || cudaStreamWaitEvent(aux, fork, 0) != cudaSuccess)
    return false;
  {
    ProfScope ps(kKFilter, aux);
    k_filter_transform_blk<MM><<<dim3((unsigned)((g.K + kFtK - 1) / kFtK), (unsigned)fy), 256, 0,
                                 aux>>>(w, Vb, g.C, g.K, M, sg);
  }
  if (cudaEventRecord(join, aux) != cudaSuccess) return false;
  {
    ProfScope ps(kKInput, st);
    k_input_transform_blk<MM><<<dim3((unsigned)sg.ntb, (unsigned)sg.nch), sg.CC * sg.TB, csm,
                                st>>>(x, Ub, g, M, sg);
  }
  return cudaStreamWaitEvent(st, join, 0) == cudaSuccess;
}

template <SPLIT_TPARAMS>
static int launch_split(const float* x, const float* w, float* y, const LayerGeom& g,
                        const LayerMats& M, void* ws, size_t ws_bytes, cudaStream_t st) {
  using Cfg = FusedCfg<FUSED_TARGS>;
  using SC = SplitCfg<SPLIT_TARGS>;
  if (g.K % Cfg::KB != 0) return kFallback;
  const SplitGeom sg = split_geom(g, Cfg::TB, Cfg::KB, CC);
  if (ws_bytes < split_ws_bytes(sg)) return kFallback;
  float* Vb = (float*)ws;
  float* Ub = (float*)((char*)ws + (((size_t)sg.vb_floats() * 4 + 255) & ~(size_t)255));
  int* err = nullptr;
  {
    int rc = wait_error_flag(&err);
    if (rc != WINO_OK) return rc;
  }
  static bool attr_set[16] = {false};
  int dev = 0;
  WINO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 16 && !attr_set[dev]) {
    WINO_CUDA_TRY(cudaFuncSetAttribute(k_gemm_otx<SPLIT_TARGS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SC::SMEM));
    attr_set[dev] = true;
  }
  const int64_t nblk = (int64_t)sg.nkb * sg.ntb;
  static_assert(CC * Cfg::TB <= 256, "one input-transform thread per (channel, tile) of a chunk");
  if (nblk > 0x7fffffffLL || !launch_split_transforms<MM>(x, w, g, M, sg, Ub, Vb, st))
    return kFallback;
  {
    ProfScope ps(kKFused, st);
    k_gemm_otx<SPLIT_TARGS><<<(unsigned)nblk, Cfg::NT, SC::SMEM, st>>>(Ub, Vb, y, g, M, sg, err);
  }
  note_launches(3);
  WINO_CUDA_TRY(cudaGetLastError());
  return WINO_OK;
}

// The cluster form of a tile shape: the same transforms and blocked
// layouts, then k_gemm_otx_cl.
template <CL_TPARAMS>
static size_t cl_ws_for(const LayerGeom& g) {
  using Cfg = ClCfg<CL_TARGS>;
  if (g.F != Cfg::F || g.K % Cfg::KB != 0) return 0;
  return split_ws_bytes(split_geom(g, Cfg::TB, Cfg::KB, CC));
}

template <CL_TPARAMS>
static int launch_split_cl(const float* x, const float* w, float* y, const LayerGeom& g,
                           const LayerMats& M, void* ws, size_t ws_bytes, cudaStream_t st) {
  using Cfg = ClCfg<CL_TARGS>;
  if (g.K % Cfg::KB != 0) return kFallback;
  const SplitGeom sg = split_geom(g, Cfg::TB, Cfg::KB, CC);
  if (ws_bytes < split_ws_bytes(sg)) return kFallback;
  float* Vb = (float*)ws;
  float* Ub = (float*)((char*)ws + (((size_t)sg.vb_floats() * 4 + 255) & ~(size_t)255));
  int* err = nullptr;
  {
    int rc = wait_error_flag(&err);
    if (rc != WINO_OK) return rc;
  }
  static bool attr_set[16] = {false};
  int dev = 0;
  WINO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 16 && !attr_set[dev]) {
    WINO_CUDA_TRY(cudaFuncSetAttribute(k_gemm_otx_cl<CL_TARGS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Cfg::SMEM));
    attr_set[dev] = true;
  }
  const int64_t nctas = (int64_t)NCL * sg.nkb * sg.ntb;
  static_assert(CC * Cfg::TB <= 256, "one input-transform thread per (channel, tile) of a chunk");
  if (nctas > 0x7fffffffLL || !launch_split_transforms<MM>(x, w, g, M, sg, Ub, Vb, st))
    return kFallback;
  {
    ProfScope ps(kKFused, st);
    k_gemm_otx_cl<CL_TARGS><<<(unsigned)nctas, Cfg::NT, Cfg::SMEM, st>>>(Ub, Vb, y, g, M, sg,
                                                                        err);
  }
  note_launches(3);
  WINO_CUDA_TRY(cudaGetLastError());
  return WINO_OK;
}

// Tile shapes of the split variant per m, as
// (MM, LX, LT, LK, FPL, MT, MK, CC, NS, MINB) -> TB = LT MT tiles x KB =
// LK MK output channels per CTA, CC channels per chunk, NS stages, MINB CTAs
// per SM for the register budget.  The layer autotuner times each.  (A
// 32 x 16 tile with an 8 x 8 microtile per thread and two CTAs per SM was
// measured slower: its register cap forces spills.)  The shared-memory path
// delivers one float per lane per 4 FMA lanes of the SM, so a thread tile of
// MT x MK outputs per frequency keeps the FMA pipe busy only when
// MT MK / (MT + MK) >= 4: the 4 x 8 tiles of the F(4x4) shapes cap it near
// 67%.  8 x 16 tiles for F(4x4) (one frequency per thread, four frequency
// groups per warp) need 9-warp CTAs, which three warps on one SM
// sub-partition cap at 168 registers: measured 14-25% slower than shape 1
// on the VGG16 stack (spills, one CTA per SM).  8 x 8 tiles (ratio 4, 112
// registers, no spills; 16 x 32 outputs per CTA, 9 warps) measured 18-35%
// slower: one CTA per SM does not hide the per-chunk waits and the epilogue.
// The cluster shapes below get 8 x 8 tiles at several CTAs per SM by
// splitting the frequencies over the CTAs of a cluster.
#define SPLIT_M2_0 2, 2, 4, 4, 1, 8, 16, 8, 2, 1
#define SPLIT_M4_0 4, 1, 4, 8, 3, 4, 8, 8, 2, 1
#define SPLIT_M4_1 4, 1, 8, 4, 3, 4, 8, 8, 2, 1
#define SPLIT_M4_2 4, 1, 8, 4, 3, 4, 8, 4, 4, 1
#define SPLIT_M6_0 6, 8, 1, 4, 1, 8, 16, 4, 2, 1
#define SPLIT_M6_1 6, 8, 2, 2, 1, 8, 16, 4, 3, 1
#define SPLIT_M6_2 6, 8, 2, 2, 1, 8, 16, 2, 4, 1
// Cluster tile shapes, as (MM, NCL, LX, LT, LK, MT, MK, CC, NS, MINB): 32
// (the last of each m: 16) tiles x 32 output channels per cluster, 8 x 8
// outputs of one frequency per thread, alpha^2 / NCL frequencies per CTA.
// The 16-tile shapes halve the work per cluster, and with it the last,
// partly filled wave of the deep VGG16 stages (784 clusters at stage 4 are
// 5.2 waves of 152 SMs' resident clusters; 256 at stage 5 are 1.7).  32 x
// 64 blocks (one warp per frequency, 6 or 8 CTAs per cluster, two per SM)
// measured 10-25% slower than the best shape on every VGG16 stage; CL_M4_2
// with four stages 5% slower, with two stages (96 registers, seven CTAs per
// SM) 3-7% slower; F(6x6) over 8 CTAs of two warps (16 tiles, six CTAs per
// SM) 2% slower than CL_M6_2; 16 x 64 blocks in 16-channel chunks over 6
// CTAs (half the chunk steps, and one k block at K = 64) were never the
// autotuner's pick on a VGG16 stage.  A persistent form (one cluster per
// resident cluster slot walking the blocks, its stage ring running on from
// one block's chunks into the next block's, the epilogue's accumulators in
// a region of their own behind a split cluster barrier) was bit-identical
// and 30-80% slower on every stage: that region costs the stages or the
// CTAs per SM the main loop needs (two stages at four CTAs per SM, or three
// at three, against three at five here).
#define CL_M4_0 4, 3, 2, 4, 4, 8, 8, 8, 3, 2
#define CL_M4_1 4, 3, 2, 4, 4, 8, 8, 8, 2, 3
#define CL_M4_2 4, 6, 2, 4, 4, 8, 8, 8, 3, 4
#define CL_M6_0 6, 4, 2, 4, 4, 8, 8, 8, 2, 2
#define CL_M6_1 6, 8, 2, 4, 4, 8, 8, 8, 3, 3
#define CL_M4_3 4, 3, 4, 2, 4, 8, 8, 8, 2, 5
#define CL_M6_2 6, 4, 4, 2, 4, 8, 8, 8, 2, 4

// Tile shapes per m: the single-CTA ones first, then the cluster ones.
int split_configs(int m) { return m == 2 ? 1 : m == 4 ? 7 : 6; }

size_t split_workspace_bytes(const LayerGeom& g) {
  size_t b = 0;
  auto mx = [&](size_t v) { b = v > b ? v : b; };
  if (g.F == 16) mx(split_ws_for<SPLIT_M2_0>(g));
  if (g.F == 36) {
    mx(split_ws_for<SPLIT_M4_0>(g));
    mx(split_ws_for<SPLIT_M4_1>(g));
    mx(split_ws_for<SPLIT_M4_2>(g));
    mx(cl_ws_for<CL_M4_0>(g));
    mx(cl_ws_for<CL_M4_1>(g));
    mx(cl_ws_for<CL_M4_2>(g));
    mx(cl_ws_for<CL_M4_3>(g));
  }
  if (g.F == 64) {
    mx(split_ws_for<SPLIT_M6_0>(g));
    mx(split_ws_for<SPLIT_M6_1>(g));
    mx(split_ws_for<SPLIT_M6_2>(g));
    mx(cl_ws_for<CL_M6_0>(g));
    mx(cl_ws_for<CL_M6_1>(g));
    mx(cl_ws_for<CL_M6_2>(g));
  }
  return b;
}

// Two-kernel variant (blocked U and V in the workspace); `cfg` picks the
// tile shape (0 .. split_configs(m) - 1).
int layer_forward_split(const float* x, const float* w, float* y, const LayerGeom& g,
                        const LayerMats& M, void* ws, size_t ws_bytes, cudaStream_t st,
                        int cfg) {
  if (g.dim != 2 || M.r != 3 || (M.m != 2 && M.m != 4 && M.m != 6) || g.K % 32 != 0)
    return kFallback;
  if (cfg < 0 || cfg >= split_configs(M.m)) return kFallback;
  if (M.m == 2) return launch_split<SPLIT_M2_0>(x, w, y, g, M, ws, ws_bytes, st);
  if (M.m == 4) {
    switch (cfg) {
      case 0: return launch_split<SPLIT_M4_0>(x, w, y, g, M, ws, ws_bytes, st);
      case 1: return launch_split<SPLIT_M4_1>(x, w, y, g, M, ws, ws_bytes, st);
      case 2: return launch_split<SPLIT_M4_2>(x, w, y, g, M, ws, ws_bytes, st);
      case 3: return launch_split_cl<CL_M4_0>(x, w, y, g, M, ws, ws_bytes, st);
      case 4: return launch_split_cl<CL_M4_1>(x, w, y, g, M, ws, ws_bytes, st);
      case 5: return launch_split_cl<CL_M4_2>(x, w, y, g, M, ws, ws_bytes, st);
      default: return launch_split_cl<CL_M4_3>(x, w, y, g, M, ws, ws_bytes, st);
    }
  }
  switch (cfg) {
    case 0: return launch_split<SPLIT_M6_0>(x, w, y, g, M, ws, ws_bytes, st);
    case 1: return launch_split<SPLIT_M6_1>(x, w, y, g, M, ws, ws_bytes, st);
    case 2: return launch_split<SPLIT_M6_2>(x, w, y, g, M, ws, ws_bytes, st);
    case 3: return launch_split_cl<CL_M6_0>(x, w, y, g, M, ws, ws_bytes, st);
    case 4: return launch_split_cl<CL_M6_1>(x, w, y, g, M, ws, ws_bytes, st);
    default: return launch_split_cl<CL_M6_2>(x, w, y, g, M, ws, ws_bytes, st);
  }
}

}  // namespace wino
