// sweep_order.cuh -- summation-order variants of the point sweep (Sec. 5).
// Included by sweep_order_f32.cu (the FP32 form) and sweep_order_f64.cu (the
// mixed form), each instantiating the kernels of one value type.
//
// The paper's error tables evaluate every transform in the Huffman order of
// Barabasz et al., and its error curves also show that order with the
// transforms in FP64 and the Hadamard product in FP32.  The paper defines
// neither; the reading implemented here: each output of a transform is one
// dot product over a row of G, B^T or A^T (a 2D transform is two passes,
// left factor first); its non-zero terms are rounded products c_k x_k,
// added along the Huffman tree of |c_k| (the FP32 entries): the two live
// nodes of least weight are replaced by their sum, whose weight is the FP64
// sum of theirs; ties go to the node created first (leaves in column order,
// then merged nodes in creation order).  FP32 form: products and sums in
// FP32.  Mixed form: the same trees over the FP64 matrices, FP64 products
// and sums, U and V rounded to FP32, P = U .* V in FP32, the output
// transform in FP64 and Y rounded once.
//
// GPU layout: one warp per instance, its lanes taking 32 trials at a time.
// The instance's matrices (rows padded to 16 bytes) and trees live once per
// warp in shared memory and are read as broadcasts; the trees are therefore
// warp-uniform and no merge loop diverges.  A tree is packed per matrix row:
// byte 0 = merge count | root slot << 4, byte 1 + s = merge s as first slot
// | second slot << 4 (the sum takes the first slot).  The values being merged
// need dynamic slot indices, so each lane keeps them in the warp's shared
// memory as [slot][lane] (bank = lane, conflict-free).  A row's tree is
// applied to all the vectors it multiplies at once, or all rows' trees in
// lock step, so 5-10 independent merge chains overlap.  The 2D Hadamard
// product P = U .* V waits in shared memory ([element][lane]) for the output
// transform; everything else a trial needs stays in registers.
//
// Error sums: per trial the outputs' errors in FP32 (row-major); each lane
// adds the errors of its trials t = lane, lane + 32, ... in FP64 in trial
// order, and the 32 lane sums are combined by a fixed butterfly of
// shuffles (lane l with l ^ 16, then ^ 8, ^ 4, ^ 2, ^ 1), the same in both
// kernels.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "../../include/wino.h"
#include "common.cuh"
#include "construct.cuh"
#include "sweep_eval.cuh"

namespace wino {
namespace {

constexpr int kOrderWarps = 4;  // warps (instances) per block
constexpr int kOrderThreads = 32 * kOrderWarps;
constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ constexpr int pad_to(int n, int v) { return (n + v - 1) / v * v; }
__host__ __device__ constexpr size_t pad16(size_t b) { return (b + 15) & ~(size_t)15; }

// Byte layout of one warp's shared-memory region.  HUFF = false (the plain
// fmaf order of the wide sizes) keeps only the matrices and P.
template <int DIM, int M, int R, typename T, bool HUFF = true>
struct OrderLayout {
  static constexpr int A = M + R - 1;
  static constexpr int V = 16 / (int)sizeof(T);  // elements per 16-byte load
  static constexpr int GS = pad_to(R, V);        // row strides (elements)
  static constexpr int BS = pad_to(A, V);
  static constexpr int WG = (R + 3) / 4;  // tree words per row
  static constexpr int WB = (A + 3) / 4;
  static constexpr int NSLOT = HUFF ? A * A + 1 : 0;  // + one dummy slot for padded merges
  static constexpr int A4 = pad_to(A, 4), M4 = pad_to(M, 4);  // program row widths
  static constexpr size_t G_OFF = 0;
  static constexpr size_t BT_OFF = G_OFF + sizeof(T) * A * GS;
  static constexpr size_t AT_OFF = BT_OFF + sizeof(T) * A * BS;
  static constexpr size_t TG_OFF = AT_OFF + sizeof(T) * M * BS;
  static constexpr int HW = HUFF ? 1 : 0;
  static constexpr size_t TB_OFF = TG_OFF + 4 * (size_t)A * WG * HW;
  static constexpr size_t TA_OFF = TB_OFF + 4 * (size_t)A * WB * HW;
  // lock-step merge programs of the three row sets (G, B^T, A^T): per step
  // one word per row, then each row's root offset
  static constexpr size_t PG_OFF = pad16(TA_OFF + 4 * (size_t)M * WB * HW);
  static constexpr size_t PB_OFF = PG_OFF + 4 * (size_t)(R - 1) * A4 * HW;
  static constexpr size_t PA_OFF = PB_OFF + 4 * (size_t)(A - 1) * A4 * HW;
  static constexpr size_t RG_OFF = PA_OFF + 4 * (size_t)(A - 1) * M4 * HW;
  static constexpr size_t RB_OFF = RG_OFF + 4 * (size_t)A4 * HW;
  static constexpr size_t RA_OFF = RB_OFF + 4 * (size_t)A4 * HW;
  static constexpr size_t SL_OFF = pad16(RA_OFF + 4 * (size_t)M4 * HW);
  static constexpr size_t P_OFF = SL_OFF + sizeof(T) * NSLOT * 32;
  static constexpr size_t BYTES = pad16(P_OFF + (DIM == 2 ? 4 * (size_t)A * A * 32 : 0));
};

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return __double2float_rn(v); }
__device__ __forceinline__ float from_f64(double v, float*) { return __double2float_rn(v); }
__device__ __forceinline__ double from_f64(double v, double*) { return v; }

// Huffman tree of one matrix row of N coefficients (shared memory), packed
// into (N + 3) / 4 words; leaf weights are the |FP32-rounded| entries, zero
// entries left out.
template <int N, typename T>
__device__ __noinline__ void make_tree(const T* row, uint32_t* tw) {
  double wt[2 * N];
  int slot[2 * N];
  bool live[2 * N];
  int n_live = 0, last = 0;
  for (int k = 0; k < N; ++k) {
    wt[k] = fabs((double)to_f32(row[k]));
    live[k] = wt[k] > 0.0;
    slot[k] = k;
    if (live[k]) {
      ++n_live;
      last = k;
    }
  }
  uint32_t w[(N + 3) / 4];
  for (int q = 0; q < (N + 3) / 4; ++q) w[q] = 0u;
  int nodes = N, s = 0;
  while (n_live > 1) {
    int f = -1, g = -1;
    for (int id = 0; id < nodes; ++id)  // least weight, earliest node on ties
      if (live[id] && (f < 0 || wt[id] < wt[f])) f = id;
    for (int id = 0; id < nodes; ++id)
      if (live[id] && id != f && (g < 0 || wt[id] < wt[g])) g = id;
    const uint32_t byte = (uint32_t)slot[f] | ((uint32_t)slot[g] << 4);
    w[(s + 1) >> 2] |= byte << (8 * ((s + 1) & 3));
    wt[nodes] = __dadd_rn(wt[f], wt[g]);
    slot[nodes] = slot[f];
    live[nodes] = true;
    live[f] = false;
    live[g] = false;
    ++nodes;
    ++s;
    --n_live;
  }
  const int root = s == 0 ? last : slot[nodes - 1];
  w[0] |= (uint32_t)s | ((uint32_t)root << 4);
  for (int q = 0; q < (N + 3) / 4; ++q) tw[q] = w[q];
}

// N coefficients of a shared-memory row (16-byte aligned, zero-padded) in
// 16-byte loads.
template <int N>
__device__ __forceinline__ void load_row(const float* s, float (&c)[N]) {
  constexpr int NP = pad_to(N, 4);
  float t[NP];
#pragma unroll
  for (int q = 0; q < NP / 4; ++q) {
    const float4 v = reinterpret_cast<const float4*>(s)[q];
    t[4 * q] = v.x;
    t[4 * q + 1] = v.y;
    t[4 * q + 2] = v.z;
    t[4 * q + 3] = v.w;
  }
#pragma unroll
  for (int k = 0; k < N; ++k) c[k] = t[k];
}
template <int N>
__device__ __forceinline__ void load_row(const double* s, double (&c)[N]) {
  constexpr int NP = pad_to(N, 2);
  double t[NP];
#pragma unroll
  for (int q = 0; q < NP / 2; ++q) {
    const double2 v = reinterpret_cast<const double2*>(s)[q];
    t[2 * q] = v.x;
    t[2 * q + 1] = v.y;
  }
#pragma unroll
  for (int k = 0; k < N; ++k) c[k] = t[k];
}

// Byte offset, from this lane's slot 0, of slot q.
template <typename T>
__host__ __device__ constexpr uint32_t slot_off(int q) {
  return (uint32_t)q * 32u * (uint32_t)sizeof(T);
}

// Lock-step merge program of NR rows of N entries (row j's slots are
// j * N .. j * N + N - 1): step s holds one word per row, (first slot's byte
// offset) | (second slot's byte offset) << 16 for row j's merge s, or the
// dummy slot twice once row j has no merge s left; roots[j] = the byte
// offset of row j's root.  Lane j < NR writes row j's column from its tree;
// returns the step count (the largest merge count), the same in every lane.
template <int N, int NR, int NRP, int W, typename T>
__device__ __forceinline__ int make_program(const uint32_t* trees, uint32_t* prog,
                                            uint32_t* roots, int dummy) {
  const int lane = threadIdx.x & 31;
  int cnt = 0;
  if (lane < NR) cnt = (int)(trees[lane * W] & 15u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt = max(cnt, __shfl_xor_sync(kFull, cnt, o));
  if (lane < NR) {
    const uint32_t* tw = trees + lane * W;
    const int mine = (int)(tw[0] & 15u);
    for (int s = 0; s < cnt; ++s) {
      uint32_t op = slot_off<T>(dummy) | (slot_off<T>(dummy) << 16);
      if (s < mine) {
        const uint32_t b = (tw[(s + 1) >> 2] >> (8 * ((s + 1) & 3))) & 255u;
        op = slot_off<T>(lane * N + (int)(b & 15u)) |
             (slot_off<T>(lane * N + (int)(b >> 4)) << 16);
      }
      prog[s * NRP + lane] = op;
    }
    roots[lane] = slot_off<T>(lane * N + (int)((tw[0] >> 4) & 15u));
  }
  return cnt;
}

// Slot q of this lane is sv[q * 32].
//
// tree_apply: out[v] = sum_k c[k] x[v * xv + k * xk] for v < NV, all along
// the tree of row j of a row set: its merges are column j of the set's
// program (make_program), its merge count is word 0 of its packed tree tw,
// its root offset roots[j].  Those offsets address slots j * N + ..., so the
// slot base moves back by j * N slots; vector v uses slots v * N + ....  The
// NV sums are independent chains merged in lock step: per merge the 2 NV
// loads issue before the NV stores.
template <int N, int NV, int NRP, typename T, typename X>
__device__ __forceinline__ void tree_apply(const T* c_s, const X* x, int xv, int xk,
                                           const uint32_t* prog, const uint32_t* roots,
                                           const uint32_t* tw, int j, T* sv, T (&out)[NV]) {
  T c[N];
  load_row<N>(c_s, c);
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int k = 0; k < N; ++k) sv[(v * N + k) * 32] = mul_rn(c[k], (T)x[v * xv + k * xk]);
  char* svb = reinterpret_cast<char*>(sv) - slot_off<T>(j * N);
  const int cnt = (int)(tw[0] & 15u);
#pragma unroll 1
  for (int s = 0; s < cnt; ++s) {
    const uint32_t op = prog[s * NRP + j];
    char* pa = svb + (op & 0xffffu);
    const char* pb = svb + (op >> 16);
    T va[NV], vb[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      va[v] = *reinterpret_cast<const T*>(pa + slot_off<T>(v * N));
      vb[v] = *reinterpret_cast<const T*>(pb + slot_off<T>(v * N));
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) *reinterpret_cast<T*>(pa + slot_off<T>(v * N)) = add_rn(va[v], vb[v]);
  }
  const char* pr = svb + roots[j];
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = *reinterpret_cast<const T*>(pr + slot_off<T>(v * N));
}

// rows_apply: out[j] = sum_k c[j][k] x[k] for j < NR (row stride S), row j
// along its own tree, by the lock-step program `prog` of `steps` steps
// (make_program): per step all NR loads pairs issue before the NR stores.
template <int N, int NR, int NRP, int S, typename T, typename X>
__device__ __forceinline__ void rows_apply(const T* c_s, const X* x, const uint32_t* prog,
                                           int steps, const uint32_t* roots, T* sv,
                                           T (&out)[NR]) {
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    T c[N];
    load_row<N>(c_s + j * S, c);
#pragma unroll
    for (int k = 0; k < N; ++k) sv[(j * N + k) * 32] = mul_rn(c[k], (T)x[k]);
  }
  char* svb = reinterpret_cast<char*>(sv);
#pragma unroll 1
  for (int s = 0; s < steps; ++s) {
    uint32_t op[NRP];
#pragma unroll
    for (int q = 0; q < NRP / 4; ++q) {
      const uint4 w = reinterpret_cast<const uint4*>(prog + s * NRP)[q];
      op[4 * q] = w.x;
      op[4 * q + 1] = w.y;
      op[4 * q + 2] = w.z;
      op[4 * q + 3] = w.w;
    }
    T va[NR], vb[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      va[j] = *reinterpret_cast<const T*>(svb + (op[j] & 0xffffu));
      vb[j] = *reinterpret_cast<const T*>(svb + (op[j] >> 16));
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) *reinterpret_cast<T*>(svb + (op[j] & 0xffffu)) = add_rn(va[j], vb[j]);
  }
#pragma unroll
  for (int j = 0; j < NR; ++j) out[j] = *reinterpret_cast<const T*>(svb + roots[j]);
}

// The FP32 L1 error of trial record r (layout of sweep_eval.cuh) in this
// lane, against the instance in shared memory at `base`.
template <int DIM, int M, int R, typename T>
__device__ __forceinline__ float order_trial(const unsigned char* base, const float* __restrict__ r,
                                             T* sv, float* pl, int sg, int sb, int sa) {
  using L = OrderLayout<DIM, M, R, T>;
  using S = SweepShape<DIM, M, R>;
  constexpr int A = L::A;
  const T* Gs = reinterpret_cast<const T*>(base + L::G_OFF);
  const T* BTs = reinterpret_cast<const T*>(base + L::BT_OFF);
  const T* ATs = reinterpret_cast<const T*>(base + L::AT_OFF);
  const uint32_t* tG = reinterpret_cast<const uint32_t*>(base + L::TG_OFF);
  const uint32_t* tB = reinterpret_cast<const uint32_t*>(base + L::TB_OFF);
  const uint32_t* tA = reinterpret_cast<const uint32_t*>(base + L::TA_OFF);
  const uint32_t* pG = reinterpret_cast<const uint32_t*>(base + L::PG_OFF);
  const uint32_t* pB = reinterpret_cast<const uint32_t*>(base + L::PB_OFF);
  const uint32_t* pA = reinterpret_cast<const uint32_t*>(base + L::PA_OFF);
  const uint32_t* rG = reinterpret_cast<const uint32_t*>(base + L::RG_OFF);
  const uint32_t* rB = reinterpret_cast<const uint32_t*>(base + L::RB_OFF);
  const uint32_t* rA = reinterpret_cast<const uint32_t*>(base + L::RA_OFF);
  // g and d in 16-byte loads (the record is 16-byte aligned)
  constexpr int NIN = pad_to(S::NG + S::ND, 4);
  float in[NIN];
#pragma unroll
  for (int q = 0; q < NIN / 4; ++q) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(r) + q);
    in[4 * q] = v.x;
    in[4 * q + 1] = v.y;
    in[4 * q + 2] = v.z;
    in[4 * q + 3] = v.w;
  }
  const float* g = in;
  const float* d = in + S::NG;
  const float* yh = r + S::NG + S::ND;
  const float* yl = yh + S::NO;
  float e = 0.0f;
  if constexpr (DIM == 1) {
    // u = G g, v = B^T d, p = u .* v (FP32), y = A^T p
    T u[A], v[A], y[M];
    rows_apply<R, A, L::A4, L::GS>(Gs, g, pG, sg, rG, sv, u);
    rows_apply<A, A, L::A4, L::BS>(BTs, d, pB, sb, rB, sv, v);
    float p[A];
#pragma unroll
    for (int i = 0; i < A; ++i) p[i] = __fmul_rn(to_f32(u[i]), to_f32(v[i]));
    rows_apply<A, M, L::M4, L::BS>(ATs, p, pA, sa, rA, sv, y);
#pragma unroll
    for (int j = 0; j < M; ++j) e = __fadd_rn(e, abs_err(to_f32(y[j]), __ldg(yh + j), __ldg(yl + j)));
  } else {
    // per frequency row i: W_i = G_i g, U_i = W_i G^T, T_i = B^T_i d,
    // V_i = T_i B, P_i = U_i .* V_i (FP32, to shared memory); then per output
    // row a: Z_a = A^T_a P, Y_a = Z_a A, errors in row-major order
#pragma unroll 1
    for (int i = 0; i < A; ++i) {
      T Wi[R], Ui[A], Ti[A], Vi[A];
      tree_apply<R, R, L::A4>(Gs + i * L::GS, g, 1, R, pG, rG, tG + i * L::WG, i, sv, Wi);
      rows_apply<R, A, L::A4, L::GS>(Gs, Wi, pG, sg, rG, sv, Ui);
      tree_apply<A, A, L::A4>(BTs + i * L::BS, d, 1, A, pB, rB, tB + i * L::WB, i, sv, Ti);
      rows_apply<A, A, L::A4, L::BS>(BTs, Ti, pB, sb, rB, sv, Vi);
#pragma unroll
      for (int j = 0; j < A; ++j) pl[(i * A + j) * 32] = __fmul_rn(to_f32(Ui[j]), to_f32(Vi[j]));
    }
#pragma unroll 1
    for (int a = 0; a < M; ++a) {
      T Za[A], Ya[M];
      tree_apply<A, A, L::M4>(ATs + a * L::BS, pl, 32, A * 32, pA, rA, tA + a * L::WB, a, sv,
                              Za);
      rows_apply<A, M, L::M4, L::BS>(ATs, Za, pA, sa, rA, sv, Ya);
#pragma unroll
      for (int b = 0; b < M; ++b)
        e = __fadd_rn(e, abs_err(to_f32(Ya[b]), __ldg(yh + a * M + b), __ldg(yl + a * M + b)));
    }
  }
  return e;
}

// The same error in the plain fmaf order of the lane-per-instance sweep
// (tile_err_1d / tile_err_2d in sweep_eval.cuh, operation for operation),
// the matrices read from shared memory: used for the wide 2D sizes whose
// per-lane form would not fit the registers.
template <int DIM, int M, int R>
__device__ __forceinline__ float fma_trial(const unsigned char* base, const float* __restrict__ r,
                                           float* pl) {
  using L = OrderLayout<DIM, M, R, float, false>;
  using S = SweepShape<DIM, M, R>;
  constexpr int A = L::A;
  const float* Gs = reinterpret_cast<const float*>(base + L::G_OFF);
  const float* BTs = reinterpret_cast<const float*>(base + L::BT_OFF);
  const float* ATs = reinterpret_cast<const float*>(base + L::AT_OFF);
  constexpr int NIN = pad_to(S::NG + S::ND, 4);
  float in[NIN];
#pragma unroll
  for (int q = 0; q < NIN / 4; ++q) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(r) + q);
    in[4 * q] = v.x;
    in[4 * q + 1] = v.y;
    in[4 * q + 2] = v.z;
    in[4 * q + 3] = v.w;
  }
  const float* g = in;
  const float* d = in + S::NG;
  const float* yh = r + S::NG + S::ND;
  const float* yl = yh + S::NO;
  float e = 0.0f;
  if constexpr (DIM == 1) {
    float p[A];
#pragma unroll
    for (int i = 0; i < A; ++i) {
      float gr[R], br[A];
      load_row<R>(Gs + i * L::GS, gr);
      load_row<A>(BTs + i * L::BS, br);
      float u = 0.0f, v = 0.0f;
#pragma unroll
      for (int k = 0; k < R; ++k) u = fmaf(gr[k], g[k], u);
#pragma unroll
      for (int l = 0; l < A; ++l) v = fmaf(br[l], d[l], v);
      p[i] = __fmul_rn(u, v);
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
      float ar[A];
      load_row<A>(ATs + j * L::BS, ar);
      float y = 0.0f;
#pragma unroll
      for (int i = 0; i < A; ++i) y = fmaf(ar[i], p[i], y);
      e = __fadd_rn(e, abs_err(y, __ldg(yh + j), __ldg(yl + j)));
    }
  } else {
    // per frequency row i: W_i = G_i g, T_i = B^T_i d, then U[i][j], V[i][j],
    // P[i][j] = U .* V to shared memory; Z = A^T P (i ascending), Y = Z A
#pragma unroll 1
    for (int i = 0; i < A; ++i) {
      float gi[R], bi[A], Wi[R], Ti[A];
      load_row<R>(Gs + i * L::GS, gi);
      load_row<A>(BTs + i * L::BS, bi);
#pragma unroll
      for (int k = 0; k < R; ++k) {
        float acc = 0.0f;
#pragma unroll
        for (int l = 0; l < R; ++l) acc = fmaf(gi[l], g[l * R + k], acc);
        Wi[k] = acc;
      }
#pragma unroll
      for (int l = 0; l < A; ++l) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < A; ++k) acc = fmaf(bi[k], d[k * A + l], acc);
        Ti[l] = acc;
      }
#pragma unroll 2
      for (int j = 0; j < A; ++j) {
        float gj[R], bj[A];
        load_row<R>(Gs + j * L::GS, gj);
        load_row<A>(BTs + j * L::BS, bj);
        float u = 0.0f, v = 0.0f;
#pragma unroll
        for (int k = 0; k < R; ++k) u = fmaf(Wi[k], gj[k], u);
#pragma unroll
        for (int l = 0; l < A; ++l) v = fmaf(Ti[l], bj[l], v);
        pl[(i * A + j) * 32] = __fmul_rn(u, v);
      }
    }
#pragma unroll 1
    for (int a = 0; a < M; ++a) {
      float ar[A], Za[A];
      load_row<A>(ATs + a * L::BS, ar);
#pragma unroll
      for (int j = 0; j < A; ++j) {
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < A; ++i) acc = fmaf(ar[i], pl[(i * A + j) * 32], acc);
        Za[j] = acc;
      }
#pragma unroll 2
      for (int b = 0; b < M; ++b) {
        float br[A];
        load_row<A>(ATs + b * L::BS, br);
        float y = 0.0f;
#pragma unroll
        for (int j = 0; j < A; ++j) y = fmaf(Za[j], br[j], y);
        e = __fadd_rn(e, abs_err(y, __ldg(yh + a * M + b), __ldg(yl + a * M + b)));
      }
    }
  }
  return e;
}

// One instance on one warp: sorted finite points a[0..alpha-2] (the same in
// every lane) -> err = sum_t ||yhat_t - y_t||_1 / ysum, +inf when two points
// coincide.  HUFF: the Huffman order, trial sums per lane then a butterfly.
// !HUFF (T = float): the plain fmaf order and the plain sweep's chunked
// trial sums (each round's 32 errors gathered in trial order), so its bits
// are the lane-per-instance sweep's.  Not inlined: both kernels run this one
// body.
template <int DIM, int M, int R, typename T, bool HUFF>
__device__ __noinline__ double order_instance(const double* a, unsigned char* base,
                                              const float* __restrict__ rec, int trials,
                                              double ysum) {
  using L = OrderLayout<DIM, M, R, T, HUFF>;
  constexpr int A = L::A;
  const int lane = threadIdx.x & 31;
  T* Gs = reinterpret_cast<T*>(base + L::G_OFF);
  T* BTs = reinterpret_cast<T*>(base + L::BT_OFF);
  T* ATs = reinterpret_cast<T*>(base + L::AT_OFF);
  int ok = 0;
  if (lane == 0) {  // the FP64 matrices, stored as T with zero-padded rows
    double ATd[M * A], Gd[A * R], BTd[A * A];
    ok = build_matrices<double>(a, M, R, ATd, Gd, BTd) ? 1 : 0;
    if (ok) {
      for (int i = 0; i < A; ++i)
        for (int k = 0; k < L::GS; ++k)
          Gs[i * L::GS + k] = k < R ? from_f64(Gd[i * R + k], (T*)nullptr) : (T)0;
      for (int i = 0; i < A; ++i)
        for (int k = 0; k < L::BS; ++k)
          BTs[i * L::BS + k] = k < A ? from_f64(BTd[i * A + k], (T*)nullptr) : (T)0;
      for (int j = 0; j < M; ++j)
        for (int k = 0; k < L::BS; ++k)
          ATs[j * L::BS + k] = k < A ? from_f64(ATd[j * A + k], (T*)nullptr) : (T)0;
    }
  }
  ok = __shfl_sync(kFull, ok, 0);
  if (!ok) return (double)INFINITY;
  __syncwarp();
  constexpr int REC = SweepShape<DIM, M, R>::REC;
  float* pl = reinterpret_cast<float*>(base + L::P_OFF) + lane;
  if constexpr (!HUFF) {
    static_assert(kTrialChunk % 32 == 0, "chunks are whole rounds of 32 trials");
    double num = 0.0;
    ChunkSum chunk;
    const int rounds = (trials + 31) / 32;
    for (int rd = 0; rd < rounds; ++rd) {
      const int t = rd * 32 + lane;
      float e = 0.0f;
      if (t < trials) e = fma_trial<DIM, M, R>(base, rec + (int64_t)t * REC, pl);
      const int n_here = min(32, trials - rd * 32);
      for (int j = 0; j < 32; ++j) {  // this round's errors in trial order
        const float ej = __shfl_sync(kFull, e, j);
        if (j < n_here) chunk.add(ej);
      }
      if ((rd + 1) % (kTrialChunk / 32) == 0 || rd + 1 == rounds) {
        num += chunk.value();
        chunk = ChunkSum();
      }
    }
    return num / ysum;
  }
  // one tree per lane: G rows, then B^T rows, then A^T rows
  if (lane < A)
    make_tree<R>(Gs + lane * L::GS, reinterpret_cast<uint32_t*>(base + L::TG_OFF) + lane * L::WG);
  else if (lane < 2 * A)
    make_tree<A>(BTs + (lane - A) * L::BS,
                 reinterpret_cast<uint32_t*>(base + L::TB_OFF) + (lane - A) * L::WB);
  else if (lane < 2 * A + M)
    make_tree<A>(ATs + (lane - 2 * A) * L::BS,
                 reinterpret_cast<uint32_t*>(base + L::TA_OFF) + (lane - 2 * A) * L::WB);
  __syncwarp();
  // the lock-step programs of the three row sets
  auto u32 = [&](size_t off) { return reinterpret_cast<uint32_t*>(base + off); };
  const int dummy = L::NSLOT - 1;
  const int sg = make_program<R, A, L::A4, L::WG, T>(u32(L::TG_OFF), u32(L::PG_OFF),
                                                     u32(L::RG_OFF), dummy);
  const int sb = make_program<A, A, L::A4, L::WB, T>(u32(L::TB_OFF), u32(L::PB_OFF),
                                                     u32(L::RB_OFF), dummy);
  const int sa = make_program<A, M, L::M4, L::WB, T>(u32(L::TA_OFF), u32(L::PA_OFF),
                                                     u32(L::RA_OFF), dummy);
  __syncwarp();
  T* sv = reinterpret_cast<T*>(base + L::SL_OFF) + lane;
  double num = 0.0;
  for (int t = lane; t < trials; t += 32)
    num += (double)order_trial<DIM, M, R, T>(base, rec + (int64_t)t * REC, sv, pl, sg, sb, sa);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) num += __shfl_xor_sync(kFull, num, o);
  return num / ysum;
}

// Mask sweep: one warp per (valid mask, c) instance.
template <int DIM, int M, int R, typename T, bool HUFF>
__global__ void __launch_bounds__(kOrderThreads, HUFF ? 3 : 2)
    k_order_sweep(const float* __restrict__ rec, int trials, const double* __restrict__ c_grid,
                  int n_c, double d, const MaskList masks, const double* __restrict__ ysum,
                  double* __restrict__ err) {
  using L = OrderLayout<DIM, M, R, T, HUFF>;
  extern __shared__ __align__(16) unsigned char order_smem[];
  const int warp = threadIdx.x >> 5;
  const int64_t inst = (int64_t)blockIdx.x * kOrderWarps + warp;
  if (inst >= (int64_t)masks.n * n_c) return;  // the whole warp
  const int qv = (int)(inst / n_c);
  const int ci = (int)(inst - (int64_t)qv * n_c);
  double pts[kMaxAlpha];
  mask_points(masks.mask[qv], L::A, c_grid[ci], d, pts);  // valid: the host kept valid masks
  const double e =
      order_instance<DIM, M, R, T, HUFF>(pts, order_smem + warp * L::BYTES, rec, trials, *ysum);
  if ((threadIdx.x & 31) == 0) err[(int64_t)masks.q[qv] * n_c + ci] = e;
}

// Explicit point sets: one warp per set.
template <int DIM, int M, int R, typename T, bool HUFF>
__global__ void __launch_bounds__(kOrderThreads, HUFF ? 3 : 2)
    k_order_pointset(const float* __restrict__ rec, int trials, const double* __restrict__ pts,
                     int n_sets, const double* __restrict__ ysum, double* __restrict__ err) {
  using L = OrderLayout<DIM, M, R, T, HUFF>;
  extern __shared__ __align__(16) unsigned char order_smem[];
  const int warp = threadIdx.x >> 5;
  const int s = blockIdx.x * kOrderWarps + warp;
  if (s >= n_sets) return;  // the whole warp
  double a[kMaxAlpha];
  for (int i = 0; i < L::A - 1; ++i) a[i] = pts[(int64_t)s * (L::A - 1) + i];
  const double e = order_instance<DIM, M, R, T, HUFF>(a, order_smem + warp * L::BYTES, rec,
                                                      trials, *ysum);
  if ((threadIdx.x & 31) == 0) err[s] = e;
}

}  // namespace

// Launches of one form: T = float, HUFF (the FP32 Huffman order), T =
// double, HUFF (its FP64-transform form) or T = float, !HUFF (the plain fmaf
// order, for the wide sizes).  SIZES is the size list compiled for the form.
// Each kernel is allowed its dynamic shared memory (above the 48 KB default
// for the larger sizes) before its launch.
#define WINO_ORDER_SIZES_HUFF(X) WINO_SWEEP_SIZES(X) WINO_SWEEP_SIZES_WIDE(X)
template <typename T, bool HUFF>
int order_sweep_launch_t(const SweepSize& s, const float* rec, int trials, const double* c_grid,
                         int n_c, const MaskList& masks, const double* ysum, double* err,
                         cudaStream_t st) {
  const int64_t n = (int64_t)masks.n * n_c;
  if (n == 0) return WINO_OK;
  const unsigned grid = (unsigned)((n + kOrderWarps - 1) / kOrderWarps);
#define WINO_ORDER_CASE(I, D, MM, RR)                                                        \
  if (s.dim == D && s.m == MM && s.r == RR) {                                                 \
    const size_t smem = kOrderWarps * OrderLayout<D, MM, RR, T, HUFF>::BYTES;                 \
    WINO_CUDA_TRY(cudaFuncSetAttribute((const void*)k_order_sweep<D, MM, RR, T, HUFF>,        \
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                                       (int)smem));                                           \
    k_order_sweep<D, MM, RR, T, HUFF><<<grid, kOrderThreads, smem, st>>>(                     \
        rec, trials, c_grid, n_c, s.d, masks, ysum, err);                                     \
    note_launches(1);                                                                         \
    WINO_CUDA_TRY(cudaGetLastError());                                                        \
    return WINO_OK;                                                                           \
  }
  if constexpr (HUFF) {
    WINO_ORDER_SIZES_HUFF(WINO_ORDER_CASE)
  } else {
    WINO_SWEEP_SIZES_WIDE(WINO_ORDER_CASE)
  }
#undef WINO_ORDER_CASE
  return WINO_EUNSUPPORTED;
}

template <typename T, bool HUFF>
int order_pointset_launch_t(int dim, int m, int r, const float* rec, int trials,
                            const double* pts, int n_sets, const double* ysum, double* err,
                            cudaStream_t st) {
  if (n_sets <= 0) return WINO_OK;
  const unsigned grid = (unsigned)((n_sets + kOrderWarps - 1) / kOrderWarps);
#define WINO_ORDER_CASE(I, D, MM, RR)                                                        \
  if (dim == D && m == MM && r == RR) {                                                       \
    const size_t smem = kOrderWarps * OrderLayout<D, MM, RR, T, HUFF>::BYTES;                 \
    WINO_CUDA_TRY(cudaFuncSetAttribute((const void*)k_order_pointset<D, MM, RR, T, HUFF>,     \
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                                       (int)smem));                                           \
    k_order_pointset<D, MM, RR, T, HUFF><<<grid, kOrderThreads, smem, st>>>(                  \
        rec, trials, pts, n_sets, ysum, err);                                                 \
    note_launches(1);                                                                         \
    WINO_CUDA_TRY(cudaGetLastError());                                                        \
    return WINO_OK;                                                                           \
  }
  if constexpr (HUFF) {
    WINO_ORDER_SIZES_HUFF(WINO_ORDER_CASE)
  } else {
    WINO_SWEEP_SIZES_WIDE(WINO_ORDER_CASE)
  }
#undef WINO_ORDER_CASE
  return WINO_EUNSUPPORTED;
}

}  // namespace wino
