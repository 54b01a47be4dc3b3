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
// GPU layout: one lane per instance, as in the plain sweep (sweep.cu), with
// the same trials, chunking and FP64 trial sums.  The trees depend on the
// instance (c moves the magnitudes), so each lane builds its own once and
// keeps them packed per matrix row: byte 0 = merge count | root slot << 4,
// byte 1 + s = merge s as first slot | second slot << 4 (the sum takes the
// first slot).  Merging needs per-lane dynamic slot indices, so the values
// being merged live in shared memory as [slot][thread]: bank = thread mod 32
// whatever the slot, and the lanes' different trees never conflict.  All
// lanes of a warp share a mask, hence the positions of the zero entries and
// every merge count: the merge loops do not diverge.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "common.cuh"
#include "construct.cuh"
#include "sweep_eval.cuh"

namespace wino {
namespace {

constexpr int kOrderThreads = 128;

template <int N>
struct Tree {
  uint32_t w[(N + 3) / 4];
};

// Huffman tree of one matrix row (N FP64 entries; leaf weights are the
// |FP32-rounded| entries, zero entries left out).
template <int N>
__device__ __noinline__ void make_tree(const double* row, uint32_t* tw) {
  double wt[2 * N];
  int slot[2 * N];
  bool live[2 * N];
  int n_live = 0, last = 0;
  for (int k = 0; k < N; ++k) {
    wt[k] = fabs((double)__double2float_rn(row[k]));
    live[k] = wt[k] > 0.0;
    slot[k] = k;
    if (live[k]) {
      ++n_live;
      last = k;
    }
  }
  for (int q = 0; q < (N + 3) / 4; ++q) tw[q] = 0u;
  int nodes = N, s = 0;
  while (n_live > 1) {
    int f = -1, g = -1;
    for (int id = 0; id < nodes; ++id)  // least weight, earliest node on ties
      if (live[id] && (f < 0 || wt[id] < wt[f])) f = id;
    for (int id = 0; id < nodes; ++id)
      if (live[id] && id != f && (g < 0 || wt[id] < wt[g])) g = id;
    const uint32_t byte = (uint32_t)slot[f] | ((uint32_t)slot[g] << 4);
    tw[(s + 1) >> 2] |= byte << (8 * ((s + 1) & 3));
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
  tw[0] |= (uint32_t)s | ((uint32_t)root << 4);
}

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return __double2float_rn(v); }

// Shared-memory slot q of this thread is sv[q * kOrderThreads].
//
// tree_apply: out[v * os] = sum_k c[k] x[v * xv + k * xk] for v < NV, all
// along the one tree tw.  The NV sums are independent chains, merged in
// lock step: per merge the 2 NV loads issue before the NV stores, so the
// chains overlap instead of waiting on one another.
template <int N, int NV, typename T, typename X>
__device__ __forceinline__ void tree_apply(const T* c, const X* x, int xv, int xk,
                                           const uint32_t* tw, T* sv, T* out, int os) {
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int k = 0; k < N; ++k)
      sv[(v * N + k) * kOrderThreads] = mul_rn(c[k], (T)x[v * xv + k * xk]);
  const uint32_t w0 = tw[0];
  const int cnt = (int)(w0 & 15u);
  uint32_t cur = w0 >> 8;  // merge bytes still unread in the current word
  int left = 3, q = 0;
#pragma unroll 1
  for (int s = 0; s < cnt; ++s) {
    if (left == 0) {
      cur = tw[++q];
      left = 4;
    }
    const int a = (int)(cur & 15u), b = (int)((cur >> 4) & 15u);
    cur >>= 8;
    --left;
    T va[NV], vb[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      va[v] = sv[(v * N + a) * kOrderThreads];
      vb[v] = sv[(v * N + b) * kOrderThreads];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) sv[(v * N + a) * kOrderThreads] = add_rn(va[v], vb[v]);
  }
  const int root = (int)((w0 >> 4) & 15u);
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v * os] = sv[(v * N + root) * kOrderThreads];
}

// rows_apply: out[j] = sum_k c[j * N + k] x[k] for j < NR, row j along its
// own tree trees[j]; the rows' merges run in lock step like tree_apply's.
template <int N, int NR, typename T, typename X>
__device__ __forceinline__ void rows_apply(const T* c, const X* x, const Tree<N>* trees, T* sv,
                                           T* out) {
#pragma unroll
  for (int j = 0; j < NR; ++j)
#pragma unroll
    for (int k = 0; k < N; ++k)
      sv[(j * N + k) * kOrderThreads] = mul_rn(c[j * N + k], (T)x[k]);
  uint32_t cur[NR];
  int cnt[NR], left[NR], q[NR];
  int most = 0;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const uint32_t w0 = trees[j].w[0];
    cnt[j] = (int)(w0 & 15u);
    cur[j] = w0 >> 8;
    left[j] = 3;
    q[j] = 0;
    most = max(most, cnt[j]);
  }
#pragma unroll 1
  for (int s = 0; s < most; ++s) {
    int a[NR], b[NR];
    T va[NR], vb[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      if (s < cnt[j]) {
        if (left[j] == 0) {
          cur[j] = trees[j].w[++q[j]];
          left[j] = 4;
        }
        a[j] = (int)(cur[j] & 15u);
        b[j] = (int)((cur[j] >> 4) & 15u);
        cur[j] >>= 8;
        --left[j];
        va[j] = sv[(j * N + a[j]) * kOrderThreads];
        vb[j] = sv[(j * N + b[j]) * kOrderThreads];
      }
    }
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (s < cnt[j]) sv[(j * N + a[j]) * kOrderThreads] = add_rn(va[j], vb[j]);
  }
#pragma unroll
  for (int j = 0; j < NR; ++j)
    out[j] = sv[(j * N + (int)((trees[j].w[0] >> 4) & 15u)) * kOrderThreads];
}

template <int DIM, int M, int R, typename T>
struct OrderEval;

// 1D: u = G g, v = B^T d, p = u .* v (FP32), y = A^T p.
template <int M, int R, typename T>
__device__ __forceinline__ float order_err_1d(const OrderEval<1, M, R, T>& Q,
                                              const float* __restrict__ rc) {
  constexpr int A = M + R - 1;
  const float* g = rc;
  const float* d = rc + R;
  const float* yh = d + A;
  const float* yl = yh + M;
  T u[A], v[A], y[M];
  rows_apply<R, A>(Q.G, g, Q.tG, Q.sv, u);
  rows_apply<A, A>(Q.BT, d, Q.tB, Q.sv, v);
  float p[A];
#pragma unroll
  for (int i = 0; i < A; ++i) p[i] = __fmul_rn(to_f32(u[i]), to_f32(v[i]));
  rows_apply<A, M>(Q.AT, p, Q.tA, Q.sv, y);
  float e = 0.0f;
#pragma unroll
  for (int j = 0; j < M; ++j) e = __fadd_rn(e, abs_err(to_f32(y[j]), yh[j], yl[j]));
  return e;
}

// 2D, each pass one matrix row's tree over all the vectors it multiplies:
// W = G g (row i of G over the columns of g), U = W G^T (row j of G over
// the rows of W), T = B^T d, V = T B, P = U .* V (FP32), Z = A^T P,
// Y = Z A; the per-trial error summed over Y in row-major order.
template <int M, int R, typename T>
__device__ __forceinline__ float order_err_2d(const OrderEval<2, M, R, T>& Q,
                                              const float* __restrict__ rc) {
  constexpr int A = M + R - 1;
  const float* g = rc;
  const float* d = rc + R * R;
  const float* yh = d + A * A;
  const float* yl = yh + M * M;
  T W[A * R], U[A * A], Tm[A * A], Z[M * A];
  float P[A * A], Y[M * M];
#pragma unroll 1
  for (int i = 0; i < A; ++i)  // W[i][k] = sum_l G[i][l] g[l][k]
    tree_apply<R, R>(&Q.G[i * R], g, 1, R, Q.tG[i].w, Q.sv, &W[i * R], 1);
#pragma unroll 1
  for (int j = 0; j < A; ++j)  // U[i][j] = sum_k W[i][k] G[j][k]
    tree_apply<R, A>(&Q.G[j * R], W, R, 1, Q.tG[j].w, Q.sv, &U[j], A);
#pragma unroll 1
  for (int i = 0; i < A; ++i)  // T[i][l] = sum_k BT[i][k] d[k][l]
    tree_apply<A, A>(&Q.BT[i * A], d, 1, A, Q.tB[i].w, Q.sv, &Tm[i * A], 1);
#pragma unroll 1
  for (int j = 0; j < A; ++j) {  // V[i][j] = sum_l T[i][l] BT[j][l]; P = U .* V
    T Vj[A];
    tree_apply<A, A>(&Q.BT[j * A], Tm, A, 1, Q.tB[j].w, Q.sv, Vj, 1);
#pragma unroll
    for (int i = 0; i < A; ++i) P[i * A + j] = __fmul_rn(to_f32(U[i * A + j]), to_f32(Vj[i]));
  }
#pragma unroll 1
  for (int a = 0; a < M; ++a)  // Z[a][j] = sum_i AT[a][i] P[i][j]
    tree_apply<A, A>(&Q.AT[a * A], P, 1, A, Q.tA[a].w, Q.sv, &Z[a * A], 1);
#pragma unroll 1
  for (int b = 0; b < M; ++b) {  // Y[a][b] = sum_j Z[a][j] AT[b][j]
    T Yb[M];
    tree_apply<A, M>(&Q.AT[b * A], Z, A, 1, Q.tA[b].w, Q.sv, Yb, 1);
#pragma unroll
    for (int a = 0; a < M; ++a) Y[a * M + b] = to_f32(Yb[a]);
  }
  float e = 0.0f;
#pragma unroll
  for (int q = 0; q < M * M; ++q) e = __fadd_rn(e, abs_err(Y[q], yh[q], yl[q]));
  return e;
}

// One instance: its matrices (FP32 for the FP32 form, FP64 for the mixed
// form), its trees, and this thread's shared-memory slots.
template <int DIM, int M, int R, typename T>
struct OrderEval {
  static constexpr int A = M + R - 1;
  static constexpr int REC = SweepShape<DIM, M, R>::REC;
  T AT[M * A], G[A * R], BT[A * A];
  Tree<R> tG[A];
  Tree<A> tB[A];
  Tree<A> tA[M];
  T* sv;
  __device__ __forceinline__ float operator()(const float* buf) const {
    if constexpr (DIM == 1)
      return order_err_1d<M, R, T>(*this, buf);
    else
      return order_err_2d<M, R, T>(*this, buf);
  }
};

__device__ __forceinline__ float from_f64(double v, float*) { return __double2float_rn(v); }
__device__ __forceinline__ double from_f64(double v, double*) { return v; }

// Builds the instance from sorted finite points a[0..alpha-2]; false when
// two coincide (the matrices are then all zero).
template <int DIM, int M, int R, typename T>
__device__ __forceinline__ bool order_build(const double* a, OrderEval<DIM, M, R, T>& Q) {
  constexpr int A = M + R - 1;
  double ATd[M * A], Gd[A * R], BTd[A * A];
#pragma unroll
  for (int i = 0; i < M * A; ++i) ATd[i] = 0.0;
#pragma unroll
  for (int i = 0; i < A * R; ++i) Gd[i] = 0.0;
#pragma unroll
  for (int i = 0; i < A * A; ++i) BTd[i] = 0.0;
  const bool ok = build_matrices<double>(a, M, R, ATd, Gd, BTd);
#pragma unroll
  for (int i = 0; i < M * A; ++i) Q.AT[i] = from_f64(ATd[i], (T*)nullptr);
#pragma unroll
  for (int i = 0; i < A * R; ++i) Q.G[i] = from_f64(Gd[i], (T*)nullptr);
#pragma unroll
  for (int i = 0; i < A * A; ++i) Q.BT[i] = from_f64(BTd[i], (T*)nullptr);
  for (int i = 0; i < A; ++i) make_tree<R>(&Gd[i * R], Q.tG[i].w);
  for (int i = 0; i < A; ++i) make_tree<A>(&BTd[i * A], Q.tB[i].w);
  for (int j = 0; j < M; ++j) make_tree<A>(&ATd[j * A], Q.tA[j].w);
  return ok;
}

// One lane's instance from its sorted finite points a[0..alpha-2], over
// trial chunks [ch0, ch1) (lane_eval_ev's contract).  Not inlined: both
// kernels below run this one body.
template <int DIM, int M, int R, typename T>
__device__ __noinline__ void order_lane(const double* a, T* sv, const float* __restrict__ rec,
                                        int trials, int ch0, int ch1, double ysum, bool partial,
                                        double* __restrict__ out, int64_t stride, bool active) {
  OrderEval<DIM, M, R, T> Q;
  Q.sv = sv;
  const bool ok = order_build<DIM, M, R, T>(a, Q);
  lane_eval_ev(Q, ok, rec, trials, ch0, ch1, ysum, partial, out, stride, active);
}

// Mask sweep: the grid of k_sweep_eval (one warp per valid mask, block of
// 32 c values and chunk group; lanes own instances).
template <int DIM, int M, int R, typename T>
__global__ void __launch_bounds__(kOrderThreads)
    k_order_sweep(const float* __restrict__ rec, int trials, const double* __restrict__ c_grid,
                  int n_c, double d, const MaskList masks, const double* __restrict__ ysum,
                  double* __restrict__ err, int split, int ch_per, double* __restrict__ part,
                  int64_t n_out) {
  constexpr int A = M + R - 1;
  extern __shared__ __align__(16) unsigned char order_smem[];
  T* sv = reinterpret_cast<T*>(order_smem);  // A * A slots per thread
  const int lane = threadIdx.x & 31;
  const int nblk = (n_c + 31) >> 5;
  const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= (int64_t)masks.n * nblk * split) return;
  const int grp = (int)(item % split);
  const int cell = (int)(item / split);
  const int qv = cell / nblk;
  const int ci = (cell - qv * nblk) * 32 + lane;
  const bool active = ci < n_c;
  const double c = active ? c_grid[ci] : c_grid[0];
  const int64_t o = (int64_t)masks.q[qv] * n_c + ci;
  const int nch = trial_chunks(trials);
  const int ch0 = split == 1 ? 0 : grp * ch_per;
  const int ch1 = split == 1 ? nch : min(ch0 + ch_per, nch);
  double pts[kMaxAlpha];
  mask_points(masks.mask[qv], A, c, d, pts);  // valid: the host kept valid masks only
  order_lane<DIM, M, R, T>(pts, sv + threadIdx.x, rec, trials, ch0, ch1, *ysum, split > 1,
                           split == 1 ? err + o : part + o, n_out, active);
}

// Explicit point sets, one lane per set.
template <int DIM, int M, int R, typename T>
__global__ void __launch_bounds__(kOrderThreads)
    k_order_pointset(const float* __restrict__ rec, int trials, const double* __restrict__ pts,
                     int n_sets, const double* __restrict__ ysum, double* __restrict__ err) {
  constexpr int A = M + R - 1;
  extern __shared__ __align__(16) unsigned char order_smem[];
  T* sv = reinterpret_cast<T*>(order_smem);  // A * A slots per thread
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = s < n_sets;
  const int ss = active ? s : 0;
  double a[kMaxAlpha];
#pragma unroll
  for (int i = 0; i < A - 1; ++i) a[i] = pts[(int64_t)ss * (A - 1) + i];
  order_lane<DIM, M, R, T>(a, sv + threadIdx.x, rec, trials, 0, trial_chunks(trials), *ysum,
                           false, err + ss, 0, active);
}

}  // namespace

// Dynamic shared memory of the order kernels of size (m, r): A * A value
// slots per thread.
template <typename T>
inline size_t order_smem_bytes_t(int m, int r) {
  const size_t a = (size_t)(m + r - 1);
  return a * a * kOrderThreads * sizeof(T);
}

// The kernel tables of one value type T (float: the FP32 Huffman form,
// double: the mixed form); each kernel returned is allowed its dynamic
// shared memory (above the 48 KB default for the larger sizes).
template <typename T>
EvalFn order_sweep_kernel_t(int dim, int m, int r) {
  EvalFn fn = nullptr;
#define WINO_ORDER_CASE(I, D, MM, RR) \
  if (dim == D && m == MM && r == RR) fn = k_order_sweep<D, MM, RR, T>;
  WINO_SWEEP_SIZES(WINO_ORDER_CASE)
#undef WINO_ORDER_CASE
  if (fn && cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)order_smem_bytes_t<T>(m, r)) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return fn;
}

template <typename T>
PointsetFn order_pointset_kernel_t(int dim, int m, int r) {
  PointsetFn fn = nullptr;
#define WINO_ORDER_CASE(I, D, MM, RR) \
  if (dim == D && m == MM && r == RR) fn = k_order_pointset<D, MM, RR, T>;
  WINO_SWEEP_SIZES(WINO_ORDER_CASE)
#undef WINO_ORDER_CASE
  if (fn && cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)order_smem_bytes_t<T>(m, r)) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return fn;
}

}  // namespace wino
