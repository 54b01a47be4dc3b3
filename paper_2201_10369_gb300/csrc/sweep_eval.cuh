// sweep_eval.cuh -- device pieces of the point sweep shared by the per-size
// kernels (sweep.cu) and the persistent planned sweep (sweep_plan.cu).
//
// Trial records: one per trial, [g | d | hi(y) | lo(y)] in FP32, padded to a
// multiple of 4 floats, where y is the FP64 direct correlation of the tile
// (Eq. (1)) and hi = RN32(y), lo = RN32(y - hi).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace wino {

__host__ __device__ constexpr int round4(int v) { return (v + 3) & ~3; }

template <int DIM, int M, int R>
struct SweepShape {
  static constexpr int A = M + R - 1;
  static constexpr int NG = DIM == 1 ? R : R * R;
  static constexpr int ND = DIM == 1 ? A : A * A;
  static constexpr int NO = DIM == 1 ? M : M * M;
  static constexpr int REC = round4(NG + ND + 2 * NO);
};

template <int M, int R>
struct Mats {
  static constexpr int A = M + R - 1;
  float AT[M * A], G[A * R], BT[A * A];
};

// Builds one instance's matrices in FP64 (Sec. 4.1-4.2) and rounds them once
// to FP32 into registers.  Returns false for coinciding points.
template <int M, int R>
__device__ __forceinline__ bool build_instance(unsigned mask, double c, double d,
                                               Mats<M, R>& Mx) {
  constexpr int A = M + R - 1;
  double pts[kMaxAlpha];
  mask_points(mask, A, c, d, pts);
  double ATd[M * A], Gd[A * R], BTd[A * A];
  const bool ok = build_matrices<double>(pts, M, R, ATd, Gd, BTd);
#pragma unroll
  for (int i = 0; i < M * A; ++i) Mx.AT[i] = __double2float_rn(ATd[i]);
#pragma unroll
  for (int i = 0; i < A * R; ++i) Mx.G[i] = __double2float_rn(Gd[i]);
#pragma unroll
  for (int i = 0; i < A * A; ++i) Mx.BT[i] = __double2float_rn(BTd[i]);
  return ok;
}

// The same from explicit finite points a[0] < ... < a[alpha-2] (infinity is
// the extra point); false when two coincide.
template <int M, int R>
__device__ __forceinline__ bool build_from_points(const double* a, Mats<M, R>& Mx) {
  constexpr int A = M + R - 1;
  double ATd[M * A], Gd[A * R], BTd[A * A];
  const bool ok = build_matrices<double>(a, M, R, ATd, Gd, BTd);
#pragma unroll
  for (int i = 0; i < M * A; ++i) Mx.AT[i] = __double2float_rn(ATd[i]);
#pragma unroll
  for (int i = 0; i < A * R; ++i) Mx.G[i] = __double2float_rn(Gd[i]);
#pragma unroll
  for (int i = 0; i < A * A; ++i) Mx.BT[i] = __double2float_rn(BTd[i]);
  return ok;
}

// |yhat - y| with y = hi + lo, in FP32.
__device__ __forceinline__ float abs_err(float yhat, float hi, float lo) {
  return fabsf(__fsub_rn(__fsub_rn(yhat, hi), lo));
}

// 1D F(m, r): u = G g, v = BT d, p = u .* v, y = AT p  (Eq. (8)).
template <int M, int R>
__device__ __forceinline__ float tile_err_1d(const Mats<M, R>& Mx, const float* __restrict__ rc) {
  constexpr int A = M + R - 1;
  const float* g = rc;
  const float* d = rc + R;
  const float* yh = d + A;
  const float* yl = yh + M;
  float p[A];
#pragma unroll
  for (int i = 0; i < A; ++i) {
    float u = 0.0f, v = 0.0f;
#pragma unroll
    for (int k = 0; k < R; ++k) u = fmaf(Mx.G[i * R + k], g[k], u);
#pragma unroll
    for (int l = 0; l < A; ++l) v = fmaf(Mx.BT[i * A + l], d[l], v);
    p[i] = __fmul_rn(u, v);
  }
  float e = 0.0f;
#pragma unroll
  for (int j = 0; j < M; ++j) {
    float y = 0.0f;
#pragma unroll
    for (int i = 0; i < A; ++i) y = fmaf(Mx.AT[j * A + i], p[i], y);
    e = __fadd_rn(e, abs_err(y, yh[j], yl[j]));
  }
  return e;
}

// 2D F(m x m, r x r), Eq. (9), streamed one frequency row i at a time:
//   W_i = G_i g, U_i = W_i G^T, T_i = BT_i d, V_i = T_i B, P_i = U_i .* V_i,
//   Z += AT[:, i] P_i  (i ascending),  then Y = Z A.
template <int M, int R>
__device__ __forceinline__ float tile_err_2d(const Mats<M, R>& Mx, const float* __restrict__ rc) {
  constexpr int A = M + R - 1;
  const float* g = rc;
  const float* d = rc + R * R;
  const float* yh = d + A * A;
  const float* yl = yh + M * M;
  float Z[M * A];
#pragma unroll
  for (int i = 0; i < A; ++i) {
    float Wi[R], Ti[A];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      float acc = 0.0f;
#pragma unroll
      for (int l = 0; l < R; ++l) acc = fmaf(Mx.G[i * R + l], g[l * R + k], acc);
      Wi[k] = acc;
    }
#pragma unroll
    for (int l = 0; l < A; ++l) {
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < A; ++k) acc = fmaf(Mx.BT[i * A + k], d[k * A + l], acc);
      Ti[l] = acc;
    }
#pragma unroll
    for (int j = 0; j < A; ++j) {
      float u = 0.0f, v = 0.0f;
#pragma unroll
      for (int k = 0; k < R; ++k) u = fmaf(Wi[k], Mx.G[j * R + k], u);
#pragma unroll
      for (int l = 0; l < A; ++l) v = fmaf(Ti[l], Mx.BT[j * A + l], v);
      const float p = __fmul_rn(u, v);
#pragma unroll
      for (int a = 0; a < M; ++a)
        Z[a * A + j] = (i == 0) ? fmaf(Mx.AT[a * A + i], p, 0.0f)
                                : fmaf(Mx.AT[a * A + i], p, Z[a * A + j]);
    }
  }
  float e = 0.0f;
#pragma unroll
  for (int a = 0; a < M; ++a)
#pragma unroll
    for (int b = 0; b < M; ++b) {
      float y = 0.0f;
#pragma unroll
      for (int j = 0; j < A; ++j) y = fmaf(Z[a * A + j], Mx.AT[b * A + j], y);
      e = __fadd_rn(e, abs_err(y, yh[a * M + b], yl[a * M + b]));
    }
  return e;
}

// Summation order of the error's numerator, fixed for every execution path:
// trials are taken in chunks of kTrialChunk; each chunk's per-trial FP32
// sums are accumulated in trial order by ChunkSum below, whose result is
// widened to FP64, and the chunk sums are added in FP64 in ascending chunk
// order.  A path may therefore evaluate the chunks of one instance in
// different warps (partials in memory, combined by k_sweep_combine) and
// still return the same bits as one lane running them all.
constexpr int kTrialChunk = 128;
__host__ __device__ constexpr int trial_chunks(int trials) {
  return (trials + kTrialChunk - 1) / kTrialChunk;
}

// Compensated FP32 sum of one chunk's per-trial errors: the running sum is
// the unevaluated pair hi + lo; each term is added to hi with Knuth's TwoSum
// (six rounded FP32 operations that recover the rounding error of hi + e
// exactly) and that error is added to lo.  The chunk's value is hi + lo in
// FP64.  For n terms of one sign the result is within (n u)^2 (u = 2^-24)
// of the exact sum -- about 6e-11 relative for n = 128 -- as close as an
// FP64 running sum needs to be here, at FP32 cost: on this part an FP64
// operation occupies the FP64 unit 64 times as long as an FP32 one, and a
// per-trial FP64 add would bound the small sweep sizes.
struct ChunkSum {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float e) {
    const float s = __fadd_rn(hi, e);
    const float bv = __fsub_rn(s, hi);
    const float av = __fsub_rn(s, bv);
    const float r = __fadd_rn(__fsub_rn(hi, av), __fsub_rn(e, bv));
    hi = s;
    lo = __fadd_rn(lo, r);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Sum over trials [t0, t1) (one chunk, ChunkSum) of the per-trial FP32 L1
// error; `ev(buf)` returns one trial's error from its record (Ev::REC
// floats).
template <class Ev>
__device__ __forceinline__ double chunk_error_ev(const Ev& ev, const float* __restrict__ rec,
                                                 int t0, int t1) {
  constexpr int REC = Ev::REC;
  ChunkSum num;
  const float4* r4 = reinterpret_cast<const float4*>(rec);
  auto load = [&](int t, float (&buf)[REC]) {
#pragma unroll
    for (int q = 0; q < REC / 4; ++q) {
      const float4 v = __ldg(r4 + (int64_t)t * (REC / 4) + q);
      buf[4 * q + 0] = v.x;
      buf[4 * q + 1] = v.y;
      buf[4 * q + 2] = v.z;
      buf[4 * q + 3] = v.w;
    }
  };
  int t = t0;
  if constexpr (Ev::PAIRS) {
    // short tiles: two trials per iteration, two independent evaluations
    // in flight; their errors still join the sum in trial order
    for (; t + 1 < t1; t += 2) {
      float b0[REC], b1[REC];
      load(t, b0);
      load(t + 1, b1);
      const float e0 = ev(b0), e1 = ev(b1);
      num.add(e0);
      num.add(e1);
    }
  }
  for (; t < t1; ++t) {
    float buf[REC];
    load(t, buf);
    num.add(ev(buf));
  }
  return num.value();
}

// One lane's instance (evaluator ev; ok = false when two points coincide)
// over trial chunks [ch0, ch1) of `trials` warp-uniform trial records.
// partial == false (the lane owns every chunk):
// *out = sum_t ||yhat_t - y_t||_1 / sum_t ||y_t||_1, +inf when two points
// coincide.  partial == true: out[ch * stride] = the chunk's sum (+inf when
// two points coincide), for k_sweep_combine.  Per trial the m (m^2) terms are
// summed in FP32, the trial sums in FP64 in the chunked order above.
template <class Ev>
__device__ __forceinline__ void lane_eval_ev(const Ev& ev, bool ok, const float* __restrict__ rec,
                                             int trials, int ch0, int ch1, double ysum,
                                             bool partial, double* __restrict__ out,
                                             int64_t stride, bool active) {
  double num = 0.0;
  for (int ch = ch0; ch < ch1; ++ch) {
    const int t0 = ch * kTrialChunk;
    const double s = chunk_error_ev(ev, rec, t0, min(t0 + kTrialChunk, trials));
    if (partial) {
      if (active) out[(int64_t)ch * stride] = ok ? s : (double)INFINITY;
    } else {
      num += s;
    }
  }
  if (!partial && active) *out = ok ? num / ysum : (double)INFINITY;
}

// The plain-order tile error of matrices Mx (fmaf, inner index ascending).
template <int DIM, int M, int R>
struct PlainEval {
  static constexpr int REC = SweepShape<DIM, M, R>::REC;
  static constexpr bool PAIRS = DIM == 1;
  const Mats<M, R>& Mx;
  __device__ __forceinline__ float operator()(const float* buf) const {
    return DIM == 1 ? tile_err_1d<M, R>(Mx, buf) : tile_err_2d<M, R>(Mx, buf);
  }
};

template <int DIM, int M, int R>
__device__ __forceinline__ void lane_eval_mats(const Mats<M, R>& Mx, bool ok,
                                               const float* __restrict__ rec, int trials,
                                               int ch0, int ch1, double ysum, bool partial,
                                               double* __restrict__ out, int64_t stride,
                                               bool active) {
  lane_eval_ev(PlainEval<DIM, M, R>{Mx}, ok, rec, trials, ch0, ch1, ysum, partial, out, stride,
               active);
}

// lane_eval_mats for the instance (mask, c, d) of a sweep.
template <int DIM, int M, int R>
__device__ __forceinline__ void lane_eval(const float* __restrict__ rec, int trials,
                                          unsigned mask, double c, double d, int ch0, int ch1,
                                          double ysum, bool partial, double* __restrict__ out,
                                          int64_t stride, bool active) {
  Mats<M, R> Mx;
  const bool ok = build_instance<M, R>(mask, c, d, Mx);
  lane_eval_mats<DIM, M, R>(Mx, ok, rec, trials, ch0, ch1, ysum, partial, out, stride, active);
}

// Valid masks of one size (at most 256) and their positions in the caller's
// subset list.
struct MaskList {
  unsigned char mask[256];
  short q[256];  // index of the mask in the caller's subset list
  int n;
};

// Mask-sweep kernel of one size (k_sweep_eval in sweep.cu): (rec, trials,
// c_grid, n_c, d, masks, ysum, err, split, ch_per, part, n_out), one warp per
// (mask, 32 c values, chunk group).
typedef void (*EvalFn)(const float*, int, const double*, int, double, const MaskList,
                       const double*, double*, int, int, double*, int64_t);
// Point-set kernel of one size: (rec, trials, sorted finite points, n_sets,
// ysum, err), one lane per set.
typedef void (*PointsetFn)(const float*, int, const double*, int, const double*, double*);

// Warp-per-instance sweeps (sweep_order_f32.cu, sweep_order_f64.cu): enqueue
// the sweep of one size's valid masks over c_grid (err[q * n_c + k] for the
// caller's subset index q), or of n_sets explicit sorted point sets, in
// order 0 (the plain fmaf order: the wide sizes only), 1 (Huffman, FP32) or
// 2 (Huffman, FP64 transforms; orders 1 and 2 for every size of
// WINO_SWEEP_SIZES and WINO_SWEEP_SIZES_WIDE), else WINO_EUNSUPPORTED.
int order_sweep_launch(int order, const SweepSize& s, const float* rec, int trials,
                       const double* c_grid, int n_c, const MaskList& masks, const double* ysum,
                       double* err, cudaStream_t st);
int order_pointset_launch(int order, int dim, int m, int r, const float* rec, int trials,
                          const double* pts, int n_sets, const double* ysum, double* err,
                          cudaStream_t st);

// Partial chunk sums -> errors: err[i] = (sum over chunks ascending of
// part[ch * stride + i]) / ysum of the instance's size, where the size is
// size_of[i] (or 0 when size_of is null).  sweep.cu.
int sweep_combine(const double* part, int n_chunks, int64_t stride, int64_t n,
                  const unsigned char* size_of, const double* ysum, double* err, cudaStream_t st);

// How many warps a chunk-split sweep launch aims for: enough items that a
// launch of few instances still fills every SM several times over.
int sweep_target_warps();
// The same for one size of the per-size sweep, whose sizes share the GPU
// (sweep.cu).
int sweep_split_warps();

// Sizes the sweep is compiled for, as (index, dim, m, r) cases.
#define WINO_SWEEP_SIZES(X) \
  X(0, 1, 2, 3)             \
  X(1, 1, 3, 3)             \
  X(2, 1, 4, 3)             \
  X(3, 1, 5, 3)             \
  X(4, 1, 6, 3)             \
  X(5, 1, 7, 3)             \
  X(6, 1, 8, 3)             \
  X(7, 1, 2, 5)             \
  X(8, 1, 3, 5)             \
  X(9, 1, 4, 5)             \
  X(10, 1, 5, 5)            \
  X(11, 1, 6, 5)            \
  X(12, 2, 2, 3)            \
  X(13, 2, 3, 3)            \
  X(14, 2, 4, 3)            \
  X(15, 2, 5, 3)            \
  X(16, 2, 6, 3)            \
  X(17, 2, 2, 5)            \
  X(18, 2, 3, 5)            \
  X(19, 2, 4, 5)

// Wide sizes: 2D F(7x7,3x3) and F(8x8,3x3) (alpha 9, 10), whose per-lane
// tile does not fit the registers: swept only by the warp-per-instance
// kernels of sweep_order.cuh (plain order and Huffman orders alike).
#define WINO_SWEEP_SIZES_WIDE(X) \
  X(20, 2, 7, 3)                 \
  X(21, 2, 8, 3)

inline bool sweep_wide(int dim, int m, int r) {
#define WINO_WIDE_CASE(I, D, MM, RR) \
  if (dim == D && m == MM && r == RR) return true;
  WINO_SWEEP_SIZES_WIDE(WINO_WIDE_CASE)
#undef WINO_WIDE_CASE
  return false;
}

// Index of (dim, m, r) in WINO_SWEEP_SIZES, or -1.
inline int sweep_kind(int dim, int m, int r) {
#define WINO_KIND_CASE(I, D, MM, RR) \
  if (dim == D && m == MM && r == RR) return I;
  WINO_SWEEP_SIZES(WINO_KIND_CASE)
#undef WINO_KIND_CASE
  return -1;
}

// Host: record width (floats) of a size.
inline int sweep_rec_width(int dim, int m, int r) {
  const int a = m + r - 1;
  const int ng = dim == 1 ? r : r * r, nd = dim == 1 ? a : a * a, no = dim == 1 ? m : m * m;
  return round4(ng + nd + 2 * no);
}

// Dense FP32 flops of one trial of one instance (cost model for scheduling
// and the roofline): 1D 2(a r + a^2 + m a) + a;
// 2D 2(a r^2 + a^2 r) + 4 a^3 + a^2 + 2(m a^2 + m^2 a).
inline double sweep_trial_flops(int dim, int m, int r) {
  const double a = m + r - 1;
  if (dim == 1) return 2 * (a * r + a * a + m * a) + a;
  return 2 * (a * r * r + a * a * r) + 4 * a * a * a + a * a + 2 * (m * a * a + m * m * a);
}

// k_sweep_prepare launcher (sweep.cu): trial records and per-block partial
// sums of |y| for one size, then their fixed-order total into *ysum.
int sweep_prepare(float* rec, double* partial, double* ysum, int dim, int m, int r, int trials,
                  uint64_t seed, cudaStream_t st);
inline int sweep_prepare_blocks(int trials) { return (trials + 255) / 256; }

}  // namespace wino
