// sweep.cu -- the batched FP32-versus-FP64 point sweep (Sec. 6.1-6.3).
//
// For every (size, subset mask, c) instance the paper's measurement is
//   err = sum_t ||yhat_t - y_t||_1 / sum_t ||y_t||_1
// over `trials` random single-tile problems (Sec. 6: random inputs, L1
// distance to a double-precision direct convolution).
//
// Device work per size:
//   k_sweep_prepare  one thread per trial: draws g, d (SplitMix64 counter
//                    stream), computes the FP64 direct correlation y of the
//                    tile and stores one record per trial
//                    [g | d | hi(y) | lo(y)]  (hi = RN32(y), lo = RN32(y - hi))
//                    plus per-block FP64 partial sums of |y|;
//   k_sweep_ysum     fixed-order reduction of the partials -> sum_t ||y_t||_1;
//   k_sweep_eval     one warp per (mask, 32 consecutive c): each lane builds
//                    its instance's matrices in FP64 (Sec. 4.1-4.2), rounds
//                    them once to FP32 into registers, and runs all trials
//                    with the FP32 Winograd tile; the trial records are
//                    warp-uniform loads.  Per trial the lane sums
//                    |(yhat - hi) - lo| over the m (m^2) outputs in FP32
//                    and adds that to an FP64 accumulator.
// The FP32 tile follows the library's fixed operation order (fmaf over the
// inner index ascending, one rounded Hadamard multiply), so yhat is
// bit-identical to any implementation of the same order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "../../include/wino.h"
#include "common.cuh"

namespace wino {

// ---------------------------------------------------------------------------
// Counter-based SplitMix64 (Steele, Lea, Flood 2014): the n-th output of the
// generator started at `seed` is the finaliser of seed + n * 0x9E3779B97F4A7C15.
// Trial input idx (idx < 256: kernel g, idx >= 256: data d) of trial t of
// size (dim, m, r) uses counter n = 1 + idx + 2^12 (t + 2^20 (r + 2^4 (m +
// 2^4 dim))); its top 24 bits k give the exact FP32 value k * 2^-23 - 1.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
  uint64_t z = seed + n * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float trial_value(uint64_t seed, int dim, int m, int r, int t,
                                             int idx) {
  uint64_t ctr = (((((uint64_t)dim * 16u + (uint64_t)m) * 16u + (uint64_t)r) << 20) +
                  (uint64_t)t)
                     << 12;
  ctr += (uint64_t)idx;
  const uint64_t z = splitmix64_at(seed, ctr + 1u);
  return (float)((int)(z >> 40)) * 0x1p-23f - 1.0f;  // exact: k < 2^24
}

__host__ __device__ constexpr int round4(int v) { return (v + 3) & ~3; }

struct SizeShape {
  int dim, m, r, alpha, nin_g, nin_d, nout, rec;
};

static SizeShape shape_of(int dim, int m, int r) {
  SizeShape s;
  s.dim = dim;
  s.m = m;
  s.r = r;
  s.alpha = m + r - 1;
  s.nin_g = dim == 1 ? r : r * r;
  s.nin_d = dim == 1 ? s.alpha : s.alpha * s.alpha;
  s.nout = dim == 1 ? m : m * m;
  s.rec = round4(s.nin_g + s.nin_d + 2 * s.nout);
  return s;
}

// ---------------------------------------------------------------------------
// k_sweep_prepare: one thread per trial.
// ---------------------------------------------------------------------------
__global__ void k_sweep_prepare(float* __restrict__ rec, double* __restrict__ partial, int dim,
                                int m, int r, int trials, int recw, uint64_t seed) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int A = m + r - 1;
  const int ng = dim == 1 ? r : r * r, nd = dim == 1 ? A : A * A, no = dim == 1 ? m : m * m;
  double s = 0.0;
  if (t < trials) {
    float* out = rec + (int64_t)t * recw;
    float g[kMaxR * kMaxR], d[kMaxAlpha * kMaxAlpha];
    for (int i = 0; i < ng; ++i) g[i] = trial_value(seed, dim, m, r, t, i);
    for (int i = 0; i < nd; ++i) d[i] = trial_value(seed, dim, m, r, t, 256 + i);
    for (int i = 0; i < ng; ++i) out[i] = g[i];
    for (int i = 0; i < nd; ++i) out[ng + i] = d[i];
    for (int o = 0; o < no; ++o) {
      const int a = dim == 1 ? 0 : o / m, b = dim == 1 ? o : o % m;
      double acc = 0.0;
      if (dim == 1) {
        for (int k = 0; k < r; ++k) acc = fma((double)g[k], (double)d[b + k], acc);
      } else {
        for (int u = 0; u < r; ++u)
          for (int v = 0; v < r; ++v)
            acc = fma((double)g[u * r + v], (double)d[(a + u) * A + b + v], acc);
      }
      const float hi = __double2float_rn(acc);
      const float lo = __double2float_rn(acc - (double)hi);
      out[ng + nd + o] = hi;
      out[ng + nd + no + o] = lo;
      s += fabs(acc);
    }
    for (int i = ng + nd + 2 * no; i < recw; ++i) out[i] = 0.0f;
  }
  // block partial of |y| (warp shuffle, then lane 0 of each warp in order)
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += ws[w];
    partial[blockIdx.x] = b;
  }
}

__global__ void k_sweep_ysum(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += partial[i];
    *out = s;
  }
}

// ---------------------------------------------------------------------------
// Register-resident FP32 tile evaluation (compile-time sizes).
// ---------------------------------------------------------------------------
template <int M, int R>
struct Mats {
  static constexpr int A = M + R - 1;
  float AT[M * A], G[A * R], BT[A * A];
};

// Builds the instance matrices (FP64, rounded once) into registers.
// Returns false for coinciding points.
template <int M, int R>
__device__ __forceinline__ bool build_instance(unsigned mask, double c, double d, Mats<M, R>& Mx) {
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

// |yhat - y| summed over the tile, y = hi + lo; FP32.
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

struct MaskList {
  unsigned char mask[256];
  short q[256];  // index of the mask in the caller's subset list
  int n;
};

// One warp per (valid mask, block of 32 c values); lanes own instances.
template <int DIM, int M, int R>
__global__ void __launch_bounds__(128) k_sweep_eval(const float* __restrict__ rec, int trials,
                                                    const double* __restrict__ c_grid, int n_c,
                                                    double d, const MaskList masks,
                                                    const double* __restrict__ ysum,
                                                    double* __restrict__ err) {
  constexpr int A = M + R - 1;
  constexpr int NG = DIM == 1 ? R : R * R;
  constexpr int ND = DIM == 1 ? A : A * A;
  constexpr int NO = DIM == 1 ? M : M * M;
  constexpr int REC = round4(NG + ND + 2 * NO);
  const int lane = threadIdx.x & 31;
  const int nblk = (n_c + 31) >> 5;
  const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= masks.n * nblk) return;
  const int qv = item / nblk;
  const int ci = (item - qv * nblk) * 32 + lane;
  const bool active = ci < n_c;
  const double c = active ? c_grid[ci] : c_grid[0];
  Mats<M, R> Mx;
  const bool ok = build_instance<M, R>(masks.mask[qv], c, d, Mx);

  double num = 0.0;
  const float4* r4 = reinterpret_cast<const float4*>(rec);
  for (int t = 0; t < trials; ++t) {
    float buf[REC];
#pragma unroll
    for (int q = 0; q < REC / 4; ++q) {
      const float4 v = __ldg(r4 + (int64_t)t * (REC / 4) + q);
      buf[4 * q + 0] = v.x;
      buf[4 * q + 1] = v.y;
      buf[4 * q + 2] = v.z;
      buf[4 * q + 3] = v.w;
    }
    const float e = (DIM == 1) ? tile_err_1d<M, R>(Mx, buf) : tile_err_2d<M, R>(Mx, buf);
    num += (double)e;
  }
  if (active) {
    double* out = err + (int64_t)masks.q[qv] * n_c + ci;
    *out = ok ? num / *ysum : (double)INFINITY;
  }
}

typedef void (*EvalFn)(const float*, int, const double*, int, double, const MaskList,
                       const double*, double*);

static EvalFn eval_kernel(int dim, int m, int r) {
#define WINO_EVAL_CASE(D, MM, RR) \
  if (dim == D && m == MM && r == RR) return k_sweep_eval<D, MM, RR>;
  WINO_EVAL_CASE(1, 2, 3)
  WINO_EVAL_CASE(1, 3, 3)
  WINO_EVAL_CASE(1, 4, 3)
  WINO_EVAL_CASE(1, 5, 3)
  WINO_EVAL_CASE(1, 6, 3)
  WINO_EVAL_CASE(1, 7, 3)
  WINO_EVAL_CASE(1, 8, 3)
  WINO_EVAL_CASE(1, 2, 5)
  WINO_EVAL_CASE(1, 3, 5)
  WINO_EVAL_CASE(1, 4, 5)
  WINO_EVAL_CASE(1, 5, 5)
  WINO_EVAL_CASE(1, 6, 5)
  WINO_EVAL_CASE(2, 2, 3)
  WINO_EVAL_CASE(2, 3, 3)
  WINO_EVAL_CASE(2, 4, 3)
  WINO_EVAL_CASE(2, 5, 3)
  WINO_EVAL_CASE(2, 6, 3)
#undef WINO_EVAL_CASE
  return nullptr;
}

// Valid masks of a size among the caller's subsets (same rule as
// mask_points: popcount alpha - 2, and bits 4 / 7 unused when |d| = 1).
static MaskList valid_masks(const SweepSize& s, const unsigned char* subsets, int n_subsets) {
  MaskList L;
  memset(&L, 0, sizeof(L));
  const int alpha = s.m + s.r - 1;
  for (int q = 0; q < n_subsets && L.n < 256; ++q) {
    const unsigned mk = subsets[q];
    int cnt = 0;
    for (int b = 0; b < 8; ++b) cnt += (mk >> b) & 1u;
    if (cnt != alpha - 2) continue;
    if (fabs(s.d) == 1.0 && (mk & 0x90u)) continue;
    L.mask[L.n] = (unsigned char)mk;
    L.q[L.n] = (short)q;
    ++L.n;
  }
  return L;
}

int error_sweep(const double* c_grid, int n_c, const SweepSize* sizes, int n_sizes,
                const unsigned char* subsets, int n_subsets, int trials, unsigned long long seed,
                double* err_out, cudaStream_t st) {
  std::vector<SizeShape> shp(n_sizes);
  std::vector<size_t> rec_off(n_sizes);
  size_t rec_total = 0;
  const int prep_threads = 256;
  const int nb_prep = (trials + prep_threads - 1) / prep_threads;
  for (int s = 0; s < n_sizes; ++s) {
    shp[s] = shape_of(sizes[s].dim, sizes[s].m, sizes[s].r);
    if (!eval_kernel(sizes[s].dim, sizes[s].m, sizes[s].r)) {
      set_error("sweep size not compiled: 1D r=3 m=2..8, 1D r=5 m=2..6, 2D r=3 m=2..6");
      return WINO_EUNSUPPORTED;
    }
    rec_off[s] = rec_total;
    rec_total += (size_t)trials * shp[s].rec;
  }
  // scratch layout: records | partials | ysum | c_grid | err
  const size_t n_err = (size_t)n_sizes * n_subsets * n_c;
  size_t off_part = rec_total * sizeof(float);
  off_part = (off_part + 255) & ~(size_t)255;
  size_t off_ysum = off_part + (size_t)n_sizes * nb_prep * sizeof(double);
  off_ysum = (off_ysum + 255) & ~(size_t)255;
  size_t off_c = off_ysum + (size_t)n_sizes * sizeof(double);
  off_c = (off_c + 255) & ~(size_t)255;
  size_t off_err = off_c + (size_t)n_c * sizeof(double);
  off_err = (off_err + 255) & ~(size_t)255;
  const size_t total = off_err + n_err * sizeof(double);
  void* base = nullptr;
  int rc = scratch_get(kScratchSweep, total, &base);
  if (rc != WINO_OK) return rc;
  char* b = (char*)base;
  float* rec = (float*)b;
  double* part = (double*)(b + off_part);
  double* ysum = (double*)(b + off_ysum);
  double* cg = (double*)(b + off_c);
  double* err = (double*)(b + off_err);

  WINO_CUDA_TRY(cudaMemcpyAsync(cg, c_grid, n_c * sizeof(double), cudaMemcpyHostToDevice, st));
  std::vector<MaskList> ml(n_sizes);
  for (int s = 0; s < n_sizes; ++s) {
    const SizeShape& z = shp[s];
    ProfScope ps(kKSweepPrep, st);
    k_sweep_prepare<<<nb_prep, prep_threads, 0, st>>>(rec + rec_off[s], part + (size_t)s * nb_prep,
                                                       z.dim, z.m, z.r, trials, z.rec, seed);
    k_sweep_ysum<<<1, 32, 0, st>>>(part + (size_t)s * nb_prep, nb_prep, ysum + s);
    ml[s] = valid_masks(sizes[s], subsets, n_subsets);
    note_launches(2);
  }
  WINO_CUDA_TRY(cudaGetLastError());
  const int nblk = (n_c + 31) / 32;
  for (int s = 0; s < n_sizes; ++s) {
    if (ml[s].n == 0) continue;
    const int items = ml[s].n * nblk;
    const int warps_per_block = 4;
    const int grid = (items + warps_per_block - 1) / warps_per_block;
    EvalFn fn = eval_kernel(sizes[s].dim, sizes[s].m, sizes[s].r);
    ProfScope ps(kKSweepEval, st);
    fn<<<grid, 32 * warps_per_block, 0, st>>>(rec + rec_off[s], trials, cg, n_c, sizes[s].d,
                                               ml[s], ysum + s, err + (size_t)s * n_subsets * n_c);
    note_launches(1);
  }
  WINO_CUDA_TRY(cudaGetLastError());
  WINO_CUDA_TRY(
      cudaMemcpyAsync(err_out, err, n_err * sizeof(double), cudaMemcpyDeviceToHost, st));
  WINO_CUDA_TRY(cudaStreamSynchronize(st));
  // invalid (size, mask) pairs: NaN
  for (int s = 0; s < n_sizes; ++s) {
    std::vector<char> valid(n_subsets, 0);
    for (int i = 0; i < ml[s].n; ++i) valid[ml[s].q[i]] = 1;
    for (int q = 0; q < n_subsets; ++q)
      if (!valid[q])
        for (int k = 0; k < n_c; ++k) err_out[((size_t)s * n_subsets + q) * n_c + k] = NAN;
  }
  return WINO_OK;
}

}  // namespace wino

namespace wino {

// Device FP64 construction for a batch of instances (the sweep's matrix
// build, exposed for parity checks): one thread per c.
__global__ void k_instance_matrices(const double* __restrict__ cg, int n_c, int m, int r,
                                    double d, unsigned mask, double* __restrict__ AT,
                                    double* __restrict__ G, double* __restrict__ BT,
                                    unsigned char* __restrict__ sing) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_c) return;
  const int A = m + r - 1;
  double pts[kMaxAlpha];
  mask_points(mask, A, cg[k], d, pts);
  const bool ok = build_matrices<double>(pts, m, r, AT + (int64_t)k * m * A,
                                         G + (int64_t)k * A * r, BT + (int64_t)k * A * A);
  sing[k] = ok ? 0 : 1;
}

int instance_matrices(const double* c_grid, int n_c, const SweepSize& s, unsigned mask,
                      double* AT, double* G, double* BT, unsigned char* singular,
                      cudaStream_t st) {
  const int A = s.m + s.r - 1;
  const size_t nAT = (size_t)n_c * s.m * A, nG = (size_t)n_c * A * s.r, nBT = (size_t)n_c * A * A;
  const size_t bytes = (n_c + nAT + nG + nBT) * sizeof(double) + n_c + 1024;
  void* base = nullptr;
  int rc = scratch_get(kScratchSweep, bytes, &base);
  if (rc != WINO_OK) return rc;
  double* cg = (double*)base;
  double* dAT = cg + n_c;
  double* dG = dAT + nAT;
  double* dBT = dG + nG;
  unsigned char* ds = (unsigned char*)(dBT + nBT);
  WINO_CUDA_TRY(cudaMemcpyAsync(cg, c_grid, n_c * sizeof(double), cudaMemcpyHostToDevice, st));
  k_instance_matrices<<<(n_c + 127) / 128, 128, 0, st>>>(cg, n_c, s.m, s.r, s.d, mask, dAT, dG,
                                                         dBT, ds);
  note_launches(1);
  WINO_CUDA_TRY(cudaGetLastError());
  WINO_CUDA_TRY(cudaMemcpyAsync(AT, dAT, nAT * sizeof(double), cudaMemcpyDeviceToHost, st));
  WINO_CUDA_TRY(cudaMemcpyAsync(G, dG, nG * sizeof(double), cudaMemcpyDeviceToHost, st));
  WINO_CUDA_TRY(cudaMemcpyAsync(BT, dBT, nBT * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (singular)
    WINO_CUDA_TRY(cudaMemcpyAsync(singular, ds, n_c, cudaMemcpyDeviceToHost, st));
  WINO_CUDA_TRY(cudaStreamSynchronize(st));
  return WINO_OK;
}

}  // namespace wino
