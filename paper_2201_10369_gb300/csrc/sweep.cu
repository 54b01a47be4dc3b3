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
//                    tile, stores the trial record (sweep_eval.cuh) and a
//                    per-block FP64 partial sum of |y|;
//   k_sweep_ysum     fixed-order total of the partials -> sum_t ||y_t||_1;
//   k_sweep_eval     one warp per (mask, 32 consecutive c): each lane builds
//                    its instance's matrices in FP64, rounds them once to
//                    FP32 into registers and runs all trials with the FP32
//                    Winograd tile; trial records are warp-uniform loads.
//                    A size with too few instances to fill the GPU spreads
//                    each instance's trial chunks over several warps
//                    (k_sweep_combine adds their partials in fixed order).
// The FP32 tile follows the library's fixed operation order (fmaf over the
// inner index ascending, one rounded Hadamard multiply), so yhat is
// bit-identical to any implementation of the same order.  sweep_plan.cu
// runs the same evaluation as one persistent launch over all sizes.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/wino.h"
#include "common.cuh"
#include "sweep_eval.cuh"

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
  // block partial of |y| (warp shuffle, then the warps' sums in order)
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

int sweep_prepare(float* rec, double* partial, double* ysum, int dim, int m, int r, int trials,
                  uint64_t seed, cudaStream_t st) {
  const int nb = sweep_prepare_blocks(trials);
  {
    ProfScope ps(kKSweepPrep, st);
    k_sweep_prepare<<<nb, 256, 0, st>>>(rec, partial, dim, m, r, trials,
                                        sweep_rec_width(dim, m, r), seed);
  }
  k_sweep_ysum<<<1, 32, 0, st>>>(partial, nb, ysum);
  note_launches(2);
  WINO_CUDA_TRY(cudaGetLastError());
  return WINO_OK;
}

// One warp per (valid mask, block of 32 c values, chunk group); lanes own
// instances.  split == 1: each lane runs every trial and writes its error to
// err.  split > 1: the trial chunks are spread over `split` warps of ch_per
// chunks each, which write partial sums to part (chunk stride n_out, the
// size of the err block); k_sweep_combine turns them into errors.
template <int DIM, int M, int R>
__global__ void __launch_bounds__(128) k_sweep_eval(const float* __restrict__ rec, int trials,
                                                    const double* __restrict__ c_grid, int n_c,
                                                    double d, const MaskList masks,
                                                    const double* __restrict__ ysum,
                                                    double* __restrict__ err, int split,
                                                    int ch_per, double* __restrict__ part,
                                                    int64_t n_out) {
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
  lane_eval<DIM, M, R>(rec, trials, masks.mask[qv], c, d, ch0, ch1, *ysum, split > 1,
                       split == 1 ? err + o : part + o, n_out, active);
}

// err[i] = (sum over chunks ascending of part[ch * stride + i]) / ysum of the
// instance's size.
__global__ void k_sweep_combine(const double* __restrict__ part, int n_chunks, int64_t stride,
                                int64_t n, const unsigned char* __restrict__ size_of,
                                const double* __restrict__ ysum, double* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double num = 0.0;
  for (int ch = 0; ch < n_chunks; ++ch) num += part[(int64_t)ch * stride + i];
  err[i] = num / ysum[size_of ? size_of[i] : 0];
}

int sweep_combine(const double* part, int n_chunks, int64_t stride, int64_t n,
                  const unsigned char* size_of, const double* ysum, double* err, cudaStream_t st) {
  if (n <= 0) return WINO_OK;
  k_sweep_combine<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, n_chunks, stride, n, size_of,
                                                              ysum, err);
  note_launches(1);
  WINO_CUDA_TRY(cudaGetLastError());
  return WINO_OK;
}

// The warps a size's launch aims for when its sizes run beside each other
// on the internal streams: an eighth of sweep_target_warps() (four warps
// per SM).  Splitting an instance's chunks over more warps rebuilds its FP64
// matrices in each of them; on the full grid the split targets 1/2, 1/4,
// 1/8, 1/16, 1/32, 1/64 of sweep_target_warps() and no split measured
// 8.21, 8.01, 7.79, 7.88, 8.10, 9.0 and 9.3 ms (1/1: 8.49 ms).
int sweep_split_warps() { return sweep_target_warps() / 8; }

int sweep_target_warps() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      (void)cudaGetLastError();
      sms = 1;
    }
  }
  // 8 resident warps per SM (2 CTAs x 4 warps at the sweep's register use),
  // four rounds of them
  return sms * 8 * 4;
}

static EvalFn eval_kernel(int dim, int m, int r) {
#define WINO_EVAL_CASE(I, D, MM, RR) \
  if (dim == D && m == MM && r == RR) return k_sweep_eval<D, MM, RR>;
  WINO_SWEEP_SIZES(WINO_EVAL_CASE)
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

// Auxiliary streams of the per-size sweep (per device, created on first
// use): the sizes' evaluation launches are spread over them so that one
// size's last, partly filled wave overlaps the next size's work; the
// caller's stream forks to them after the trial records and joins them
// before the results are copied.  (Full grid: 2, 4 and 6 streams measured
// 8.5, 8.4 and 7.85 ms against 7.8 ms for three.)
constexpr int kSweepStreams = 3;
static int sweep_streams(cudaStream_t** aux, cudaEvent_t** ev) {
  static cudaStream_t streams[16][kSweepStreams];
  static cudaEvent_t events[16][kSweepStreams + 1];
  static bool made[16] = {false};
  static std::mutex mu;
  int dev = 0;
  WINO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 16) {
    set_error("device index out of range");
    return WINO_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!made[dev]) {
    for (int i = 0; i < kSweepStreams; ++i)
      WINO_CUDA_TRY(cudaStreamCreateWithFlags(&streams[dev][i], cudaStreamNonBlocking));
    for (int i = 0; i <= kSweepStreams; ++i)
      WINO_CUDA_TRY(cudaEventCreateWithFlags(&events[dev][i], cudaEventDisableTiming));
    made[dev] = true;
  }
  *aux = streams[dev];
  *ev = events[dev];
  return WINO_OK;
}

int error_sweep(const double* c_grid, int n_c, const SweepSize* sizes, int n_sizes,
                const unsigned char* subsets, int n_subsets, int trials, unsigned long long seed,
                int order, double* err_out, cudaStream_t st) {
  std::vector<size_t> rec_off(n_sizes);
  size_t rec_total = 0;
  const int nb_prep = sweep_prepare_blocks(trials);
  for (int s = 0; s < n_sizes; ++s) {
    if (!eval_kernel(sizes[s].dim, sizes[s].m, sizes[s].r) &&
        !sweep_wide(sizes[s].dim, sizes[s].m, sizes[s].r)) {
      set_error("sweep size not compiled: 1D r=3 m=2..8, 1D r=5 m=2..6, 2D r=3 m=2..8, "
                "2D r=5 m=2..4");
      return WINO_EUNSUPPORTED;
    }
    rec_off[s] = rec_total;
    rec_total += (size_t)trials * sweep_rec_width(sizes[s].dim, sizes[s].m, sizes[s].r);
  }
  // per size: its valid masks and, when its items alone cannot fill the
  // GPU, how many warps share each instance's trial chunks
  std::vector<MaskList> ml(n_sizes);
  std::vector<int> split(n_sizes, 1);
  const int nblk = (n_c + 31) / 32;
  const int n_chunks = trial_chunks(trials);
  // sizes to auxiliary streams, longest first to the least loaded (the
  // sizes of one stream run in order, so they can share a chunk buffer)
  std::vector<int> lane(n_sizes, 0), by_cost(n_sizes);
  {
    std::vector<double> cost(n_sizes), load(kSweepStreams, 0.0);
    for (int s = 0; s < n_sizes; ++s) {
      by_cost[s] = s;
      cost[s] = sweep_trial_flops(sizes[s].dim, sizes[s].m, sizes[s].r) *
                valid_masks(sizes[s], subsets, n_subsets).n;
    }
    std::stable_sort(by_cost.begin(), by_cost.end(),
                     [&](int a, int b2) { return cost[a] > cost[b2]; });
    for (int s : by_cost) {
      int l = 0;
      for (int i = 1; i < kSweepStreams; ++i)
        if (load[i] < load[l]) l = i;
      lane[s] = l;
      load[l] += cost[s];
    }
  }
  size_t n_part = 0;
  for (int s = 0; s < n_sizes; ++s) {
    ml[s] = valid_masks(sizes[s], subsets, n_subsets);
    const int items = ml[s].n * nblk;
    if (order == 0 && !sweep_wide(sizes[s].dim, sizes[s].m, sizes[s].r) && items > 0 &&
        items < sweep_split_warps())
      split[s] = std::min(n_chunks, (sweep_split_warps() + items - 1) / items);
    if (split[s] > 1) n_part = std::max(n_part, (size_t)n_chunks * n_subsets * n_c);
  }
  // scratch layout: records | partials | ysum | c_grid | err | chunk partials
  const size_t n_err = (size_t)n_sizes * n_subsets * n_c;
  size_t off_part = rec_total * sizeof(float);
  off_part = (off_part + 255) & ~(size_t)255;
  size_t off_ysum = off_part + (size_t)n_sizes * nb_prep * sizeof(double);
  off_ysum = (off_ysum + 255) & ~(size_t)255;
  size_t off_c = off_ysum + (size_t)n_sizes * sizeof(double);
  off_c = (off_c + 255) & ~(size_t)255;
  size_t off_err = off_c + (size_t)n_c * sizeof(double);
  off_err = (off_err + 255) & ~(size_t)255;
  size_t off_chunk = off_err + n_err * sizeof(double);
  off_chunk = (off_chunk + 255) & ~(size_t)255;
  const size_t total = off_chunk + (size_t)kSweepStreams * n_part * sizeof(double);
  void* base = nullptr;
  int rc = scratch_get(kScratchSweep, total, &base);
  if (rc != WINO_OK) return rc;
  char* b = (char*)base;
  float* rec = (float*)b;
  double* part = (double*)(b + off_part);
  double* ysum = (double*)(b + off_ysum);
  double* cg = (double*)(b + off_c);
  double* err = (double*)(b + off_err);
  double* chunk = (double*)(b + off_chunk);

  WINO_CUDA_TRY(cudaMemcpyAsync(cg, c_grid, n_c * sizeof(double), cudaMemcpyHostToDevice, st));
  for (int s = 0; s < n_sizes; ++s) {
    rc = sweep_prepare(rec + rec_off[s], part + (size_t)s * nb_prep, ysum + s, sizes[s].dim,
                       sizes[s].m, sizes[s].r, trials, seed, st);
    if (rc != WINO_OK) return rc;
  }
  cudaStream_t* aux = nullptr;
  cudaEvent_t* ev = nullptr;
  rc = sweep_streams(&aux, &ev);
  if (rc != WINO_OK) return rc;
  {
    // profiled as one phase, fork to join (its launches overlap)
    ProfScope ps(order != 0 ? kKSweepOrder : kKSweepEval, st);
    WINO_CUDA_TRY(cudaEventRecord(ev[kSweepStreams], st));
    for (int i = 0; i < kSweepStreams; ++i)
      WINO_CUDA_TRY(cudaStreamWaitEvent(aux[i], ev[kSweepStreams], 0));
    for (int s : by_cost) {
      if (ml[s].n == 0) continue;
      const cudaStream_t st_s = aux[lane[s]];
      double* chunk_s = chunk + (size_t)lane[s] * n_part;
      const int64_t n_out = (int64_t)n_subsets * n_c;
      const int ch_per = (n_chunks + split[s] - 1) / split[s];
      const int sp = (n_chunks + ch_per - 1) / ch_per;  // groups actually holding chunks
      const int64_t warps = (int64_t)ml[s].n * nblk * (split[s] > 1 ? sp : 1);
      const int warps_per_block = 4;
      const unsigned grid = (unsigned)((warps + warps_per_block - 1) / warps_per_block);
      double* es = err + (size_t)s * n_out;
      // the Huffman orders, and the wide sizes in any order: one warp per
      // instance (sweep_order.cuh)
      if (order != 0 || sweep_wide(sizes[s].dim, sizes[s].m, sizes[s].r)) {
        rc = order_sweep_launch(order, sizes[s], rec + rec_off[s], trials, cg, n_c, ml[s],
                                ysum + s, es, st_s);
        if (rc != WINO_OK) break;
        continue;
      }
      EvalFn fn = eval_kernel(sizes[s].dim, sizes[s].m, sizes[s].r);
      fn<<<grid, 32 * warps_per_block, 0, st_s>>>(rec + rec_off[s], trials, cg, n_c, sizes[s].d,
                                                   ml[s], ysum + s, es, split[s] > 1 ? sp : 1,
                                                   ch_per, chunk_s, n_out);
      note_launches(1);
      if (split[s] > 1) {
        rc = sweep_combine(chunk_s, n_chunks, n_out, n_out, nullptr, ysum + s, es, st_s);
        if (rc != WINO_OK) break;
      }
    }
    // join (also after a failed launch): the caller's stream waits for every
    // auxiliary stream
    for (int i = 0; i < kSweepStreams; ++i) {
      WINO_CUDA_TRY(cudaEventRecord(ev[i], aux[i]));
      WINO_CUDA_TRY(cudaStreamWaitEvent(st, ev[i], 0));
    }
  }
  if (rc != WINO_OK) return rc;
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

// ---------------------------------------------------------------------------
// Explicit point sets (the comparison sets of Tables 7-8, Chebyshev nodes):
// one lane per set, the sweep's trials and summation order.
// ---------------------------------------------------------------------------
template <int DIM, int M, int R>
__global__ void __launch_bounds__(128) k_pointset_eval(const float* __restrict__ rec, int trials,
                                                       const double* __restrict__ pts, int n_sets,
                                                       const double* __restrict__ ysum,
                                                       double* __restrict__ err) {
  constexpr int A = M + R - 1;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = s < n_sets;
  const int ss = active ? s : 0;
  double a[A - 1];
#pragma unroll
  for (int i = 0; i < A - 1; ++i) a[i] = pts[(int64_t)ss * (A - 1) + i];
  Mats<M, R> Mx;
  const bool ok = build_from_points<M, R>(a, Mx);
  lane_eval_mats<DIM, M, R>(Mx, ok, rec, trials, 0, trial_chunks(trials), *ysum, false, err + ss,
                            0, active);
}

static PointsetFn pointset_kernel(int dim, int m, int r) {
#define WINO_PSET_CASE(I, D, MM, RR) \
  if (dim == D && m == MM && r == RR) return k_pointset_eval<D, MM, RR>;
  WINO_SWEEP_SIZES(WINO_PSET_CASE)
#undef WINO_PSET_CASE
  return nullptr;
}

// points: [n_sets][alpha-1] sorted finite points (host); err_out host.
int pointset_error(int dim, int m, int r, const double* sorted, int n_sets, int trials,
                   unsigned long long seed, int order, double* err_out, cudaStream_t st) {
  PointsetFn fn = pointset_kernel(dim, m, r);
  const bool wide = sweep_wide(dim, m, r);
  if (!fn && !wide) {
    set_error("point-set sizes: 1D r=3 m=2..8, 1D r=5 m=2..6, 2D r=3 m=2..8, 2D r=5 m=2..4");
    return WINO_EUNSUPPORTED;
  }
  const int A = m + r - 1;
  const int nb = sweep_prepare_blocks(trials);
  const size_t rec_b = (size_t)trials * sweep_rec_width(dim, m, r) * sizeof(float);
  size_t o_part = (rec_b + 255) & ~(size_t)255;
  size_t o_ysum = (o_part + (size_t)nb * 8 + 255) & ~(size_t)255;
  size_t o_pts = (o_ysum + 8 + 255) & ~(size_t)255;
  size_t o_err = (o_pts + (size_t)n_sets * (A - 1) * 8 + 255) & ~(size_t)255;
  const size_t total = o_err + (size_t)n_sets * 8;
  void* base = nullptr;
  int rc = scratch_get(kScratchSweep, total, &base);
  if (rc != WINO_OK) return rc;
  char* b = (char*)base;
  float* rec = (float*)b;
  double* part = (double*)(b + o_part);
  double* ysum = (double*)(b + o_ysum);
  double* pts = (double*)(b + o_pts);
  double* err = (double*)(b + o_err);
  WINO_CUDA_TRY(cudaMemcpyAsync(pts, sorted, (size_t)n_sets * (A - 1) * 8,
                                cudaMemcpyHostToDevice, st));
  rc = sweep_prepare(rec, part, ysum, dim, m, r, trials, seed, st);
  if (rc != WINO_OK) return rc;
  if (order != 0 || wide) {
    ProfScope ps(order != 0 ? kKSweepOrder : kKSweepEval, st);
    rc = order_pointset_launch(order, dim, m, r, rec, trials, pts, n_sets, ysum, err, st);
    if (rc != WINO_OK) return rc;
  } else {
    ProfScope ps(kKSweepEval, st);
    fn<<<(n_sets + 127) / 128, 128, 0, st>>>(rec, trials, pts, n_sets, ysum, err);
    note_launches(1);
  }
  WINO_CUDA_TRY(cudaGetLastError());
  WINO_CUDA_TRY(cudaMemcpyAsync(err_out, err, (size_t)n_sets * 8, cudaMemcpyDeviceToHost, st));
  WINO_CUDA_TRY(cudaStreamSynchronize(st));
  return WINO_OK;
}

// ---------------------------------------------------------------------------
// Kronecker-product form of the 2D tile (Sec. 7): with row-major vec,
// vec(G g G^T) = (G (x) G) vec(g), vec(B^T d B) = (B^T (x) B^T) vec(d),
// vec(A^T M A) = (A^T (x) A^T) vec(M).  Kronecker entries: FP64 products of
// the FP64 matrix entries, rounded once to FP32.  Each row is summed with
// fmaf, column ascending, or (pairwise) as rounded products summed pairwise,
// sum(x[0..n)) = sum(x[0..h)) + sum(x[h..n)), h = ceil(n / 2).
// One block per point set (its Kronecker matrices in shared memory); threads
// take trials t = tid, tid + blockDim, ...; per-thread FP64 sums of the
// per-trial FP32 errors, added in thread order.
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ float pairwise_sum(const float* x) {
  if constexpr (N == 1) {
    return x[0];
  } else {
    constexpr int H = (N + 1) / 2;
    return __fadd_rn(pairwise_sum<H>(x), pairwise_sum<N - H>(x + H));
  }
}

// One row of a Kronecker matrix times x: fmaf, column ascending, or (PW)
// rounded products summed pairwise.
template <int COLS, bool PW>
__device__ __forceinline__ float kron_row(const float* __restrict__ k,
                                          const float (&x)[COLS]) {
  if constexpr (PW) {
    float pr[COLS];
#pragma unroll
    for (int c = 0; c < COLS; ++c) pr[c] = __fmul_rn(k[c], x[c]);
    return pairwise_sum<COLS>(pr);
  } else {
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < COLS; ++c) acc = fmaf(k[c], x[c], acc);
    return acc;
  }
}

constexpr int kKronThreads = 64;

template <int M, bool PW>
__global__ void __launch_bounds__(kKronThreads) k_pointset_kron(const float* __restrict__ rec,
                                                                int trials,
                                                                const double* __restrict__ pts,
                                                                const double* __restrict__ ysum,
                                                                double* __restrict__ err) {
  constexpr int R = 3, A = M + R - 1, A2 = A * A, R2 = R * R, M2 = M * M;
  constexpr int PP = A2 + 1;  // a thread's row of Hadamard products (padded)
  using S = SweepShape<2, M, R>;
  __shared__ float KG[A2 * R2], KB[A2 * A2], KA[M2 * A2];
  __shared__ float sp[kKronThreads * PP];
  __shared__ double ATd[M * A], Gd[A * R], BTd[A * A];
  __shared__ double part[kKronThreads];
  __shared__ int s_ok;
  const int set = blockIdx.x, tid = threadIdx.x;
  if (tid == 0) {
    double a[A - 1];
    for (int i = 0; i < A - 1; ++i) a[i] = pts[(int64_t)set * (A - 1) + i];
    s_ok = build_matrices<double>(a, M, R, ATd, Gd, BTd) ? 1 : 0;
  }
  __syncthreads();
  for (int e = tid; e < A2 * R2; e += kKronThreads) {
    const int i = e / (A * R2), j = (e / R2) % A, k = (e % R2) / R, l = e % R;
    KG[e] = __double2float_rn(__dmul_rn(Gd[i * R + k], Gd[j * R + l]));
  }
  for (int e = tid; e < A2 * A2; e += kKronThreads) {
    const int i = e / (A * A2), j = (e / A2) % A, k = (e % A2) / A, l = e % A;
    KB[e] = __double2float_rn(__dmul_rn(BTd[i * A + k], BTd[j * A + l]));
  }
  for (int e = tid; e < M2 * A2; e += kKronThreads) {
    const int a = e / (M * A2), b = (e / A2) % M, i = (e % A2) / A, j = e % A;
    KA[e] = __double2float_rn(__dmul_rn(ATd[a * A + i], ATd[b * A + j]));
  }
  __syncthreads();
  float* my = sp + tid * PP;
  double num = 0.0;
  for (int t = tid; t < trials; t += kKronThreads) {
    const float* rc = rec + (int64_t)t * S::REC;  // [g | d | hi(y) | lo(y)]
    float g[R2], d[A2];
#pragma unroll
    for (int i = 0; i < R2; ++i) g[i] = rc[i];
#pragma unroll
    for (int i = 0; i < A2; ++i) d[i] = rc[R2 + i];
#pragma unroll 1
    for (int i = 0; i < A2; ++i)
      my[i] = __fmul_rn(kron_row<R2, PW>(KG + i * R2, g), kron_row<A2, PW>(KB + i * A2, d));
    float pv[A2];
#pragma unroll
    for (int i = 0; i < A2; ++i) pv[i] = my[i];
    float e = 0.0f;
#pragma unroll 1
    for (int j = 0; j < M2; ++j) {
      const float yj = kron_row<A2, PW>(KA + j * A2, pv);
      e = __fadd_rn(e, abs_err(yj, rc[R2 + A2 + j], rc[R2 + A2 + M2 + j]));
    }
    num += (double)e;
  }
  part[tid] = num;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int q = 0; q < kKronThreads; ++q) tot += part[q];
    err[set] = s_ok ? tot / *ysum : (double)INFINITY;
  }
}

typedef void (*KronFn)(const float*, int, const double*, const double*, double*);

static KronFn kron_kernel(int m, bool pw) {
  switch (m) {
    case 2: return pw ? k_pointset_kron<2, true> : k_pointset_kron<2, false>;
    case 3: return pw ? k_pointset_kron<3, true> : k_pointset_kron<3, false>;
    case 4: return pw ? k_pointset_kron<4, true> : k_pointset_kron<4, false>;
    case 5: return pw ? k_pointset_kron<5, true> : k_pointset_kron<5, false>;
    case 6: return pw ? k_pointset_kron<6, true> : k_pointset_kron<6, false>;
    default: return nullptr;
  }
}

// points: [n_sets][alpha-1] sorted finite points (host); err_out host.
int pointset_error_kron(int m, int r, const double* sorted, int n_sets, int trials,
                        unsigned long long seed, int pairwise, double* err_out,
                        cudaStream_t st) {
  KronFn fn = r == 3 ? kron_kernel(m, pairwise != 0) : nullptr;
  if (!fn) {
    set_error("Kronecker-product form: 2D F(m x m, 3 x 3), m = 2..6");
    return WINO_EUNSUPPORTED;
  }
  const int A = m + r - 1;
  const int nb = sweep_prepare_blocks(trials);
  const size_t rec_b = (size_t)trials * sweep_rec_width(2, m, r) * sizeof(float);
  size_t o_part = (rec_b + 255) & ~(size_t)255;
  size_t o_ysum = (o_part + (size_t)nb * 8 + 255) & ~(size_t)255;
  size_t o_pts = (o_ysum + 8 + 255) & ~(size_t)255;
  size_t o_err = (o_pts + (size_t)n_sets * (A - 1) * 8 + 255) & ~(size_t)255;
  const size_t total = o_err + (size_t)n_sets * 8;
  void* base = nullptr;
  int rc = scratch_get(kScratchSweep, total, &base);
  if (rc != WINO_OK) return rc;
  char* b = (char*)base;
  float* rec = (float*)b;
  double* part = (double*)(b + o_part);
  double* ysum = (double*)(b + o_ysum);
  double* pts = (double*)(b + o_pts);
  double* err = (double*)(b + o_err);
  WINO_CUDA_TRY(cudaMemcpyAsync(pts, sorted, (size_t)n_sets * (A - 1) * 8,
                                cudaMemcpyHostToDevice, st));
  rc = sweep_prepare(rec, part, ysum, 2, m, r, trials, seed, st);
  if (rc != WINO_OK) return rc;
  {
    ProfScope ps(kKSweepEval, st);
    fn<<<n_sets, kKronThreads, 0, st>>>(rec, trials, pts, ysum, err);
    note_launches(1);
  }
  WINO_CUDA_TRY(cudaGetLastError());
  WINO_CUDA_TRY(cudaMemcpyAsync(err_out, err, (size_t)n_sets * 8, cudaMemcpyDeviceToHost, st));
  WINO_CUDA_TRY(cudaStreamSynchronize(st));
  return WINO_OK;
}

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
  if (singular) WINO_CUDA_TRY(cudaMemcpyAsync(singular, ds, n_c, cudaMemcpyDeviceToHost, st));
  WINO_CUDA_TRY(cudaStreamSynchronize(st));
  return WINO_OK;
}

}  // namespace wino
