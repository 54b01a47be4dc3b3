// abi.cu -- the C ABI front (include/wino.h): argument validation, host
// FP64 matrix construction, scratch management, dispatch to the kernels.
// No arithmetic of the method runs here except the matrix construction
// (Sec. 4.1-4.2), which the paper and the ABI place on the host in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/wino.h"
#include "common.cuh"

namespace wino {

static thread_local std::string g_last_error = "";

void set_error(const std::string& msg) { g_last_error = msg; }

static std::atomic<unsigned long long> g_launches{0};
void note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
            ") in " + what);
  return e == cudaErrorMemoryAllocation ? WINO_ENOMEM : WINO_ECUDA;
}

// ---------------------------------------------------------------------------
// Scratch: grow-only device buffers per (device, slot).  A caller-provided
// workspace (wino_set_workspace) replaces the layer slot.
// ---------------------------------------------------------------------------
namespace {
constexpr int kMaxDev = 16;
struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};
std::mutex g_scratch_mu;
Scratch g_scratch[kMaxDev][kNumScratch];
void* g_user_ws = nullptr;
size_t g_user_ws_bytes = 0;
int g_dev_ok[kMaxDev] = {0};  // 0 unknown, 1 ok, -1 not ok
int* g_wait_flag[kMaxDev] = {nullptr};
}  // namespace

int scratch_get(int slot, size_t bytes, void** ptr) {
  int dev = 0;
  WINO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) {
    set_error("device index out of range");
    return WINO_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  Scratch& s = g_scratch[dev][slot];
  if (s.bytes < bytes) {
    if (s.ptr) {
      // the previous buffer may still be in use by queued work
      WINO_CUDA_TRY(cudaDeviceSynchronize());
      WINO_CUDA_TRY(cudaFree(s.ptr));
      s.ptr = nullptr;
      s.bytes = 0;
    }
    size_t want = bytes + bytes / 8 + 256;
    cudaError_t e = cudaMalloc(&s.ptr, want);
    if (e != cudaSuccess) {
      s.ptr = nullptr;
      (void)cudaGetLastError();
      set_error("could not allocate " + std::to_string(want) + " bytes of device scratch");
      return WINO_ENOMEM;
    }
    s.bytes = want;
  }
  *ptr = s.ptr;
  return WINO_OK;
}

int side_stream(cudaStream_t* aux, cudaEvent_t* fork, cudaEvent_t* join) {
  static cudaStream_t streams[kMaxDev];
  static cudaEvent_t forks[kMaxDev], joins[kMaxDev];
  static bool made[kMaxDev] = {false};
  static std::mutex mu;
  int dev = 0;
  WINO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) {
    set_error("device index out of range");
    return WINO_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!made[dev]) {
    WINO_CUDA_TRY(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
    WINO_CUDA_TRY(cudaEventCreateWithFlags(&forks[dev], cudaEventDisableTiming));
    WINO_CUDA_TRY(cudaEventCreateWithFlags(&joins[dev], cudaEventDisableTiming));
    made[dev] = true;
  }
  *aux = streams[dev];
  *fork = forks[dev];
  *join = joins[dev];
  return WINO_OK;
}

int wait_error_flag(int** ptr) {
  int* (&flags)[kMaxDev] = g_wait_flag;
  int dev = 0;
  WINO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) {
    set_error("device index out of range");
    return WINO_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!flags[dev]) {
    int* p = nullptr;
    WINO_CUDA_TRY(cudaMalloc(&p, sizeof(int)));
    WINO_CUDA_TRY(cudaMemset(p, 0, sizeof(int)));
    flags[dev] = p;
  }
  *ptr = flags[dev];
  return WINO_OK;
}

static int check_device() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    set_error("no CUDA device available");
    return WINO_EUNSUPPORTED;
  }
  if (dev < 0 || dev >= kMaxDev) return WINO_EUNSUPPORTED;
  if (g_dev_ok[dev] == 0) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
      (void)cudaGetLastError();
      g_dev_ok[dev] = -1;
    } else {
      g_dev_ok[dev] = (p.major == 10 && p.minor == 3) ? 1 : -1;
    }
  }
  if (g_dev_ok[dev] != 1) {
    set_error("this library is built for sm_103 (GB300) only");
    return WINO_EUNSUPPORTED;
  }
  return WINO_OK;
}

// Validates a point set (alpha values, exactly one +inf) and writes the
// alpha - 1 sorted finite points to fin (never more).  Returns WINO_OK /
// WINO_EINVAL.
static int canonical_points(const double* points, int alpha, double* fin) {
  if (!points) {
    set_error("points is NULL");
    return WINO_EINVAL;
  }
  int n_inf = 0, nf = 0;
  for (int i = 0; i < alpha; ++i) {
    double p = points[i];
    if (isnan(p) || (isinf(p) && p < 0)) {
      set_error("points must be finite or +INFINITY");
      return WINO_EINVAL;
    }
    if (isinf(p)) {
      ++n_inf;
    } else {
      if (nf == alpha - 1) {
        set_error("exactly one point must be +INFINITY");
        return WINO_EINVAL;
      }
      fin[nf++] = p;
    }
  }
  if (n_inf != 1) {
    set_error("exactly one point must be +INFINITY");
    return WINO_EINVAL;
  }
  sort_points(fin, nf);
  return WINO_OK;
}

static int build_layer_mats(const double* points, int m, int r, LayerMats* M) {
  if (m < 1 || r < 1 || r > kMaxR || m + r - 1 > kMaxAlpha || m + r - 1 < 2) {
    set_error("unsupported (m, r): need m >= 1, 1 <= r <= 7, m + r - 1 <= 12");
    return WINO_EINVAL;
  }
  const int alpha = m + r - 1;
  double fin[kMaxAlpha];
  int st = canonical_points(points, alpha, fin);
  if (st != WINO_OK) return st;
  double AT[kMaxAlpha * kMaxAlpha], G[kMaxAlpha * kMaxR], BT[kMaxAlpha * kMaxAlpha];
  if (!build_matrices<double>(fin, m, r, AT, G, BT)) {
    set_error("two finite points coincide (singular Vandermonde system)");
    return WINO_ESINGULAR;
  }
  memset(M, 0, sizeof(*M));
  for (int i = 0; i < m * alpha; ++i) M->AT[i] = (float)AT[i];
  for (int i = 0; i < alpha * r; ++i) M->G[i] = (float)G[i];
  for (int i = 0; i < alpha * alpha; ++i) M->BT[i] = (float)BT[i];
  M->m = m;
  M->r = r;
  M->alpha = alpha;
  return WINO_OK;
}

static int make_geom(int dim, int N, int C, int K, int H, int W, int pad, int m, int r,
                     LayerGeom* g) {
  if (N < 0 || C < 1 || K < 1 || W < 1 || H < 1 || pad < 0 || m < 1 || r < 1) {
    set_error("invalid layer shape");
    return WINO_EINVAL;
  }
  g->dim = dim;
  g->N = N;
  g->C = C;
  g->K = K;
  g->H = (dim == 1) ? 1 : H;
  g->W = W;
  g->pad = pad;
  g->Wo = W + 2 * pad - r + 1;
  g->Ho = (dim == 1) ? 1 : H + 2 * pad - r + 1;
  if (g->Wo < 1 || g->Ho < 1) {
    set_error("kernel larger than the padded input");
    return WINO_EINVAL;
  }
  g->tw = (g->Wo + m - 1) / m;
  g->th = (dim == 1) ? 1 : (g->Ho + m - 1) / m;
  g->T = (int64_t)N * g->th * g->tw;
  const int alpha = m + r - 1;
  g->F = (dim == 1) ? alpha : alpha * alpha;
  return WINO_OK;
}

}  // namespace wino

using namespace wino;

extern "C" {

int wino_make_matrices(const double* points, int m, int r, double* AT, double* G, double* BT) {
  if (!AT || !G || !BT) {
    set_error("output pointer is NULL");
    return WINO_EINVAL;
  }
  if (m < 1 || r < 1 || m + r - 1 < 2 || m + r - 1 > WINO_MAX_ALPHA) {
    set_error("need m >= 1, r >= 1, 2 <= m + r - 1 <= 12");
    return WINO_EINVAL;
  }
  const int alpha = m + r - 1;
  double fin[kMaxAlpha];
  int st = canonical_points(points, alpha, fin);
  if (st != WINO_OK) return st;
  if (!build_matrices<double>(fin, m, r, AT, G, BT)) {
    set_error("two finite points coincide (singular Vandermonde system)");
    return WINO_ESINGULAR;
  }
  return WINO_OK;
}

static int conv_common(int dim, const void* x, const void* w, void* y, int N, int C, int K,
                       int H, int W, int pad, const double* points, int m, int r, int dtype,
                       void* stream) {
  if (dtype < WINO_F32 || dtype > WINO_SPLIT_BF16X6) {
    set_error("unknown dtype");
    return WINO_EINVAL;
  }
  LayerMats M;
  int st = build_layer_mats(points, m, r, &M);
  if (st != WINO_OK) return st;
  LayerGeom g;
  st = make_geom(dim, N, C, K, H, W, pad, m, r, &g);
  if (st != WINO_OK) return st;
  if (N == 0) return WINO_OK;
  if (!x || !w || !y) {
    set_error("x, w and y must be device pointers");
    return WINO_EINVAL;
  }
  st = check_device();
  if (st != WINO_OK) return st;
  size_t need = layer_workspace_bytes(g, dtype);
  void* ws = nullptr;
  if (g_user_ws) {
    if (g_user_ws_bytes < need) {
      set_error("caller workspace too small: need " + std::to_string(need) + " bytes");
      return WINO_ENOMEM;
    }
    ws = g_user_ws;
  } else {
    st = scratch_get(kScratchLayer, need, &ws);
    if (st != WINO_OK) return st;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == WINO_F32)
    return layer_forward_f32((const float*)x, (const float*)w, (float*)y, g, M, ws, need, s);
  return layer_forward_tc((const float*)x, (const float*)w, (float*)y, g, M, dtype, ws, need, s);
}

int wino_conv1d(const void* x, const void* w, void* y, int N, int C, int K, int L, int pad,
                const double* points, int m, int r, int dtype, void* cuda_stream) {
  return conv_common(1, x, w, y, N, C, K, 1, L, pad, points, m, r, dtype, cuda_stream);
}

int wino_conv2d(const void* x, const void* w, void* y, int N, int C, int K, int H, int W,
                int pad, const double* points, int m, int r, int dtype, void* cuda_stream) {
  return conv_common(2, x, w, y, N, C, K, H, W, pad, points, m, r, dtype, cuda_stream);
}

size_t wino_workspace_bytes(int N, int C, int K, int H, int W, int m, int r, int dtype) {
  LayerGeom g;
  if (make_geom(2, N, C, K, H, W, 1, m, r, &g) != WINO_OK) return 0;
  return layer_workspace_bytes(g, dtype);
}

int wino_set_workspace(void* dev_ptr, size_t bytes) {
  if ((dev_ptr == nullptr) != (bytes == 0)) {
    set_error("workspace pointer and size must be both set or both zero");
    return WINO_EINVAL;
  }
  g_user_ws = dev_ptr;
  g_user_ws_bytes = bytes;
  return WINO_OK;
}

int wino_direct_conv_f64(const void* x, const void* w, void* y64, int dim, int N, int C, int K,
                         int H, int W, int pad, int r, void* cuda_stream) {
  if (dim != 1 && dim != 2) {
    set_error("dim must be 1 or 2");
    return WINO_EINVAL;
  }
  LayerGeom g;
  int st = make_geom(dim, N, C, K, H, W, pad, 1, r, &g);
  if (st != WINO_OK) return st;
  if (N == 0) return WINO_OK;
  if (!x || !w || !y64) {
    set_error("x, w and y64 must be device pointers");
    return WINO_EINVAL;
  }
  st = check_device();
  if (st != WINO_OK) return st;
  return direct_conv_f64((const float*)x, (const float*)w, (double*)y64, dim, N, C, K, g.H, W,
                         pad, r, (cudaStream_t)cuda_stream);
}

int wino_error_stats(const void* yhat_f32, const void* y_f64, int64_t n, double* out4,
                     void* cuda_stream) {
  if (!out4 || n < 0 || (n > 0 && (!yhat_f32 || !y_f64))) {
    set_error("invalid arguments to wino_error_stats");
    return WINO_EINVAL;
  }
  if (n == 0) {
    out4[0] = out4[1] = out4[2] = out4[3] = 0.0;
    return WINO_OK;
  }
  int st = check_device();
  if (st != WINO_OK) return st;
  return error_stats((const float*)yhat_f32, (const double*)y_f64, n, out4,
                     (cudaStream_t)cuda_stream);
}

int wino_error_sweep(const double* c_grid, int n_c, const wino_size* sizes, int n_sizes,
                     const unsigned char* subsets, int n_subsets, int trials,
                     unsigned long long seed, double* err_out, void* cuda_stream) {
  return wino_error_sweep_order(c_grid, n_c, sizes, n_sizes, subsets, n_subsets, trials, seed,
                                WINO_ORDER_FMA, err_out, cuda_stream);
}

int wino_error_sweep_order(const double* c_grid, int n_c, const wino_size* sizes, int n_sizes,
                           const unsigned char* subsets, int n_subsets, int trials,
                           unsigned long long seed, int order, double* err_out,
                           void* cuda_stream) {
  if (order < WINO_ORDER_FMA || order > WINO_ORDER_HUFFMAN_MIXED) {
    set_error("order must be WINO_ORDER_FMA, WINO_ORDER_HUFFMAN or WINO_ORDER_HUFFMAN_MIXED");
    return WINO_EINVAL;
  }
  if (!c_grid || !sizes || !subsets || !err_out || n_c < 1 || n_sizes < 1 || n_subsets < 1 ||
      trials < 1 || trials > (1 << 20)) {
    set_error("invalid sweep arguments (counts must be >= 1, trials <= 2^20)");
    return WINO_EINVAL;
  }
  for (int i = 0; i < n_c; ++i)
    if (!(c_grid[i] > 0.0) || isinf(c_grid[i])) {
      set_error("c values must be finite and > 0");
      return WINO_EINVAL;
    }
  for (int s = 0; s < n_sizes; ++s) {
    const wino_size& z = sizes[s];
    if ((z.dim != 1 && z.dim != 2) || z.m < 1 || z.r < 1 || z.m + z.r - 1 > 10 ||
        z.m + z.r - 1 < 3 || !(z.d > 0.0) || isinf(z.d)) {
      set_error("sweep sizes need dim in {1,2}, 3 <= m + r - 1 <= 10, d > 0");
      return WINO_EINVAL;
    }
  }
  int st = check_device();
  if (st != WINO_OK) return st;
  return error_sweep(c_grid, n_c, reinterpret_cast<const SweepSize*>(sizes), n_sizes, subsets,
                     n_subsets, trials, seed, order, err_out, (cudaStream_t)cuda_stream);
}

int wino_pointset_error(int dim, int m, int r, const double* points, int n_sets, int trials,
                        unsigned long long seed, double* err_out, void* cuda_stream) {
  return wino_pointset_error_order(dim, m, r, points, n_sets, trials, seed, WINO_ORDER_FMA,
                                   err_out, cuda_stream);
}

int wino_pointset_error_order(int dim, int m, int r, const double* points, int n_sets,
                              int trials, unsigned long long seed, int order, double* err_out,
                              void* cuda_stream) {
  const int alpha = m + r - 1;
  if (order < WINO_ORDER_FMA || order > WINO_ORDER_HUFFMAN_MIXED) {
    set_error("order must be WINO_ORDER_FMA, WINO_ORDER_HUFFMAN or WINO_ORDER_HUFFMAN_MIXED");
    return WINO_EINVAL;
  }
  if (!points || !err_out || n_sets < 1 || trials < 1 || trials > (1 << 20) ||
      (dim != 1 && dim != 2) || m < 1 || r < 1 || alpha < 3 || alpha > 10) {
    set_error("invalid point-set sweep arguments");
    return WINO_EINVAL;
  }
  std::vector<double> sorted((size_t)n_sets * (alpha - 1));
  for (int q = 0; q < n_sets; ++q) {
    double fin[kMaxAlpha];
    int st = canonical_points(points + (size_t)q * alpha, alpha, fin);
    if (st != WINO_OK) return st;
    for (int i = 0; i < alpha - 1; ++i) sorted[(size_t)q * (alpha - 1) + i] = fin[i];
  }
  int st = check_device();
  if (st != WINO_OK) return st;
  return pointset_error(dim, m, r, sorted.data(), n_sets, trials, seed, order, err_out,
                        (cudaStream_t)cuda_stream);
}

int wino_pointset_error_kron(int m, int r, const double* points, int n_sets, int trials,
                             unsigned long long seed, int pairwise, double* err_out,
                             void* cuda_stream) {
  const int alpha = m + r - 1;
  if (!points || !err_out || n_sets < 1 || n_sets > (1 << 20) || trials < 1 ||
      trials > (1 << 20) || m < 1 || r < 1 || alpha < 3 || alpha > 10) {
    set_error("invalid Kronecker point-set arguments");
    return WINO_EINVAL;
  }
  std::vector<double> sorted((size_t)n_sets * (alpha - 1));
  for (int q = 0; q < n_sets; ++q) {
    double fin[kMaxAlpha];
    int st = canonical_points(points + (size_t)q * alpha, alpha, fin);
    if (st != WINO_OK) return st;
    for (int i = 0; i < alpha - 1; ++i) sorted[(size_t)q * (alpha - 1) + i] = fin[i];
  }
  int st = check_device();
  if (st != WINO_OK) return st;
  return pointset_error_kron(m, r, sorted.data(), n_sets, trials, seed, pairwise, err_out,
                             (cudaStream_t)cuda_stream);
}

int wino_instance_matrices(const double* c_grid, int n_c, wino_size size, unsigned mask,
                           double* AT, double* G, double* BT, unsigned char* singular,
                           void* cuda_stream) {
  if (!c_grid || n_c < 1 || !AT || !G || !BT) {
    set_error("invalid arguments to wino_instance_matrices");
    return WINO_EINVAL;
  }
  const int alpha = size.m + size.r - 1;
  if (size.m < 1 || size.r < 1 || alpha < 3 || alpha > 10 || !(size.d > 0.0)) {
    set_error("need 3 <= m + r - 1 <= 10 and d > 0");
    return WINO_EINVAL;
  }
  double probe[kMaxAlpha];
  if (mask_points(mask, alpha, 1.5, size.d, probe) < 0) {
    set_error("mask invalid for this size");
    return WINO_EINVAL;
  }
  for (int i = 0; i < n_c; ++i)
    if (!(c_grid[i] > 0.0) || isinf(c_grid[i])) {
      set_error("c values must be finite and > 0");
      return WINO_EINVAL;
    }
  int st = check_device();
  if (st != WINO_OK) return st;
  SweepSize s{size.dim, size.m, size.r, size.d};
  return instance_matrices(c_grid, n_c, s, mask, AT, G, BT, singular, (cudaStream_t)cuda_stream);
}

unsigned long long wino_kernel_launches(void) { return g_launches.load(); }

const char* wino_last_error(void) { return g_last_error.c_str(); }

int wino_device_ok(void) { return check_device() == WINO_OK ? 1 : 0; }

int wino_wait_error(int* flag) {
  if (!flag) {
    set_error("flag is NULL");
    return WINO_EINVAL;
  }
  int st = check_device();
  if (st != WINO_OK) return st;
  int* d = nullptr;
  st = wait_error_flag(&d);
  if (st != WINO_OK) return st;
  WINO_CUDA_TRY(cudaDeviceSynchronize());
  WINO_CUDA_TRY(cudaMemcpy(flag, d, sizeof(int), cudaMemcpyDeviceToHost));
  WINO_CUDA_TRY(cudaMemset(d, 0, sizeof(int)));
  return WINO_OK;
}

int wino_wait_probe(int polls, long long* elapsed_ns, void* cuda_stream) {
  if (!elapsed_ns || polls < 1) {
    set_error("elapsed_ns is NULL or polls < 1");
    return WINO_EINVAL;
  }
  int st = check_device();
  if (st != WINO_OK) return st;
  return wait_probe(polls, elapsed_ns, (cudaStream_t)cuda_stream);
}

void wino_shutdown(void) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    (void)cudaGetLastError();
    return;
  }
  for (int d = 0; d < kMaxDev; ++d)
    for (int s = 0; s < kNumScratch; ++s)
      if (g_scratch[d][s].ptr) {
        if (cudaSetDevice(d) == cudaSuccess) {
          (void)cudaDeviceSynchronize();
          (void)cudaFree(g_scratch[d][s].ptr);
        }
        g_scratch[d][s].ptr = nullptr;
        g_scratch[d][s].bytes = 0;
      }
  for (int d = 0; d < kMaxDev; ++d)
    if (g_wait_flag[d]) {
      if (cudaSetDevice(d) == cudaSuccess) (void)cudaFree(g_wait_flag[d]);
      g_wait_flag[d] = nullptr;
    }
  (void)cudaSetDevice(cur);
  (void)cudaGetLastError();
}

}  // extern "C"
