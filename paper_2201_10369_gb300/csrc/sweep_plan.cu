// sweep_plan.cu -- planned sweep over an explicit list of instances
// (size, mask, c), run as ONE persistent launch captured in a CUDA graph.
//
// Instances of uneven alpha (1D and 2D, m = 2..8, r = 3, 5) are grouped by
// size into work items of 32 (one warp, one instance per lane) and ordered
// by decreasing cost (trials x dense flops per trial: longest first, so the
// last items to start are the cheapest).  A persistent grid of warps pulls
// items from an atomic counter; each item dispatches to the size's
// compile-time evaluator (sweep_eval.cuh).  A size with too few groups of
// 32 to fill the GPU on its own (fewer than four rounds of resident warps)
// gives each of its groups several items, one per range of trial chunks;
// their partial sums are combined in fixed order afterwards, per size, so
// the errors are the same bits either way.  A device-side deadline
// (%globaltimer) lets the kernel stop taking work and report WINO_ETIMEOUT
// instead of running unbounded; there is no spin-wait anywhere.  The graph
// holds the counter/status resets, the trial records of every size
// (k_sweep_prepare), the evaluation and the copies of the results to pinned
// host memory.
//
// Execution modes (the autotuner times them when mode = WINO_SWEEP_AUTO):
//   WINO_SWEEP_PERSISTENT   persistent kernel, 2 CTAs x 4 warps per SM
//   WINO_SWEEP_PERSISTENT3  persistent kernel limited to 168 registers,
//                           3 CTAs x 4 warps per SM
//   WINO_SWEEP_PER_SIZE     one grid launch per size over its items, the
//                           sizes spread over three streams (forked from
//                           and joined back to the plan's stream by
//                           events), so one size's last wave overlaps
//                           the next size's launch
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/wino.h"
#include "common.cuh"
#include "sweep_eval.cuh"

namespace wino {

// 32 instances of one size (sorted positions first .. first + count - 1)
// and the trial chunks [c0, c1) this item runs for them.
struct WorkItem {
  int size, first;
  unsigned short count, pad, c0, c1;
};

struct PlanDev {
  const WorkItem* items;
  int n_items;
  int* counter;
  int* status;
  const unsigned long long* deadline;  // absolute %globaltimer limit, 0 = none
  const double* inst_c;
  const unsigned char* inst_mask;
  const float* rec;
  const int64_t* rec_off;  // per size, floats
  const int* kind;         // per size, index into WINO_SWEEP_SIZES
  const double* dval;      // per size
  const double* ysum;      // per size
  double* err;             // per sorted instance
  double* part;            // chunk partials [chunk][sorted instance] of split sizes
  int64_t n_sorted;
  int trials;
  int n_chunks;            // trial chunks of `trials`
  int split;               // 1: no size is split, every item writes err directly
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int D, int MM, int RR>
__device__ __noinline__ void eval_item_as(const PlanDev& P, const WorkItem& w, int lane) {
  const int i = w.first + lane;
  const bool active = lane < w.count;
  const int ii = active ? i : w.first;
  // an item covering only some trial chunks leaves partial sums
  const bool partial = w.c0 != 0 || w.c1 != P.n_chunks;
  lane_eval<D, MM, RR>(P.rec + P.rec_off[w.size], P.trials, P.inst_mask[ii], P.inst_c[ii],
                       P.dval[w.size], w.c0, w.c1, P.ysum[w.size], partial,
                       partial ? P.part + i : P.err + i, P.n_sorted, active);
}

__device__ __forceinline__ void eval_item(const PlanDev& P, const WorkItem& w, int lane) {
  switch (P.kind[w.size]) {
#define WINO_PLAN_CASE(I, D, MM, RR)      \
  case I:                                 \
    eval_item_as<D, MM, RR>(P, w, lane);  \
    break;
    WINO_SWEEP_SIZES(WINO_PLAN_CASE)
#undef WINO_PLAN_CASE
    default:
      break;
  }
}

// Warp-granular persistent loop: lane 0 takes the next item (or, past the
// deadline, records WINO_ETIMEOUT and stops taking work).
template <int MIN_BLOCKS>
__global__ void __launch_bounds__(128, MIN_BLOCKS) k_sweep_persistent(const PlanDev P) {
  const int lane = threadIdx.x & 31;
  const unsigned long long limit = *P.deadline;
  for (;;) {
    int it = 0;
    if (lane == 0) {
      if (limit != 0ull && global_ns() > limit) {
        atomicExch(P.status, (int)WINO_ETIMEOUT);
        it = P.n_items;
      } else {
        it = atomicAdd(P.counter, 1);
      }
    }
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= P.n_items) return;
    eval_item(P, P.items[it], lane);
  }
}

// One warp per item of one size (no queue): the per-size mode.
template <int D, int MM, int RR>
__global__ void __launch_bounds__(128) k_sweep_items(const PlanDev P, int first_item,
                                                     int n_items) {
  const int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (it >= n_items) return;
  eval_item_as<D, MM, RR>(P, P.items[first_item + it], threadIdx.x & 31);
}

typedef void (*ItemsFn)(const PlanDev, int, int);
static ItemsFn items_kernel(int kind) {
  switch (kind) {
#define WINO_ITEMS_CASE(I, D, MM, RR) \
  case I:                             \
    return k_sweep_items<D, MM, RR>;
    WINO_SWEEP_SIZES(WINO_ITEMS_CASE)
#undef WINO_ITEMS_CASE
    default:
      return nullptr;
  }
}

__global__ void k_read_globaltimer(unsigned long long* out) { *out = global_ns(); }

// Current %globaltimer value of the current device (ns).
static int device_time_ns(unsigned long long* now) {
  static unsigned long long* h = nullptr;
  if (!h) WINO_CUDA_TRY(cudaHostAlloc((void**)&h, sizeof(*h), cudaHostAllocMapped));
  unsigned long long* d = nullptr;
  WINO_CUDA_TRY(cudaHostGetDevicePointer((void**)&d, h, 0));
  k_read_globaltimer<<<1, 1>>>(d);
  note_launches(1);
  WINO_CUDA_TRY(cudaGetLastError());
  WINO_CUDA_TRY(cudaDeviceSynchronize());
  *now = *h;
  return WINO_OK;
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
struct SweepPlan {
  int dev = 0;
  int n_sizes = 0, trials = 0;
  int64_t n_inst = 0;
  unsigned long long seed = 0;
  int mode = WINO_SWEEP_PERSISTENT;
  double max_ms = 0.0;
  std::vector<SweepSize> sizes;
  std::vector<int> kind;
  std::vector<int64_t> order;      // sorted position -> caller's instance index
  unsigned char* size_of = nullptr;  // device: size index per sorted instance
  std::vector<char> invalid;       // per caller instance: mask invalid for its size
  std::vector<WorkItem> items;     // LPT order
  std::vector<int> size_first, size_count;  // items of each size (per-size mode)
  std::vector<int64_t> inst_first, inst_count;  // sorted instances of each size
  std::vector<char> size_split;             // size's items cover chunk ranges
  // device
  void* dbuf = nullptr;
  PlanDev P{};
  int64_t* rec_off_h = nullptr;
  float* rec = nullptr;
  double* part = nullptr;
  double* ysum = nullptr;
  unsigned long long* deadline = nullptr;
  // pinned host staging
  double* err_h = nullptr;
  int* status_h = nullptr;
  unsigned long long* deadline_h = nullptr;
  std::vector<int64_t> rec_off;
  int grid = 0;
  cudaStream_t st = nullptr;
  // per-size mode: the streams the sizes run on, each size's stream, and
  // the fork (kPlanLanes) and join events
  static constexpr int kPlanLanes = 3;
  cudaStream_t lane_st[kPlanLanes] = {};
  cudaEvent_t lane_ev[kPlanLanes + 1] = {};
  std::vector<int> lane;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
};

static void plan_free(SweepPlan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->st) cudaStreamDestroy(p->st);
  for (int i = 0; i < SweepPlan::kPlanLanes; ++i)
    if (p->lane_st[i]) cudaStreamDestroy(p->lane_st[i]);
  for (int i = 0; i <= SweepPlan::kPlanLanes; ++i)
    if (p->lane_ev[i]) cudaEventDestroy(p->lane_ev[i]);
  if (p->dbuf) cudaFree(p->dbuf);
  if (p->err_h) cudaFreeHost(p->err_h);
  if (p->status_h) cudaFreeHost(p->status_h);
  if (p->deadline_h) cudaFreeHost(p->deadline_h);
  (void)cudaGetLastError();
  delete p;
}

// Enqueues the plan's work on `st` (also used for capture).
static int plan_enqueue(SweepPlan* p, int mode, cudaStream_t st) {
  WINO_CUDA_TRY(cudaMemsetAsync(p->P.counter, 0, sizeof(int), st));
  WINO_CUDA_TRY(cudaMemsetAsync(p->P.status, 0, sizeof(int), st));
  WINO_CUDA_TRY(cudaMemcpyAsync(p->deadline, p->deadline_h, sizeof(unsigned long long),
                                cudaMemcpyHostToDevice, st));
  const int nbp = sweep_prepare_blocks(p->trials);
  for (int s = 0; s < p->n_sizes; ++s) {
    int rc = sweep_prepare(p->rec + p->rec_off[s], p->part + (size_t)s * nbp, p->ysum + s,
                           p->sizes[s].dim, p->sizes[s].m, p->sizes[s].r, p->trials, p->seed,
                           st);
    if (rc != WINO_OK) return rc;
  }
  if (!p->items.empty()) {
    ProfScope ps(kKSweepEval, st);
    if (mode == WINO_SWEEP_PER_SIZE) {
      constexpr int L = SweepPlan::kPlanLanes;
      WINO_CUDA_TRY(cudaEventRecord(p->lane_ev[L], st));
      for (int i = 0; i < L; ++i) WINO_CUDA_TRY(cudaStreamWaitEvent(p->lane_st[i], p->lane_ev[L], 0));
      for (int s = 0; s < p->n_sizes; ++s) {
        if (p->size_count[s] == 0) continue;
        ItemsFn fn = items_kernel(p->kind[s]);
        fn<<<(p->size_count[s] + 3) / 4, 128, 0, p->lane_st[p->lane[s]]>>>(
            p->P, p->size_first[s], p->size_count[s]);
        note_launches(1);
      }
      WINO_CUDA_TRY(cudaGetLastError());
      for (int i = 0; i < L; ++i) {
        WINO_CUDA_TRY(cudaEventRecord(p->lane_ev[i], p->lane_st[i]));
        WINO_CUDA_TRY(cudaStreamWaitEvent(st, p->lane_ev[i], 0));
      }
    } else if (mode == WINO_SWEEP_PERSISTENT3) {
      k_sweep_persistent<3><<<p->grid, 128, 0, st>>>(p->P);
      note_launches(1);
    } else {
      k_sweep_persistent<2><<<p->grid, 128, 0, st>>>(p->P);
      note_launches(1);
    }
  }
  WINO_CUDA_TRY(cudaGetLastError());
  for (int s = 0; s < p->n_sizes; ++s) {
    if (!p->size_split[s] || p->inst_count[s] == 0) continue;
    const int64_t f = p->inst_first[s];
    int rc = sweep_combine(p->P.part + f, p->P.n_chunks, p->P.n_sorted, p->inst_count[s],
                           p->size_of + f, p->ysum, p->P.err + f, st);
    if (rc != WINO_OK) return rc;
  }
  WINO_CUDA_TRY(cudaMemcpyAsync(p->err_h, p->P.err, sizeof(double) * (size_t)p->n_inst,
                                cudaMemcpyDeviceToHost, st));
  WINO_CUDA_TRY(
      cudaMemcpyAsync(p->status_h, p->P.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  return WINO_OK;
}

static int plan_grid(int mode) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  cudaError_t e = (mode == WINO_SWEEP_PERSISTENT3)
                      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_persistent<3>,
                                                                      128, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_persistent<2>,
                                                                      128, 0);
  if (e != cudaSuccess || per < 1) per = 1;
  return sms * per;
}

static int plan_capture(SweepPlan* p) {
  if (p->exec) {
    cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
  }
  if (p->graph) {
    cudaGraphDestroy(p->graph);
    p->graph = nullptr;
  }
  p->grid = plan_grid(p->mode);
  WINO_CUDA_TRY(cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal));
  int rc = plan_enqueue(p, p->mode, p->st);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(p->st, &g);
  if (rc != WINO_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  p->graph = g;
  WINO_CUDA_TRY(cudaGraphInstantiate(&p->exec, g, 0));
  return WINO_OK;
}

// Autotuner: captures each mode and times its graph replays on the plan
// itself (best of 2 after a warm-up), keeps the fastest; results are cached
// per plan signature for the life of the process.
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_cache;

static std::string plan_signature(const SweepPlan* p) {
  std::string s = "t" + std::to_string(p->trials) + "n" + std::to_string(p->n_inst);
  for (int i = 0; i < p->n_sizes; ++i)
    s += ":" + std::to_string(p->kind[i]) + "x" + std::to_string(p->size_count[i]);
  return s;
}

static int plan_autotune(SweepPlan* p) {
  const std::string sig = plan_signature(p);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      p->mode = it->second;
      return WINO_OK;
    }
  }
  const int modes[3] = {WINO_SWEEP_PERSISTENT, WINO_SWEEP_PERSISTENT3, WINO_SWEEP_PER_SIZE};
  cudaEvent_t a, b;
  WINO_CUDA_TRY(cudaEventCreate(&a));
  WINO_CUDA_TRY(cudaEventCreate(&b));
  float best = 1e30f;
  int best_mode = WINO_SWEEP_PERSISTENT;
  for (int mi = 0; mi < 3; ++mi) {
    p->mode = modes[mi];
    int rc = plan_capture(p);
    if (rc != WINO_OK) return rc;
    float t_best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      WINO_CUDA_TRY(cudaEventRecord(a, p->st));
      WINO_CUDA_TRY(cudaGraphLaunch(p->exec, p->st));
      WINO_CUDA_TRY(cudaEventRecord(b, p->st));
      WINO_CUDA_TRY(cudaEventSynchronize(b));
      float ms = 0.0f;
      WINO_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
      if (rep > 0) t_best = std::min(t_best, ms);
    }
    if (t_best < best) {
      best = t_best;
      best_mode = modes[mi];
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  p->mode = best_mode;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[sig] = best_mode;
  return WINO_OK;
}

}  // namespace wino

using namespace wino;

extern "C" {

int wino_sweep_plan_create(const wino_size* sizes, int n_sizes, const wino_instance* inst,
                           int64_t n_inst, int trials, unsigned long long seed, int mode,
                           void** plan_out) {
  if (!plan_out || !sizes || n_sizes < 1 || n_sizes > 64 || !inst || n_inst < 1 ||
      n_inst > (int64_t)1 << 30 || trials < 1 || trials > (1 << 20) ||
      mode < WINO_SWEEP_AUTO || mode > WINO_SWEEP_PER_SIZE) {
    set_error("invalid arguments to wino_sweep_plan_create");
    return WINO_EINVAL;
  }
  *plan_out = nullptr;
  SweepPlan* p = new SweepPlan();
  p->n_sizes = n_sizes;
  p->trials = trials;
  p->n_inst = n_inst;
  p->seed = seed;
  p->sizes.resize(n_sizes);
  p->kind.resize(n_sizes);
  for (int s = 0; s < n_sizes; ++s) {
    const wino_size& z = sizes[s];
    p->sizes[s] = SweepSize{z.dim, z.m, z.r, z.d};
    p->kind[s] = sweep_kind(z.dim, z.m, z.r);
    if (p->kind[s] < 0 || !(z.d > 0.0) || isinf(z.d)) {
      plan_free(p);
      set_error("sweep size not compiled (1D r=3 m=2..8, 1D r=5 m=2..6, 2D r=3 m=2..6, 2D r=5 m=2..4) or d <= 0");
      return WINO_EUNSUPPORTED;
    }
  }
  // validate instances, group by size (stable), chunk into warp items
  p->invalid.assign(n_inst, 0);
  std::vector<std::vector<int64_t>> by_size(n_sizes);
  for (int64_t i = 0; i < n_inst; ++i) {
    const wino_instance& q = inst[i];
    if (q.size < 0 || q.size >= n_sizes || !(q.c > 0.0) || isinf(q.c)) {
      plan_free(p);
      set_error("instance with a bad size index or c <= 0");
      return WINO_EINVAL;
    }
    const SweepSize& z = p->sizes[q.size];
    double probe[kMaxAlpha];
    if (mask_points(q.mask, z.m + z.r - 1, 1.5, z.d, probe) < 0) {
      p->invalid[i] = 1;
      continue;
    }
    by_size[q.size].push_back(i);
  }
  p->size_first.assign(n_sizes, 0);
  p->size_count.assign(n_sizes, 0);
  // a size with too few groups of 32 instances to fill its share of the GPU
  // (per-size mode runs each size as one launch, beside the others)
  // spreads each group's trial chunks over several items; their partial
  // sums are combined in fixed order afterwards, so the errors are the same
  // bits either way
  const int n_chunks = trial_chunks(trials);
  p->inst_first.assign(n_sizes, 0);
  p->inst_count.assign(n_sizes, 0);
  p->size_split.assign(n_sizes, 0);
  bool any_split = false;
  std::vector<std::pair<double, WorkItem>> tmp;
  for (int s = 0; s < n_sizes; ++s) {
    const double flops = sweep_trial_flops(p->sizes[s].dim, p->sizes[s].m, p->sizes[s].r);
    const int64_t items = ((int64_t)by_size[s].size() + 31) / 32;
    int split = 1;
    if (items > 0 && items < sweep_split_warps())
      split = (int)std::min<int64_t>(n_chunks, (sweep_split_warps() + items - 1) / items);
    const int ch_per = (n_chunks + split - 1) / split;
    const int groups = (n_chunks + ch_per - 1) / ch_per;
    p->size_split[s] = groups > 1;
    any_split = any_split || groups > 1;
    p->inst_first[s] = (int64_t)p->order.size();
    p->inst_count[s] = (int64_t)by_size[s].size();
    for (size_t j = 0; j < by_size[s].size(); j += 32) {
      const int first = (int)p->order.size();
      const int count = (int)std::min<size_t>(32, by_size[s].size() - j);
      for (int l = 0; l < count; ++l) p->order.push_back(by_size[s][j + l]);
      for (int g = 0; g < groups; ++g) {
        const int c0 = g * ch_per, c1 = std::min(c0 + ch_per, n_chunks);
        const int t_in = std::min(c1 * kTrialChunk, trials) - c0 * kTrialChunk;
        WorkItem w{s, first, (unsigned short)count, 0, (unsigned short)c0, (unsigned short)c1};
        tmp.push_back({flops * t_in * count / 32.0 + 1e-9 * s, w});
      }
    }
  }
  std::stable_sort(tmp.begin(), tmp.end(),
                   [](const std::pair<double, WorkItem>& x, const std::pair<double, WorkItem>& y) {
                     return x.first > y.first;
                   });
  for (auto& t : tmp) p->items.push_back(t.second);
  // per-size mode reads the items of one size contiguously: group the LPT
  // list by size (sizes come out in decreasing cost)
  std::stable_sort(p->items.begin(), p->items.end(), [&](const WorkItem& x, const WorkItem& y) {
    const double cx = sweep_trial_flops(p->sizes[x.size].dim, p->sizes[x.size].m, p->sizes[x.size].r);
    const double cy = sweep_trial_flops(p->sizes[y.size].dim, p->sizes[y.size].m, p->sizes[y.size].r);
    if (cx != cy) return cx > cy;
    return x.size < y.size;
  });
  for (int i = (int)p->items.size() - 1; i >= 0; --i) {
    p->size_first[p->items[i].size] = i;
    p->size_count[p->items[i].size]++;
  }
  const int64_t n_sorted = (int64_t)p->order.size();
  // per-size mode: sizes to streams, costliest first to the least loaded
  {
    std::vector<double> cost(n_sizes), load(SweepPlan::kPlanLanes, 0.0);
    std::vector<int> by_cost(n_sizes);
    for (int s = 0; s < n_sizes; ++s) {
      by_cost[s] = s;
      cost[s] = sweep_trial_flops(p->sizes[s].dim, p->sizes[s].m, p->sizes[s].r) *
                p->size_count[s];
    }
    std::stable_sort(by_cost.begin(), by_cost.end(),
                     [&](int x, int y) { return cost[x] > cost[y]; });
    p->lane.assign(n_sizes, 0);
    for (int s : by_cost) {
      int l = 0;
      for (int k = 1; k < SweepPlan::kPlanLanes; ++k)
        if (load[k] < load[l]) l = k;
      p->lane[s] = l;
      load[l] += cost[s];
    }
  }

  // device buffers: records | partials | ysum | rec_off | kind | dval | c |
  // mask | err | items | counter | status | deadline
  int rc = WINO_OK;
  if (cudaGetDevice(&p->dev) != cudaSuccess) {
    (void)cudaGetLastError();
    plan_free(p);
    set_error("no CUDA device");
    return WINO_EUNSUPPORTED;
  }
  const int nbp = sweep_prepare_blocks(trials);
  p->rec_off.resize(n_sizes);
  size_t rec_total = 0;
  for (int s = 0; s < n_sizes; ++s) {
    p->rec_off[s] = (int64_t)rec_total;
    rec_total += (size_t)trials * sweep_rec_width(p->sizes[s].dim, p->sizes[s].m, p->sizes[s].r);
  }
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t o = 0;
  const size_t o_rec = o;
  o = al(o + rec_total * 4);
  const size_t o_part = o;
  o = al(o + (size_t)n_sizes * nbp * 8);
  const size_t o_ysum = o;
  o = al(o + (size_t)n_sizes * 8);
  const size_t o_off = o;
  o = al(o + (size_t)n_sizes * 8);
  const size_t o_kind = o;
  o = al(o + (size_t)n_sizes * 4);
  const size_t o_dval = o;
  o = al(o + (size_t)n_sizes * 8);
  const size_t o_c = o;
  o = al(o + (size_t)std::max<int64_t>(n_sorted, 1) * 8);
  const size_t o_mask = o;
  o = al(o + (size_t)std::max<int64_t>(n_sorted, 1));
  const size_t o_err = o;
  o = al(o + (size_t)n_inst * 8);
  const size_t o_items = o;
  o = al(o + std::max<size_t>(p->items.size(), 1) * sizeof(WorkItem));
  const size_t o_isz = o;
  o = al(o + (size_t)std::max<int64_t>(n_sorted, 1));
  const size_t o_chunk = o;
  if (any_split) o = al(o + (size_t)n_chunks * n_sorted * 8);
  const size_t o_ctr = o;
  o = al(o + 64);
  if (cudaMalloc(&p->dbuf, o) != cudaSuccess) {
    (void)cudaGetLastError();
    plan_free(p);
    set_error("could not allocate the sweep plan's device memory");
    return WINO_ENOMEM;
  }
  char* b = (char*)p->dbuf;
  p->rec = (float*)(b + o_rec);
  p->part = (double*)(b + o_part);
  p->ysum = (double*)(b + o_ysum);
  p->deadline = (unsigned long long*)(b + o_ctr + 16);
  p->size_of = (unsigned char*)(b + o_isz);
  std::vector<double> cs(n_sorted), dv(n_sizes);
  std::vector<unsigned char> ms(n_sorted), zs(n_sorted);
  for (int64_t j = 0; j < n_sorted; ++j) {
    cs[j] = inst[p->order[j]].c;
    ms[j] = inst[p->order[j]].mask;
    zs[j] = (unsigned char)inst[p->order[j]].size;
  }
  for (int s = 0; s < n_sizes; ++s) dv[s] = p->sizes[s].d;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpy(b + o_off, p->rec_off.data(), n_sizes * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b + o_kind, p->kind.data(), n_sizes * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b + o_dval, dv.data(), n_sizes * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n_sorted)
    e = cudaMemcpy(b + o_c, cs.data(), n_sorted * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n_sorted)
    e = cudaMemcpy(b + o_mask, ms.data(), n_sorted, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n_sorted)
    e = cudaMemcpy(b + o_isz, zs.data(), n_sorted, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !p->items.empty())
    e = cudaMemcpy(b + o_items, p->items.data(), p->items.size() * sizeof(WorkItem),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&p->err_h, (size_t)n_inst * 8, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&p->status_h, sizeof(int), cudaHostAllocDefault);
  if (e == cudaSuccess)
    e = cudaHostAlloc((void**)&p->deadline_h, sizeof(unsigned long long), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking);
  for (int i = 0; i < SweepPlan::kPlanLanes && e == cudaSuccess; ++i)
    e = cudaStreamCreateWithFlags(&p->lane_st[i], cudaStreamNonBlocking);
  for (int i = 0; i <= SweepPlan::kPlanLanes && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&p->lane_ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "sweep plan setup");
    plan_free(p);
    return rc;
  }
  *p->deadline_h = 0ull;
  PlanDev& P = p->P;
  P.items = (const WorkItem*)(b + o_items);
  P.n_items = (int)p->items.size();
  P.counter = (int*)(b + o_ctr);
  P.status = (int*)(b + o_ctr + 4);
  P.deadline = p->deadline;
  P.inst_c = (const double*)(b + o_c);
  P.inst_mask = (const unsigned char*)(b + o_mask);
  P.rec = p->rec;
  P.rec_off = (const int64_t*)(b + o_off);
  P.kind = (const int*)(b + o_kind);
  P.dval = (const double*)(b + o_dval);
  P.ysum = p->ysum;
  P.err = (double*)(b + o_err);
  P.part = (double*)(b + o_chunk);
  P.n_sorted = n_sorted;
  P.trials = trials;
  P.n_chunks = n_chunks;
  P.split = any_split ? 2 : 1;

  if (mode == WINO_SWEEP_AUTO) {
    rc = plan_autotune(p);
  } else {
    p->mode = mode;
  }
  if (rc == WINO_OK) rc = plan_capture(p);
  if (rc != WINO_OK) {
    plan_free(p);
    return rc;
  }
  *plan_out = p;
  return WINO_OK;
}

int wino_sweep_plan_set_deadline(void* plan, double max_ms) {
  SweepPlan* p = (SweepPlan*)plan;
  if (!p || max_ms < 0.0) {
    set_error("invalid arguments to wino_sweep_plan_set_deadline");
    return WINO_EINVAL;
  }
  p->max_ms = max_ms;
  return WINO_OK;
}

int wino_sweep_plan_run(void* plan, double* err_out, void* cuda_stream) {
  SweepPlan* p = (SweepPlan*)plan;
  if (!p || !err_out) {
    set_error("invalid arguments to wino_sweep_plan_run");
    return WINO_EINVAL;
  }
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : p->st;
  // the deadline is absolute device time: read the device clock now
  unsigned long long limit = 0ull;
  if (p->max_ms > 0.0) {
    unsigned long long now = 0ull;
    int rc = device_time_ns(&now);
    if (rc != WINO_OK) return rc;
    limit = now + (unsigned long long)(p->max_ms * 1e6);
  }
  *p->deadline_h = limit;
  WINO_CUDA_TRY(cudaGraphLaunch(p->exec, st));
  WINO_CUDA_TRY(cudaStreamSynchronize(st));
  for (int64_t i = 0; i < p->n_inst; ++i) err_out[i] = NAN;
  for (size_t j = 0; j < p->order.size(); ++j) err_out[p->order[j]] = p->err_h[j];
  if (*p->status_h == WINO_ETIMEOUT) {
    set_error("sweep stopped at its deadline before all instances were evaluated");
    return WINO_ETIMEOUT;
  }
  return WINO_OK;
}

int wino_sweep_plan_set_c(void* plan, const double* c, int64_t n) {
  SweepPlan* p = (SweepPlan*)plan;
  if (!p || !c || n != p->n_inst) {
    set_error("wino_sweep_plan_set_c needs one c per instance of the plan");
    return WINO_EINVAL;
  }
  std::vector<double> cs(p->order.size());
  for (size_t j = 0; j < p->order.size(); ++j) {
    const double v = c[p->order[j]];
    if (!(v > 0.0) || isinf(v)) {
      set_error("c values must be finite and > 0");
      return WINO_EINVAL;
    }
    cs[j] = v;
  }
  if (!cs.empty())
    WINO_CUDA_TRY(cudaMemcpyAsync((void*)p->P.inst_c, cs.data(), cs.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, p->st));
  WINO_CUDA_TRY(cudaStreamSynchronize(p->st));
  return WINO_OK;
}

int wino_sweep_plan_info(void* plan, int* mode, int* grid, int* n_items) {
  SweepPlan* p = (SweepPlan*)plan;
  if (!p) {
    set_error("plan is NULL");
    return WINO_EINVAL;
  }
  if (mode) *mode = p->mode;
  if (grid) *grid = p->grid;
  if (n_items) *n_items = (int)p->items.size();
  return WINO_OK;
}

void wino_sweep_plan_destroy(void* plan) { plan_free((SweepPlan*)plan); }

}  // extern "C"
