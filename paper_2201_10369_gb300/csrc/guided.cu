// guided.cu -- host drivers of the searches built on the sweep: the
// surrogate-guided search of a c grid, the random search it is measured
// against, and the two-parameter (c, d) sweep.  Every evaluation,
// prediction and ranking runs in the library's kernels (planned sweeps,
// the MLP's predict kernel, the top-k kernel); this file decides which grid
// points the next launch evaluates and reduces the results.
//
// Guided search (the paper has no surrogate; its Sec. 6.1 finding that the
// error over c is a rough but smooth-at-large-scale curve motivates it).
// Per valid (size, mask) row of a c grid:
//   1. the network ranks every grid c (predict kernel) and its `top` best
//      predictions (top-k kernel) plus `probe` counter-drawn random grid
//      points are evaluated exactly in one planned launch;
//   2. the 2 refine + 1 grid points centred on the network's best verified
//      proposal are evaluated in a second planned launch (the curve is
//      noisy between neighbouring c, so the best of the proposals is
//      refined before it is judged);
//   3. if the network's region -- its proposals and their refinement -- is
//      worse than guard x the best random probe, the network failed on that
//      row and the row is swept exhaustively (the plain sweep is both the
//      fallback and the judge);
//   4. the row's result is the least error evaluated.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <vector>

#include "../../include/wino.h"
#include "common.cuh"

using namespace wino;

namespace {

uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// The rule of wino_error_sweep for a mask being evaluated at a size.
bool mask_valid(unsigned mask, const wino_size& s) {
  if (__builtin_popcount(mask) != s.m + s.r - 3) return false;
  if (fabs(s.d) == 1.0 && (mask & 0x90u)) return false;
  return true;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

struct Guided {
  void* mlp = nullptr;  // borrowed
  std::vector<wino_size> sizes;
  std::vector<unsigned char> masks;
  std::vector<double> cg;
  int trials = 0;
  unsigned long long seed = 0;
  wino_guided_params prm{};
  std::vector<int> rs, rq;            // per row: size index, index into masks
  std::vector<unsigned char> rm;      // per row: mask
  float* X = nullptr;                 // device [rows * n_c][16]
  float* pred = nullptr;              // device [rows * n_c]
  int* idx = nullptr;                 // device [rows][top]
  void* verify = nullptr;             // plan: rows x (top + probe)
  void* local = nullptr;              // plan: rows x (2 refine + 1)
  uint64_t runs = 0;
};

void guided_free(Guided* g) {
  if (!g) return;
  if (g->verify) wino_sweep_plan_destroy(g->verify);
  if (g->local) wino_sweep_plan_destroy(g->local);
  cudaFree(g->X);
  cudaFree(g->pred);
  cudaFree(g->idx);
  (void)cudaGetLastError();
  delete g;
}

// A plan with `per` instances per row (c filled later with set_c).
int make_row_plan(const Guided* g, int per, void** plan) {
  std::vector<wino_instance> inst;
  inst.reserve((size_t)g->rs.size() * per);
  const double c0 = g->cg[g->cg.size() / 3];
  for (size_t r = 0; r < g->rs.size(); ++r)
    for (int j = 0; j < per; ++j) inst.push_back(wino_instance{g->rs[r], g->rm[r], c0});
  return wino_sweep_plan_create(g->sizes.data(), (int)g->sizes.size(), inst.data(),
                                (int64_t)inst.size(), g->trials, g->seed, WINO_SWEEP_PERSISTENT,
                                plan);
}

// Runs `plan` at grid points sel[r * per + j]; err (host) in the same order,
// non-finite errors as +inf.
int run_row_plan(void* plan, const std::vector<double>& cg, const std::vector<int>& sel,
                 std::vector<double>& err, cudaStream_t st) {
  std::vector<double> c(sel.size());
  for (size_t i = 0; i < sel.size(); ++i) c[i] = cg[sel[i]];
  int rc = wino_sweep_plan_set_c(plan, c.data(), (int64_t)c.size());
  if (rc != WINO_OK) return rc;
  err.assign(sel.size(), 0.0);
  rc = wino_sweep_plan_run(plan, err.data(), st);
  if (rc != WINO_OK) return rc;
  for (double& e : err)
    if (!isfinite(e)) e = INFINITY;
  return WINO_OK;
}

}  // namespace

extern "C" {

int wino_guided_create(void* mlp, const wino_size* sizes, int n_sizes, const unsigned char* masks,
                       int n_masks, const double* c_grid, int n_c, int trials,
                       unsigned long long seed, const wino_guided_params* prm, void** gs) {
  if (!gs || !mlp || !sizes || n_sizes < 1 || n_sizes > 64 || !masks || n_masks < 1 ||
      !c_grid || n_c < 2 || n_c > 8192 || trials < 1 || !prm || prm->top < 1 ||
      prm->top > n_c || prm->probe < 1 || prm->refine < 0 || 2 * prm->refine + 1 > n_c ||
      !(prm->guard >= 1.0)) {
    set_error("invalid arguments to wino_guided_create (2 <= n_c <= 8192, 1 <= top <= n_c, "
              "probe >= 1, 0 <= 2 refine + 1 <= n_c, guard >= 1)");
    return WINO_EINVAL;
  }
  *gs = nullptr;
  if (!wino_device_ok()) return WINO_EUNSUPPORTED;
  Guided* g = new Guided();
  g->mlp = mlp;
  g->sizes.assign(sizes, sizes + n_sizes);
  g->masks.assign(masks, masks + n_masks);
  g->cg.assign(c_grid, c_grid + n_c);
  g->trials = trials;
  g->seed = seed;
  g->prm = *prm;
  for (int s = 0; s < n_sizes; ++s)
    for (int q = 0; q < n_masks; ++q)
      if (mask_valid(masks[q], sizes[s])) {
        g->rs.push_back(s);
        g->rq.push_back(q);
        g->rm.push_back(masks[q]);
      }
  const int nr = (int)g->rs.size();
  if (nr == 0) {
    guided_free(g);
    set_error("no (size, mask) pair is valid");
    return WINO_EINVAL;
  }
  const size_t n = (size_t)nr * n_c;
  cudaError_t e = cudaMalloc(&g->X, n * 16 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&g->pred, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&g->idx, (size_t)nr * prm->top * sizeof(int));
  if (e != cudaSuccess) {
    guided_free(g);
    return cuda_fail(e, "wino_guided_create: cudaMalloc");
  }
  int rc = wino_mlp_grid_features(sizes, n_sizes, g->rs.data(), g->rm.data(), nr, c_grid, n_c,
                                  g->X, nullptr);
  if (rc == WINO_OK) rc = make_row_plan(g, prm->top + prm->probe, &g->verify);
  if (rc == WINO_OK) rc = make_row_plan(g, 2 * prm->refine + 1, &g->local);
  if (rc != WINO_OK) {
    guided_free(g);
    return rc;
  }
  *gs = g;
  return WINO_OK;
}

int wino_guided_run(void* gs, double* best_err, double* best_c, wino_guided_stats* stats,
                    void* cuda_stream) {
  Guided* g = (Guided*)gs;
  if (!g || !best_err || !best_c) {
    set_error("invalid arguments to wino_guided_run");
    return WINO_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nr = (int)g->rs.size(), nc = (int)g->cg.size();
  const int top = g->prm.top, probe = g->prm.probe, nl = 2 * g->prm.refine + 1;
  const int per = top + probe;
  const uint64_t run = g->runs++;
  auto t0 = std::chrono::steady_clock::now();
  // 1. rank every grid c of every row; the top proposals
  int rc = wino_mlp_predict(g->mlp, g->X, (int64_t)nr * nc, g->pred, st);
  if (rc == WINO_OK) rc = wino_topk_rows(g->pred, nr, nc, top, g->idx, st);
  if (rc != WINO_OK) return rc;
  std::vector<int> idx((size_t)nr * top);
  WINO_CUDA_TRY(cudaMemcpyAsync(idx.data(), g->idx, idx.size() * sizeof(int),
                                cudaMemcpyDeviceToHost, st));
  WINO_CUDA_TRY(cudaStreamSynchronize(st));
  const double t_rank = ms_since(t0);
  // ... verified together with `probe` random grid points per row
  std::vector<int> sel((size_t)nr * per);
  for (int r = 0; r < nr; ++r) {
    for (int j = 0; j < top; ++j) sel[(size_t)r * per + j] = idx[(size_t)r * top + j];
    for (int j = 0; j < probe; ++j) {
      const uint64_t z = splitmix64_mix(g->seed + 0x9E3779B97F4A7C15ull *
                                                      (1 + ((run * (uint64_t)nr + r) * probe + j)));
      sel[(size_t)r * per + top + j] = (int)(z % (uint64_t)nc);
    }
  }
  std::vector<double> ev;
  auto t1 = std::chrono::steady_clock::now();
  rc = run_row_plan(g->verify, g->cg, sel, ev, st);
  if (rc != WINO_OK) return rc;
  const double t_verify = ms_since(t1);
  // 2. refine around the network's best verified proposal
  auto t2 = std::chrono::steady_clock::now();
  std::vector<int> lsel((size_t)nr * nl);
  std::vector<double> net_best(nr), probe_best(nr), best_e(nr);
  std::vector<int> best_k(nr);
  for (int r = 0; r < nr; ++r) {
    const double* e = ev.data() + (size_t)r * per;
    int bt = 0;
    for (int j = 1; j < top; ++j)
      if (e[j] < e[bt]) bt = j;
    double vp = INFINITY;
    for (int j = top; j < per; ++j) vp = std::min(vp, e[j]);
    net_best[r] = e[bt];
    probe_best[r] = vp;
    int bj = 0;
    for (int j = 1; j < per; ++j)
      if (e[j] < e[bj]) bj = j;
    best_e[r] = e[bj];
    best_k[r] = sel[(size_t)r * per + bj];
    const int centre = sel[(size_t)r * per + bt];
    for (int j = 0; j < nl; ++j)
      lsel[(size_t)r * nl + j] = std::min(nc - 1, std::max(0, centre - g->prm.refine + j));
  }
  std::vector<double> le;
  rc = run_row_plan(g->local, g->cg, lsel, le, st);
  if (rc != WINO_OK) return rc;
  int64_t evaluated = (int64_t)sel.size() + (int64_t)lsel.size();
  std::vector<int> fallback;
  for (int r = 0; r < nr; ++r) {
    const double* e = le.data() + (size_t)r * nl;
    for (int j = 0; j < nl; ++j) {
      net_best[r] = std::min(net_best[r], e[j]);
      if (e[j] < best_e[r]) {
        best_e[r] = e[j];
        best_k[r] = lsel[(size_t)r * nl + j];
      }
    }
    // 3. the network's region lost to the random probe: exhaustive row
    if (net_best[r] > g->prm.guard * probe_best[r]) fallback.push_back(r);
  }
  const double t_refine = ms_since(t2);
  auto t3 = std::chrono::steady_clock::now();
  std::map<int, std::vector<int>> by_size;
  for (int r : fallback) by_size[g->rs[r]].push_back(r);
  for (auto& kv : by_size) {
    std::vector<unsigned char> mk;
    for (int r : kv.second) mk.push_back(g->rm[r]);
    std::vector<double> e((size_t)mk.size() * nc);
    rc = wino_error_sweep(g->cg.data(), nc, &g->sizes[kv.first], 1, mk.data(), (int)mk.size(),
                          g->trials, g->seed, e.data(), st);
    if (rc != WINO_OK) return rc;
    for (size_t j = 0; j < kv.second.size(); ++j) {
      const int r = kv.second[j];
      double be = INFINITY;
      int bk = 0;
      for (int k = 0; k < nc; ++k) {
        const double v = e[j * nc + k];
        if (isfinite(v) && v < be) {
          be = v;
          bk = k;
        }
      }
      best_e[r] = be;
      best_k[r] = bk;
      evaluated += nc;
    }
  }
  const double t_fallback = ms_since(t3);
  const int ns = (int)g->sizes.size(), nm = (int)g->masks.size();
  for (int i = 0; i < ns * nm; ++i) best_err[i] = best_c[i] = NAN;
  for (int r = 0; r < nr; ++r) {
    const int o = g->rs[r] * nm + g->rq[r];
    best_err[o] = best_e[r];
    best_c[o] = isfinite(best_e[r]) ? g->cg[best_k[r]] : NAN;
  }
  if (stats) {
    stats->evaluated = evaluated;
    stats->rows = nr;
    stats->fallback_rows = (int)fallback.size();
    stats->phase_ms[0] = t_rank;
    stats->phase_ms[1] = t_verify;
    stats->phase_ms[2] = t_refine;
    stats->phase_ms[3] = t_fallback;
  }
  return WINO_OK;
}

void wino_guided_destroy(void* gs) { guided_free((Guided*)gs); }

int wino_random_search(const wino_size* sizes, int n_sizes, const unsigned char* masks,
                       int n_masks, const double* c_grid, int n_c, int trials, int budget,
                       unsigned long long seed, double* best_err, void* cuda_stream) {
  if (!sizes || n_sizes < 1 || n_sizes > 64 || !masks || n_masks < 1 || !c_grid || n_c < 1 ||
      trials < 1 || budget < 1 || !best_err) {
    set_error("invalid arguments to wino_random_search");
    return WINO_EINVAL;
  }
  std::vector<wino_instance> inst;
  std::vector<int> out;  // instance block -> output index
  for (int s = 0; s < n_sizes; ++s)
    for (int q = 0; q < n_masks; ++q) {
      best_err[s * n_masks + q] = NAN;
      if (!mask_valid(masks[q], sizes[s])) continue;
      const int r = (int)out.size();
      out.push_back(s * n_masks + q);
      for (int j = 0; j < budget; ++j) {
        const uint64_t z = splitmix64_mix(seed + 0x9E3779B97F4A7C15ull *
                                                     (1 + (uint64_t)r * budget + j));
        inst.push_back(wino_instance{s, masks[q], c_grid[z % (uint64_t)n_c]});
      }
    }
  if (out.empty()) return WINO_OK;
  void* plan = nullptr;
  int rc = wino_sweep_plan_create(sizes, n_sizes, inst.data(), (int64_t)inst.size(), trials, seed,
                                  WINO_SWEEP_PERSISTENT, &plan);
  if (rc != WINO_OK) return rc;
  std::vector<double> e(inst.size());
  rc = wino_sweep_plan_run(plan, e.data(), cuda_stream);
  wino_sweep_plan_destroy(plan);
  if (rc != WINO_OK) return rc;
  for (size_t r = 0; r < out.size(); ++r) {
    double b = INFINITY;
    for (int j = 0; j < budget; ++j) {
      const double v = e[r * budget + j];
      if (isfinite(v)) b = std::min(b, v);
    }
    best_err[out[r]] = b;
  }
  return WINO_OK;
}

int wino_cd_sweep(int dim, int m, int r, const double* c_grid, int n_c, const double* d_grid,
                  int n_d, const unsigned char* masks, int n_masks, int trials,
                  unsigned long long seed, double* err_out, void* cuda_stream) {
  if (!c_grid || n_c < 1 || !d_grid || n_d < 1 || !masks || n_masks < 1 || trials < 1 ||
      !err_out || (dim != 1 && dim != 2)) {
    set_error("invalid arguments to wino_cd_sweep");
    return WINO_EINVAL;
  }
  for (int i = 0; i < n_d; ++i)
    if (!(d_grid[i] > 0.0) || isinf(d_grid[i])) {
      set_error("d values must be finite and > 0");
      return WINO_EINVAL;
    }
  const size_t row = (size_t)n_c;
  for (size_t i = 0; i < (size_t)n_d * n_masks * n_c; ++i) err_out[i] = NAN;
  // the wide 2D sizes run one warp per instance only: no planned form
  const bool wide = dim == 2 && r == 3 && (m == 7 || m == 8);
  for (int d0 = 0; d0 < n_d; d0 += 64) {
    const int nd = std::min(64, n_d - d0);
    std::vector<wino_size> sz(nd);
    for (int i = 0; i < nd; ++i) sz[i] = wino_size{dim, m, r, d_grid[d0 + i]};
    if (wide) {
      int rc = wino_error_sweep(c_grid, n_c, sz.data(), nd, masks, n_masks, trials, seed,
                                err_out + (size_t)d0 * n_masks * row, cuda_stream);
      if (rc != WINO_OK) return rc;
      continue;
    }
    std::vector<wino_instance> inst;
    std::vector<std::pair<int, int>> rows;  // (d index in chunk, mask index)
    for (int i = 0; i < nd; ++i)
      for (int q = 0; q < n_masks; ++q) {
        if (!mask_valid(masks[q], sz[i])) continue;
        rows.push_back({i, q});
        for (int k = 0; k < n_c; ++k) inst.push_back(wino_instance{i, masks[q], c_grid[k]});
      }
    if (rows.empty()) continue;
    void* plan = nullptr;
    int rc = wino_sweep_plan_create(sz.data(), nd, inst.data(), (int64_t)inst.size(), trials,
                                    seed, WINO_SWEEP_PERSISTENT, &plan);
    if (rc != WINO_OK) return rc;
    std::vector<double> e(inst.size());
    rc = wino_sweep_plan_run(plan, e.data(), cuda_stream);
    wino_sweep_plan_destroy(plan);
    if (rc != WINO_OK) return rc;
    for (size_t j = 0; j < rows.size(); ++j)
      std::copy(e.begin() + j * row, e.begin() + (j + 1) * row,
                err_out + ((size_t)(d0 + rows[j].first) * n_masks + rows[j].second) * row);
  }
  return WINO_OK;
}

}  // extern "C"
