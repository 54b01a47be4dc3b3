// patterns.cu -- the subset-pattern query over a sweep's errors (Sec. 6.2,
// Tables 2-6): which subset of the group {-1/c, -c, c, 1/c}, joined to fixed
// base points, gives the least error, at which c, and how consistently.
// Host code only; it reads the host array wino_error_sweep returns.
//
// A base is a set of d-group slots of the sweep's masks (bits 4-7 over
// [-1/d, -d, d, 1/d]; for example d = 3 with bit 6 is the base point 3,
// d = 2 with bit 7 is 1/2, d = 1 with bits 5 and 6 is the pair -1, 1); a
// candidate is a mask whose d-group bits equal the base's and that is valid
// for the size.  The order of the output and the tie rules are part of the
// contract (include/wino.h), so a caller can compare results bit for bit.
#include <math.h>

#include <algorithm>
#include <vector>

#include "../../include/wino.h"
#include "common.cuh"

using namespace wino;

namespace {

bool valid_for(unsigned mask, int alpha, double d) {
  if (__builtin_popcount(mask) != alpha - 2) return false;
  if (fabs(d) == 1.0 && (mask & 0x90u)) return false;
  return true;
}

}  // namespace

extern "C" int wino_subset_pattern(const double* err, const unsigned char* masks, int n_masks,
                                   const double* c_grid, int n_c, wino_size size,
                                   unsigned char base_mask, double c_lo, double c_hi,
                                   wino_pattern_cand* cand_out, int max_cand, int* n_cand) {
  if (!err || !masks || !c_grid || !n_cand || n_masks < 1 || n_c < 1 || max_cand < 0 ||
      (max_cand > 0 && !cand_out)) {
    set_error("wino_subset_pattern: null array or empty size");
    return WINO_EINVAL;
  }
  if (base_mask & 0x0Fu) {
    set_error("wino_subset_pattern: the base mask holds d-group bits (4-7) only");
    return WINO_EINVAL;
  }
  const int alpha = size.m + size.r - 1;
  if (size.m < 1 || size.r < 1 || alpha < 3 || alpha > WINO_MAX_ALPHA) {
    set_error("wino_subset_pattern: bad size");
    return WINO_EINVAL;
  }
  std::vector<int> window;
  for (int k = 0; k < n_c; ++k)
    if (c_grid[k] >= c_lo && c_grid[k] <= c_hi) window.push_back(k);
  struct Row {
    int q, best_k, wins;
    unsigned mask;
    double best_err;
  };
  std::vector<Row> rows;
  for (int q = 0; q < n_masks; ++q) {
    const unsigned mk = masks[q];
    if ((mk & 0xF0u) != base_mask || !valid_for(mk, alpha, size.d)) continue;
    Row r{q, -1, 0, mk, NAN};
    const double* e = err + (size_t)q * n_c;
    for (int k : window)
      if (isfinite(e[k]) && (r.best_k < 0 || e[k] < r.best_err)) {
        r.best_k = k;
        r.best_err = e[k];
      }
    rows.push_back(r);
  }
  int common = 0;
  for (int k : window) {
    bool all = !rows.empty();
    for (const Row& r : rows) all = all && isfinite(err[(size_t)r.q * n_c + k]);
    if (!all) continue;
    ++common;
    size_t w = 0;
    for (size_t i = 1; i < rows.size(); ++i) {
      const double vi = err[(size_t)rows[i].q * n_c + k], vw = err[(size_t)rows[w].q * n_c + k];
      if (vi < vw || (vi == vw && rows[i].mask < rows[w].mask)) w = i;
    }
    ++rows[w].wins;
  }
  std::sort(rows.begin(), rows.end(), [](const Row& a, const Row& b) {
    const bool fa = a.best_k >= 0, fb = b.best_k >= 0;
    if (fa != fb) return fa;
    if (fa && a.best_err != b.best_err) return a.best_err < b.best_err;
    return a.mask < b.mask;
  });
  *n_cand = (int)rows.size();
  for (int i = 0; i < (int)rows.size() && i < max_cand; ++i) {
    wino_pattern_cand& o = cand_out[i];
    o.mask = (unsigned char)rows[i].mask;
    o.best_k = rows[i].best_k;
    o.best_c = rows[i].best_k >= 0 ? c_grid[rows[i].best_k] : NAN;
    o.best_err = rows[i].best_err;
    o.win_frac = common ? (double)rows[i].wins / common : 0.0;
  }
  return WINO_OK;
}
