// patch.cuh -- input patches of consecutive tiles held by consecutive lanes,
// loaded row by row as vectors.
//
// With padding 1 and an even input width W, tile t (tile row ti, tile
// column tj) of F(m x m, 3 x 3) reads input columns m tj - 1 .. m tj + m of
// rows m ti - 1 .. m ti + m.  Its m interior columns start at an even
// column, so a row's interior loads as m / 2 eight-byte vectors (m = 4 with
// W a multiple of 4: one sixteen-byte vector); the two halo columns are the
// last interior column of tile t - 1 and the first of tile t + 1, which lie
// in the same tile row whenever they are inside the image (column -1 and
// the columns from W on are the zero padding).  When the neighbouring lanes
// hold those tiles of the same channel, the halos come from them by
// shuffle; a lane at either end of such a run loads its own.  All rows'
// loads are issued before the first shuffle, which waits on them, so that
// they are in flight together.
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace wino {

// Whether load_patch_rowvec applies: a 2D layer with padding 1, W even and
// x 8-byte aligned.
__device__ __forceinline__ bool patch_rowvec_ok(const float* x, const LayerGeom& g) {
  return g.dim == 2 && g.pad == 1 && (g.W & 1) == 0 && (((uintptr_t)x) & 7) == 0;
}

// d = the (MM + 2) x (MM + 2) input patch of tile t, channel c, rows and
// columns outside the image zero; all zero when !live (t >= T or c >= C).
// own_l / own_r: this lane loads its left / right halo itself (the lane
// before / after it does not hold tile t - 1 / t + 1 of channel c).  Every
// lane of the warp calls it, with patch_rowvec_ok true.
template <int MM>
__device__ __forceinline__ void load_patch_rowvec(const float* __restrict__ x, const LayerGeom& g,
                                                  int64_t t, int c, bool live, bool own_l,
                                                  bool own_r, float (&d)[MM + 2][MM + 2]) {
  constexpr int A = MM + 2;
  static_assert(MM % 2 == 0, "whole eight-byte vectors per row");
  int n = 0, ti = 0, tj = 0;
  if (live) {
    const int tpi = g.th * g.tw;
    n = (int)(t / tpi);
    const int rem = (int)(t - (int64_t)n * tpi);
    ti = rem / g.tw;
    tj = rem - ti * g.tw;
  }
  const int h0 = ti * MM - 1, c0 = tj * MM;
  const float* xc = x + ((int64_t)n * g.C + (live ? c : 0)) * g.H * g.W;
  const bool in_l = c0 > 0, in_r = c0 + MM < g.W;  // the halo columns inside the row
  const bool vec4 = MM % 4 == 0 && (g.W & 3) == 0 && (((uintptr_t)x) & 15) == 0;
  float v[A][MM], el[A], er[A];
#pragma unroll
  for (int i = 0; i < A; ++i) {
    const int hh = h0 + i;
#pragma unroll
    for (int j = 0; j < MM; ++j) v[i][j] = 0.0f;
    el[i] = 0.0f;
    er[i] = 0.0f;
    if (live && (unsigned)hh < (unsigned)g.H) {
      const float* row = xc + (int64_t)hh * g.W + c0;
      if (vec4) {
#pragma unroll
        for (int k = 0; k < MM / 4; ++k) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(row) + k);
          v[i][4 * k] = q.x;
          v[i][4 * k + 1] = q.y;
          v[i][4 * k + 2] = q.z;
          v[i][4 * k + 3] = q.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < MM / 2; ++k)
          if (c0 + 2 * k < g.W) {  // W even: a pair is wholly inside or outside
            const float2 p = __ldg(reinterpret_cast<const float2*>(row) + k);
            v[i][2 * k] = p.x;
            v[i][2 * k + 1] = p.y;
          }
      }
      if (own_l && in_l) el[i] = __ldg(row - 1);
      if (own_r && in_r) er[i] = __ldg(row + MM);
    }
  }
#pragma unroll
  for (int i = 0; i < A; ++i) {
    const bool rv = live && (unsigned)(h0 + i) < (unsigned)g.H;
    float l = __shfl_up_sync(0xffffffffu, v[i][MM - 1], 1);
    float r = __shfl_down_sync(0xffffffffu, v[i][0], 1);
    if (own_l) l = el[i];
    if (own_r) r = er[i];
    d[i][0] = (rv && in_l) ? l : 0.0f;
#pragma unroll
    for (int j = 0; j < MM; ++j) d[i][1 + j] = v[i][j];
    d[i][A - 1] = (rv && in_r) ? r : 0.0f;
  }
}

}  // namespace wino
