// construct.cuh -- modified Toom-Cook transform matrices in FP64.
//
// One definition used on the host (wino_make_matrices, the layer entry
// points) and on the device (the sweep builds ~5e5 matrix sets, one per
// (size, mask, c) instance, inside its kernel).  Both sides round every
// operation the same way (explicit _rn intrinsics on the device, no
// contraction on the host), so the FP32 matrices the sweep uses are
// identical to the ones the host would build.
//
// Construction (Sec. 4.1, Eqs. (10)-(11) with N_i folded into G; Sec. 4.2,
// Eq. (19) for the point at infinity), finite points a_0 < ... < a_{n-1}
// (n = alpha - 1), infinity last:
//   N_i      = prod_{j != i} (a_i - a_j)                (ascending j)
//   G[i][k]  = a_i^k / N_i,  G[n][k] = [k == r-1]       (powers by repeated
//   AT[j][i] = a_i^j,        AT[j][n] = [j == m-1]       multiplication)
//   BT[i][l] = coeff of x^l in prod_{j != i}(x - a_j)   (ascending j)
//   BT[n][l] = coeff of x^l in M'(x) = prod_j (x - a_j)
#pragma once

#include <math.h>

#ifndef WINO_HD
#ifdef __CUDACC__
#define WINO_HD __host__ __device__ __forceinline__
#else
#define WINO_HD inline
#endif
#endif

namespace wino {

constexpr int kMaxAlpha = 12;

WINO_HD double dmul(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}
WINO_HD double dsub(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dsub_rn(a, b);
#else
  return a - b;
#endif
}
WINO_HD double ddiv(double a, double b) {
#ifdef __CUDA_ARCH__
  return __ddiv_rn(a, b);
#else
  return a / b;
#endif
}

// Sorts `n` finite values ascending in place (insertion sort; n <= 11).
WINO_HD void sort_points(double* a, int n) {
  for (int i = 1; i < n; ++i) {
    double v = a[i];
    int j = i - 1;
    while (j >= 0 && a[j] > v) {
      a[j + 1] = a[j];
      --j;
    }
    a[j + 1] = v;
  }
}

// p <- p * (x - a), p of degree `deg` (ascending coefficients):
// q_l = p_{l-1} - a p_l, a rounded product then a rounded difference.
WINO_HD void poly_times_linear(double* p, int deg, double a) {
  p[deg + 1] = p[deg];
  for (int l = deg; l >= 1; --l) p[l] = dsub(p[l - 1], dmul(a, p[l]));
  p[0] = dsub(0.0, dmul(a, p[0]));
}

// Builds AT[m][alpha], G[alpha][r], BT[alpha][alpha] (row-major FP64) from
// the sorted finite points a[0..alpha-2].  Returns false when two points are
// equal (singular Vandermonde system).
template <typename Out>
WINO_HD bool build_matrices(const double* a, int m, int r, Out* AT, Out* G, Out* BT) {
  const int alpha = m + r - 1;
  const int n = alpha - 1;
  for (int i = 0; i + 1 < n; ++i)
    if (a[i] == a[i + 1]) return false;
  for (int i = 0; i < n; ++i) {
    double Ni = 1.0;
    for (int j = 0; j < n; ++j)
      if (j != i) Ni = dmul(Ni, dsub(a[i], a[j]));
    double pw = 1.0;
    for (int k = 0; k < r; ++k) {
      G[i * r + k] = (Out)ddiv(pw, Ni);
      pw = dmul(pw, a[i]);
    }
    pw = 1.0;
    for (int j = 0; j < m; ++j) {
      AT[j * alpha + i] = (Out)pw;
      pw = dmul(pw, a[i]);
    }
  }
  for (int k = 0; k < r; ++k) G[n * r + k] = (Out)(k == r - 1 ? 1.0 : 0.0);
  for (int j = 0; j < m; ++j) AT[j * alpha + n] = (Out)(j == m - 1 ? 1.0 : 0.0);

  double p[kMaxAlpha + 1];
  for (int i = 0; i <= n; ++i) {  // i == n: the row of M'(x)
    for (int l = 0; l <= alpha; ++l) p[l] = 0.0;
    p[0] = 1.0;
    int deg = 0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      poly_times_linear(p, deg, a[j]);
      ++deg;
    }
    for (int l = 0; l < alpha; ++l) BT[i * alpha + l] = (Out)(l <= deg ? p[l] : 0.0);
  }
  return true;
}

// Point set of a sweep instance: {0, inf} plus the slots selected by `mask`
// from [-1/c, -c, c, 1/c, -1/d, -d, d, 1/d] (Eqs. (20)-(25)).  Writes the
// sorted finite points and returns their count, or -1 when the mask is
// invalid for alpha (wrong popcount, or a duplicated d-slot when |d| = 1).
WINO_HD int mask_points(unsigned mask, int alpha, double c, double d, double* a) {
  int cnt = 0;
  for (int b = 0; b < 8; ++b) cnt += (mask >> b) & 1u;
  if (mask > 255u || cnt != alpha - 2) return -1;
  if (fabs(d) == 1.0 && (mask & 0x90u)) return -1;
  const double ic = ddiv(1.0, c), id = ddiv(1.0, d);
  const double slot[8] = {-ic, -c, c, ic, -id, -d, d, id};
  int n = 0;
  a[n++] = 0.0;
  for (int b = 0; b < 8; ++b)
    if ((mask >> b) & 1u) a[n++] = slot[b];
  sort_points(a, n);
  return n;
}

}  // namespace wino
