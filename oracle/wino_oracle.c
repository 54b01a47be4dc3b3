/*
 * wino_oracle.c -- plain CPU oracle for Winograd point selection.
 *
 * TEST INFRASTRUCTURE ONLY: the slow, obviously correct statement of what
 * the GPU library computes.  Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline leg may load it; the library never does.  It
 * shares no code with paper_2201_10369_gb300/.
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared wino_oracle.c -lm -lpthread
 * (-ffp-contract=off so that every a*b+c written below rounds twice unless
 * it is spelled fmaf).
 *
 * FP32 operation order (the paper does not state one; this is the reading
 * the GPU path also follows): every matrix-vector product is computed output
 * by output as acc = 0; for each inner index in ascending order
 * acc = fmaf(matrix entry, vector entry, acc).  The Hadamard product is a
 * single rounded multiply; in a layer the per-frequency products are summed
 * over input channels c in ascending order with fmaf.
 */
#include "wino_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Point sets and the modified Toom-Cook matrices (Sec. 4.1, 4.2).           */
/* ------------------------------------------------------------------------ */

int orc_canonical_points(const double* points, int alpha, double* out) {
  int n_inf = 0, nf = 0;
  double fin[ORC_MAX_ALPHA];
  if (alpha < 2 || alpha > ORC_MAX_ALPHA) return -1;
  for (int i = 0; i < alpha; ++i) {
    double p = points[i];
    if (isnan(p)) return -1;
    if (isinf(p)) {
      if (p < 0) return -1;
      ++n_inf;
    } else {
      fin[nf++] = p;
    }
  }
  if (n_inf != 1) return -1;
  /* insertion sort, ascending */
  for (int i = 1; i < nf; ++i) {
    double v = fin[i];
    int j = i - 1;
    while (j >= 0 && fin[j] > v) {
      fin[j + 1] = fin[j];
      --j;
    }
    fin[j + 1] = v;
  }
  for (int i = 0; i < nf; ++i) out[i] = fin[i];
  out[nf] = INFINITY;
  return alpha;
}

/* Multiplies the ascending coefficient vector p (degree deg) by (x - a):
 * q_l = p_{l-1} - a * p_l, one rounded multiply then one rounded subtract. */
static void poly_mul_linear(double* p, int deg, double a) {
  p[deg + 1] = p[deg];
  for (int l = deg; l >= 1; --l) p[l] = p[l - 1] - a * p[l];
  p[0] = 0.0 - a * p[0];
}

int orc_make_matrices(const double* points, int m, int r,
                      double* AT, double* G, double* BT) {
  if (m < 1 || r < 1) return -1;
  const int alpha = m + r - 1;
  if (alpha < 2 || alpha > ORC_MAX_ALPHA) return -1;
  double a[ORC_MAX_ALPHA];
  if (orc_canonical_points(points, alpha, a) < 0) return -1;
  const int nf = alpha - 1; /* finite points a_0 .. a_{alpha-2} */
  for (int i = 0; i + 1 < nf; ++i)
    if (a[i] == a[i + 1]) return -2;

  /* N_i = prod_{j != i} (a_i - a_j), factors in ascending j (Sec. 4.1). */
  double N[ORC_MAX_ALPHA];
  for (int i = 0; i < nf; ++i) {
    double prod = 1.0;
    for (int j = 0; j < nf; ++j)
      if (j != i) prod = prod * (a[i] - a[j]);
    N[i] = prod;
  }

  /* G: Vandermonde rows a_i^k scaled by 1/N_i (Eq. (10), N_i folded into G),
   * powers by repeated multiplication, then one division; last row e_{r-1}
   * for the point at infinity (Eq. (19)). */
  for (int i = 0; i < nf; ++i) {
    double pw = 1.0;
    for (int k = 0; k < r; ++k) {
      G[i * r + k] = pw / N[i];
      pw = pw * a[i];
    }
  }
  for (int k = 0; k < r; ++k) G[nf * r + k] = (k == r - 1) ? 1.0 : 0.0;

  /* AT: AT[j][i] = a_i^j (Eq. (10)); last column e_{m-1} (Eq. (19)). */
  for (int i = 0; i < nf; ++i) {
    double pw = 1.0;
    for (int j = 0; j < m; ++j) {
      AT[j * alpha + i] = pw;
      pw = pw * a[i];
    }
  }
  for (int j = 0; j < m; ++j) AT[j * alpha + nf] = (j == m - 1) ? 1.0 : 0.0;

  /* BT: row i < nf = coefficients of prod_{j != i}(x - a_j) (Eq. (11),
   * M_i = M/m_i); last row = coefficients of M'(x) = prod_j (x - a_j)
   * (Eq. (19)).  Factors multiplied in ascending j. */
  double poly[ORC_MAX_ALPHA + 1];
  for (int i = 0; i < nf; ++i) {
    int deg = 0;
    for (int l = 0; l <= alpha; ++l) poly[l] = 0.0;
    poly[0] = 1.0;
    for (int j = 0; j < nf; ++j) {
      if (j == i) continue;
      poly_mul_linear(poly, deg, a[j]);
      ++deg;
    }
    for (int l = 0; l < alpha; ++l) BT[i * alpha + l] = (l <= deg) ? poly[l] : 0.0;
  }
  {
    int deg = 0;
    for (int l = 0; l <= alpha; ++l) poly[l] = 0.0;
    poly[0] = 1.0;
    for (int j = 0; j < nf; ++j) {
      poly_mul_linear(poly, deg, a[j]);
      ++deg;
    }
    for (int l = 0; l < alpha; ++l) BT[nf * alpha + l] = poly[l];
  }
  return alpha;
}

/* ------------------------------------------------------------------------ */
/* Direct correlation (Eq. (1)).                                             */
/* ------------------------------------------------------------------------ */

void orc_direct_f64(const float* x, const float* w, double* y, int dim,
                    int N, int C, int K, int H, int W, int pad, int r) {
  const int Hin = (dim == 1) ? 1 : H;
  const int rh = (dim == 1) ? 1 : r;
  const int Ho = (dim == 1) ? 1 : H + 2 * pad - r + 1;
  const int Wo = W + 2 * pad - r + 1;
  const int padh = (dim == 1) ? 0 : pad;
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < K; ++k)
      for (int p = 0; p < Ho; ++p)
        for (int q = 0; q < Wo; ++q) {
          double acc = 0.0;
          for (int c = 0; c < C; ++c)
            for (int u = 0; u < rh; ++u)
              for (int v = 0; v < r; ++v) {
                int hh = p + u - padh, ww = q + v - pad;
                if (hh < 0 || hh >= Hin || ww < 0 || ww >= W) continue;
                double xv = (double)x[(((size_t)n * C + c) * Hin + hh) * W + ww];
                double wv = (double)w[(((size_t)k * C + c) * rh + u) * r + v];
                acc += xv * wv;
              }
          y[(((size_t)n * K + k) * Ho + p) * Wo + q] = acc;
        }
}

/* ------------------------------------------------------------------------ */
/* FP32 Winograd, one tile (Eqs. (8), (9)).                                  */
/* ------------------------------------------------------------------------ */

void orc_tile1d_f32(const float* AT, const float* G, const float* BT,
                    int m, int r, const float* g, const float* d, float* y) {
  const int alpha = m + r - 1;
  float u[ORC_MAX_ALPHA], v[ORC_MAX_ALPHA], p[ORC_MAX_ALPHA];
  for (int i = 0; i < alpha; ++i) { /* u = G g */
    float acc = 0.0f;
    for (int k = 0; k < r; ++k) acc = fmaf(G[i * r + k], g[k], acc);
    u[i] = acc;
  }
  for (int i = 0; i < alpha; ++i) { /* v = BT d */
    float acc = 0.0f;
    for (int l = 0; l < alpha; ++l) acc = fmaf(BT[i * alpha + l], d[l], acc);
    v[i] = acc;
  }
  for (int i = 0; i < alpha; ++i) p[i] = u[i] * v[i]; /* Hadamard */
  for (int j = 0; j < m; ++j) { /* y = AT p */
    float acc = 0.0f;
    for (int i = 0; i < alpha; ++i) acc = fmaf(AT[j * alpha + i], p[i], acc);
    y[j] = acc;
  }
}

/* 2D nesting of the 1D algorithm, Eq. (9): U = G g G^T, V = B^T d B,
 * Y = A^T (U .* V) A, each as two matrix products (left factor first). */
void orc_tile2d_f32(const float* AT, const float* G, const float* BT,
                    int m, int r, const float* g, const float* d, float* y) {
  const int A = m + r - 1;
  float Wk[ORC_MAX_ALPHA * ORC_MAX_ALPHA], U[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  float T[ORC_MAX_ALPHA * ORC_MAX_ALPHA], V[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  float Z[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (int i = 0; i < A; ++i) /* Wk = G g  (A x r) */
    for (int k = 0; k < r; ++k) {
      float acc = 0.0f;
      for (int l = 0; l < r; ++l) acc = fmaf(G[i * r + l], g[l * r + k], acc);
      Wk[i * r + k] = acc;
    }
  for (int i = 0; i < A; ++i) /* U = Wk G^T  (A x A) */
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
      for (int k = 0; k < r; ++k) acc = fmaf(Wk[i * r + k], G[j * r + k], acc);
      U[i * A + j] = acc;
    }
  for (int i = 0; i < A; ++i) /* T = B^T d */
    for (int l = 0; l < A; ++l) {
      float acc = 0.0f;
      for (int k = 0; k < A; ++k) acc = fmaf(BT[i * A + k], d[k * A + l], acc);
      T[i * A + l] = acc;
    }
  for (int i = 0; i < A; ++i) /* V = T B,  B[l][j] = BT[j][l] */
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
      for (int l = 0; l < A; ++l) acc = fmaf(T[i * A + l], BT[j * A + l], acc);
      V[i * A + j] = acc;
    }
  for (int i = 0; i < A * A; ++i) V[i] = U[i] * V[i]; /* Hadamard */
  for (int a = 0; a < m; ++a) /* Z = A^T P */
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
      for (int i = 0; i < A; ++i) acc = fmaf(AT[a * A + i], V[i * A + j], acc);
      Z[a * A + j] = acc;
    }
  for (int a = 0; a < m; ++a) /* Y = Z A,  A[j][b] = AT[b][j] */
    for (int b = 0; b < m; ++b) {
      float acc = 0.0f;
      for (int j = 0; j < A; ++j) acc = fmaf(Z[a * A + j], AT[b * A + j], acc);
      y[a * m + b] = acc;
    }
}

void orc_tile_direct_f32(int dim, int m, int r, const float* g,
                         const float* d, float* y) {
  const int A = m + r - 1;
  if (dim == 1) {
    for (int j = 0; j < m; ++j) {
      float acc = 0.0f;
      for (int k = 0; k < r; ++k) acc = fmaf(g[k], d[j + k], acc);
      y[j] = acc;
    }
    return;
  }
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      float acc = 0.0f;
      for (int u = 0; u < r; ++u)
        for (int v = 0; v < r; ++v) acc = fmaf(g[u * r + v], d[(a + u) * A + b + v], acc);
      y[a * m + b] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Reduced-precision operand rounding (precision form of the contraction).  */
/* ------------------------------------------------------------------------ */

static uint32_t f2u(float v) { uint32_t u; memcpy(&u, &v, 4); return u; }
static float u2f(uint32_t u) { float v; memcpy(&v, &u, 4); return v; }

/* BF16 = the top 16 bits of an FP32 value, round to nearest even. */
float orc_round_bf16(float v) {
  if (isnan(v)) return v;
  uint32_t u = f2u(v);
  uint32_t lsb = (u >> 16) & 1u;
  u = u + 0x7FFFu + lsb;
  return u2f(u & 0xFFFF0000u);
}

/* FP16 (1 sign, 5 exponent, 10 fraction bits) round to nearest even,
 * written out in terms of the representable grid: the spacing of FP16 at
 * |v| is 2^(e-10) for normal e >= -14, 2^-24 for subnormals; values at or
 * above 65520 overflow to infinity. */
float orc_round_fp16(float v) {
  if (isnan(v) || isinf(v)) return v;
  double a = fabs((double)v);
  if (a >= 65520.0) return v < 0 ? -INFINITY : INFINITY;
  int e;
  double spacing;
  if (a < 0x1p-14) {
    spacing = 0x1p-24;
  } else {
    frexp(a, &e); /* a = f * 2^e, f in [0.5, 1) -> unbiased exponent e-1 */
    spacing = ldexp(1.0, (e - 1) - 10);
  }
  double q = a / spacing;       /* exact: spacing is a power of two */
  double fl = floor(q);
  double rem = q - fl;
  double n = fl;
  if (rem > 0.5 || (rem == 0.5 && fmod(fl, 2.0) != 0.0)) n = fl + 1.0;
  double res = n * spacing;
  return (float)(v < 0 ? -res : res);
}

static float round_mode(float v, int lowp) {
  if (lowp == 2) return orc_round_fp16(v);
  return orc_round_bf16(v);
}

/* power of two 2^-E with max * 2^-E in [1, 2); 1 when max is 0. */
static float pow2_normaliser(double mx) {
  if (!(mx > 0.0) || isinf(mx)) return 1.0f;
  int e;
  frexp(mx, &e);
  return (float)ldexp(1.0, -(e - 1));
}

/* One product of the contraction over channels, in the precision form
 * `lowp` (0 FP32, 1 BF16, 2 FP16, 3 split BF16 x3, 4 split BF16 x6): u, v
 * the FP32 transform outputs, sU, sV the frequency's power-of-two scales;
 * accumulates into *acc (and, x6, the five small products into *acc_lo). */
static void mac_lowp(int lowp, float u, float v, float sU, float sV, float* acc,
                     float* acc_lo) {
  if (lowp == 0) {
    *acc = fmaf(u, v, *acc);
  } else if (lowp == 1 || lowp == 2) {
    float uq = round_mode(u * sU, lowp), vq = round_mode(v * sV, lowp);
    *acc = fmaf(uq, vq, *acc);
  } else if (lowp == 3) {
    float us = u * sU, vs = v * sV;
    float uh = orc_round_bf16(us), vh = orc_round_bf16(vs);
    float ul = orc_round_bf16(us - uh), vl = orc_round_bf16(vs - vh);
    *acc = fmaf(uh, vh, *acc);
    *acc = fmaf(uh, vl, *acc);
    *acc = fmaf(ul, vh, *acc);
  } else {
    /* three-part split: hi, mid = RN(a - hi), lo = RN((a - hi) - mid);
       the differences are exact in FP32 */
    float us = u * sU, vs = v * sV;
    float uh = orc_round_bf16(us), vh = orc_round_bf16(vs);
    float ur = us - uh, vr = vs - vh;
    float um = orc_round_bf16(ur), vm = orc_round_bf16(vr);
    float ul = orc_round_bf16(ur - um), vl = orc_round_bf16(vr - vm);
    /* hh in one accumulator, the five smaller products (below 2^-7 of hh)
       in a second one, added at the end */
    *acc = fmaf(uh, vh, *acc);
    *acc_lo = fmaf(uh, vm, *acc_lo);
    *acc_lo = fmaf(um, vh, *acc_lo);
    *acc_lo = fmaf(uh, vl, *acc_lo);
    *acc_lo = fmaf(ul, vh, *acc_lo);
    *acc_lo = fmaf(um, vm, *acc_lo);
  }
}

/* The contraction's value M[f] from its accumulators: x6 adds the small
 * products' accumulator, and the scales come off (exact: powers of two). */
static float finish_lowp(int lowp, float acc, float acc_lo, float sU, float sV) {
  if (lowp == 4) acc = acc + acc_lo;
  if (lowp != 0) acc = acc / (sU * sV);
  return acc;
}

/* ------------------------------------------------------------------------ */
/* FP32 Winograd layer.                                                      */
/* ------------------------------------------------------------------------ */

int orc_wino_layer(const float* x, const float* w, float* y, int dim,
                   int N, int C, int K, int H, int W, int pad,
                   const double* points, int m, int r, int lowp) {
  const int A = m + r - 1;
  double ATd[ORC_MAX_ALPHA * ORC_MAX_ALPHA], Gd[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  double BTd[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  int st = orc_make_matrices(points, m, r, ATd, Gd, BTd);
  if (st < 0) return st;
  float AT[ORC_MAX_ALPHA * ORC_MAX_ALPHA], G[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  float BT[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (int i = 0; i < m * A; ++i) AT[i] = (float)ATd[i];
  for (int i = 0; i < A * r; ++i) G[i] = (float)Gd[i];
  for (int i = 0; i < A * A; ++i) BT[i] = (float)BTd[i];

  const int Hin = (dim == 1) ? 1 : H;
  const int Ho = (dim == 1) ? 1 : H + 2 * pad - r + 1;
  const int Wo = W + 2 * pad - r + 1;
  const int padh = (dim == 1) ? 0 : pad;
  const int th = (dim == 1) ? 1 : (Ho + m - 1) / m;
  const int tw = (Wo + m - 1) / m;
  const int F = (dim == 1) ? A : A * A;       /* frequencies per tile */
  const int ro = (dim == 1) ? 1 : m;          /* output tile rows     */
  const int rw = (dim == 1) ? r : r * r;      /* filter taps          */
  const size_t T = (size_t)N * th * tw;

  float* V = (float*)malloc(sizeof(float) * (size_t)F * C * K);
  float* U = (float*)malloc(sizeof(float) * (size_t)F * T * C);
  if (!V || !U) { free(V); free(U); return -1; }

  /* filter transform: V[f][c][k] = (G g G^T)[f]  (1D: G g) */
  float tmpd[ORC_MAX_ALPHA * ORC_MAX_ALPHA], outt[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (int k = 0; k < K; ++k)
    for (int c = 0; c < C; ++c) {
      const float* g = w + ((size_t)k * C + c) * rw;
      if (dim == 1) {
        for (int i = 0; i < A; ++i) {
          float acc = 0.0f;
          for (int q = 0; q < r; ++q) acc = fmaf(G[i * r + q], g[q], acc);
          outt[i] = acc;
        }
      } else {
        float Wk[ORC_MAX_ALPHA * 5];
        for (int i = 0; i < A; ++i)
          for (int q = 0; q < r; ++q) {
            float acc = 0.0f;
            for (int l = 0; l < r; ++l) acc = fmaf(G[i * r + l], g[l * r + q], acc);
            Wk[i * r + q] = acc;
          }
        for (int i = 0; i < A; ++i)
          for (int j = 0; j < A; ++j) {
            float acc = 0.0f;
            for (int q = 0; q < r; ++q) acc = fmaf(Wk[i * r + q], G[j * r + q], acc);
            outt[i * A + j] = acc;
          }
      }
      for (int f = 0; f < F; ++f) V[((size_t)f * C + c) * K + k] = outt[f];
    }

  /* input transform: U[f][t][c] = (B^T d B)[f] of the zero-padded patch */
  for (int n = 0; n < N; ++n)
    for (int ti = 0; ti < th; ++ti)
      for (int tj = 0; tj < tw; ++tj) {
        size_t t = ((size_t)n * th + ti) * tw + tj;
        for (int c = 0; c < C; ++c) {
          const int pr = (dim == 1) ? 1 : A;
          for (int i = 0; i < pr; ++i)
            for (int j = 0; j < A; ++j) {
              int hh = ti * m - padh + i, ww = tj * m - pad + j;
              float v = 0.0f;
              if (hh >= 0 && hh < Hin && ww >= 0 && ww < W)
                v = x[(((size_t)n * C + c) * Hin + hh) * W + ww];
              tmpd[i * A + j] = v;
            }
          if (dim == 1) {
            for (int i = 0; i < A; ++i) {
              float acc = 0.0f;
              for (int l = 0; l < A; ++l) acc = fmaf(BT[i * A + l], tmpd[l], acc);
              outt[i] = acc;
            }
          } else {
            float Tm[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
            for (int i = 0; i < A; ++i)
              for (int l = 0; l < A; ++l) {
                float acc = 0.0f;
                for (int q = 0; q < A; ++q) acc = fmaf(BT[i * A + q], tmpd[q * A + l], acc);
                Tm[i * A + l] = acc;
              }
            for (int i = 0; i < A; ++i)
              for (int j = 0; j < A; ++j) {
                float acc = 0.0f;
                for (int l = 0; l < A; ++l) acc = fmaf(Tm[i * A + l], BT[j * A + l], acc);
                outt[i * A + j] = acc;
              }
          }
          for (int f = 0; f < F; ++f) U[((size_t)f * T + t) * C + c] = outt[f];
        }
      }

  /* precision form: per-frequency power-of-two scales, operand rounding */
  float sU[ORC_MAX_ALPHA * ORC_MAX_ALPHA], sV[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (int f = 0; f < F; ++f) { sU[f] = 1.0f; sV[f] = 1.0f; }
  if (lowp != 0) {
    double rown[ORC_MAX_ALPHA];
    for (int i = 0; i < A; ++i) {
      double s = 0.0;
      for (int l = 0; l < A; ++l) s += fabs((double)BT[i * A + l]);
      rown[i] = s;
    }
    for (int f = 0; f < F; ++f) {
      double gain = (dim == 1) ? rown[f] : rown[f / A] * rown[f % A];
      sU[f] = pow2_normaliser(gain);
      double mx = 0.0;
      for (size_t q = 0; q < (size_t)C * K; ++q) {
        double a = fabs((double)V[(size_t)f * C * K + q]);
        if (a > mx) mx = a;
      }
      sV[f] = pow2_normaliser(mx);
    }
  }

  /* contraction over c and output transform, per (tile, k) */
  float Mf[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (size_t t = 0; t < T; ++t) {
    const int n = (int)(t / ((size_t)th * tw));
    const int ti = (int)((t / tw) % th), tj = (int)(t % tw);
    for (int k = 0; k < K; ++k) {
      for (int f = 0; f < F; ++f) {
        float acc = 0.0f, acc_lo = 0.0f;  /* acc_lo: split x6's small products */
        for (int c = 0; c < C; ++c)
          mac_lowp(lowp, U[((size_t)f * T + t) * C + c], V[((size_t)f * C + c) * K + k], sU[f],
                   sV[f], &acc, &acc_lo);
        acc = finish_lowp(lowp, acc, acc_lo, sU[f], sV[f]);
        Mf[f] = acc;
      }
      if (dim == 1) {
        for (int j = 0; j < m; ++j) {
          float acc = 0.0f;
          for (int i = 0; i < A; ++i) acc = fmaf(AT[j * A + i], Mf[i], acc);
          int q = tj * m + j;
          if (q < Wo) y[((size_t)n * K + k) * Wo + q] = acc;
        }
      } else {
        float Z[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
        for (int a = 0; a < m; ++a)
          for (int j = 0; j < A; ++j) {
            float acc = 0.0f;
            for (int i = 0; i < A; ++i) acc = fmaf(AT[a * A + i], Mf[i * A + j], acc);
            Z[a * A + j] = acc;
          }
        for (int a = 0; a < ro; ++a)
          for (int b = 0; b < m; ++b) {
            float acc = 0.0f;
            for (int j = 0; j < A; ++j) acc = fmaf(Z[a * A + j], AT[b * A + j], acc);
            int p = ti * m + a, q = tj * m + b;
            if (p < Ho && q < Wo) y[(((size_t)n * K + k) * Ho + p) * Wo + q] = acc;
          }
      }
    }
  }
  free(U);
  free(V);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Counter-based trial inputs: SplitMix64.                                   */
/* ------------------------------------------------------------------------ */

uint64_t orc_splitmix64(uint64_t seed, uint64_t n) {
  /* state after n steps is seed + n * golden gamma; output = finaliser */
  uint64_t z = seed + n * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Counter: 1 + idx + 2^12 (trial + 2^20 (r + 2^4 (m + 2^4 dim))).
 * Value: top 24 bits k of the output, x = k 2^-23 - 1 (exact in FP32). */
float orc_trial_value(uint64_t seed, int dim, int m, int r, int trial, int idx) {
  uint64_t ctr = (uint64_t)dim;
  ctr = ctr * 16u + (uint64_t)m;
  ctr = ctr * 16u + (uint64_t)r;
  ctr = ctr * (1ull << 20) + (uint64_t)trial;
  ctr = ctr * (1ull << 12) + (uint64_t)idx;
  uint64_t z = orc_splitmix64(seed, ctr + 1u);
  double k = (double)(z >> 40);
  return (float)(k * 0x1p-23 - 1.0);
}

/* ------------------------------------------------------------------------ */
/* Subset masks over the proposed point families (Eqs. (20)-(25)).           */
/* ------------------------------------------------------------------------ */

int orc_mask_points(int dim, int m, int r, double d, unsigned mask,
                    double c, double* points) {
  (void)dim;
  const int alpha = m + r - 1;
  int cnt = 0;
  for (int b = 0; b < 8; ++b) cnt += (mask >> b) & 1u;
  if (mask > 255u || cnt != alpha - 2) return -1;
  if (fabs(d) == 1.0 && (mask & 0x90u)) return -1; /* -1/d, 1/d duplicate -d, d */
  const double slot[8] = {-1.0 / c, -c, c, 1.0 / c, -1.0 / d, -d, d, 1.0 / d};
  int n = 0;
  points[n++] = 0.0;
  for (int b = 0; b < 8; ++b)
    if ((mask >> b) & 1u) points[n++] = slot[b];
  points[n++] = INFINITY;
  return n;
}

/* ------------------------------------------------------------------------ */
/* The error sweep.                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
  int alpha, nin_g, nin_d, nout;
  float* g;     /* [trials][nin_g] */
  float* d;     /* [trials][nin_d] */
  double* y;    /* [trials][nout]  FP64 reference */
  double ysum;  /* sum_t ||y_t||_1 */
} size_data;

static int build_size_data(const orc_size* s, int trials, uint64_t seed, size_data* sd) {
  const int A = s->m + s->r - 1;
  sd->alpha = A;
  sd->nin_g = (s->dim == 1) ? s->r : s->r * s->r;
  sd->nin_d = (s->dim == 1) ? A : A * A;
  sd->nout = (s->dim == 1) ? s->m : s->m * s->m;
  sd->g = (float*)malloc(sizeof(float) * (size_t)trials * sd->nin_g);
  sd->d = (float*)malloc(sizeof(float) * (size_t)trials * sd->nin_d);
  sd->y = (double*)malloc(sizeof(double) * (size_t)trials * sd->nout);
  if (!sd->g || !sd->d || !sd->y) return -1;
  sd->ysum = 0.0;
  for (int t = 0; t < trials; ++t) {
    float* g = sd->g + (size_t)t * sd->nin_g;
    float* d = sd->d + (size_t)t * sd->nin_d;
    double* y = sd->y + (size_t)t * sd->nout;
    for (int i = 0; i < sd->nin_g; ++i) g[i] = orc_trial_value(seed, s->dim, s->m, s->r, t, i);
    for (int i = 0; i < sd->nin_d; ++i) d[i] = orc_trial_value(seed, s->dim, s->m, s->r, t, 256 + i);
    /* FP64 direct correlation of one tile */
    if (s->dim == 1)
      orc_direct_f64(d, g, y, 1, 1, 1, 1, 1, A, 0, s->r);
    else
      orc_direct_f64(d, g, y, 2, 1, 1, 1, A, A, 0, s->r);
    for (int j = 0; j < sd->nout; ++j) sd->ysum += fabs(y[j]);
  }
  return 0;
}

static double eval_instance(const orc_size* s, const size_data* sd, const double* pts,
                            int trials) {
  const int A = sd->alpha, m = s->m, r = s->r;
  double ATd[ORC_MAX_ALPHA * ORC_MAX_ALPHA], Gd[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  double BTd[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  int st = orc_make_matrices(pts, m, r, ATd, Gd, BTd);
  if (st == -2) return INFINITY;
  if (st < 0) return NAN;
  float AT[ORC_MAX_ALPHA * ORC_MAX_ALPHA], G[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  float BT[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (int i = 0; i < m * A; ++i) AT[i] = (float)ATd[i];
  for (int i = 0; i < A * r; ++i) G[i] = (float)Gd[i];
  for (int i = 0; i < A * A; ++i) BT[i] = (float)BTd[i];
  double num = 0.0;
  float yh[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (int t = 0; t < trials; ++t) {
    const float* g = sd->g + (size_t)t * sd->nin_g;
    const float* d = sd->d + (size_t)t * sd->nin_d;
    const double* y = sd->y + (size_t)t * sd->nout;
    if (s->dim == 1)
      orc_tile1d_f32(AT, G, BT, m, r, g, d, yh);
    else
      orc_tile2d_f32(AT, G, BT, m, r, g, d, yh);
    for (int j = 0; j < sd->nout; ++j) num += fabs((double)yh[j] - y[j]);
  }
  return num / sd->ysum;
}

typedef struct {
  const double* c_grid;
  int n_c, n_sizes, n_masks, trials, c_stride, tid, nth;
  const orc_size* sizes;
  const unsigned char* masks;
  const size_data* sd;
  double* err;
} sweep_job;

static void* sweep_worker(void* arg) {
  sweep_job* jb = (sweep_job*)arg;
  size_t idx = 0;
  for (int s = 0; s < jb->n_sizes; ++s)
    for (int q = 0; q < jb->n_masks; ++q)
      for (int k = 0; k < jb->n_c; k += jb->c_stride, ++idx) {
        if ((int)(idx % (size_t)jb->nth) != jb->tid) continue;
        const orc_size* sz = &jb->sizes[s];
        double pts[ORC_MAX_ALPHA + 2];
        double* out = &jb->err[((size_t)s * jb->n_masks + q) * jb->n_c + k];
        int a = orc_mask_points(sz->dim, sz->m, sz->r, sz->d, jb->masks[q], jb->c_grid[k], pts);
        if (a < 0) { *out = NAN; continue; }
        *out = eval_instance(sz, &jb->sd[s], pts, jb->trials);
      }
  return NULL;
}

int orc_error_sweep(const double* c_grid, int n_c, const orc_size* sizes,
                    int n_sizes, const unsigned char* masks, int n_masks,
                    int trials, uint64_t seed, double* err_out,
                    int c_stride, int n_threads) {
  if (c_stride < 1) c_stride = 1;
  if (n_threads < 1) n_threads = 1;
  size_data* sd = (size_data*)calloc((size_t)n_sizes, sizeof(size_data));
  if (!sd) return -1;
  int rc = 0;
  for (int s = 0; s < n_sizes && rc == 0; ++s) rc = build_size_data(&sizes[s], trials, seed, &sd[s]);
  if (rc == 0) {
    sweep_job* jobs = (sweep_job*)calloc((size_t)n_threads, sizeof(sweep_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int i = 0; i < n_threads; ++i) {
      sweep_job j = {c_grid, n_c, n_sizes, n_masks, trials, c_stride, i, n_threads,
                     sizes, masks, sd, err_out};
      jobs[i] = j;
    }
    for (int i = 1; i < n_threads; ++i) pthread_create(&th[i], NULL, sweep_worker, &jobs[i]);
    sweep_worker(&jobs[0]);
    for (int i = 1; i < n_threads; ++i) pthread_join(th[i], NULL);
    free(jobs);
    free(th);
  }
  for (int s = 0; s < n_sizes; ++s) { free(sd[s].g); free(sd[s].d); free(sd[s].y); }
  free(sd);
  return rc;
}

int orc_pointset_error(int dim, int m, int r, const double* points, int n_sets, int trials,
                       uint64_t seed, double* err_out) {
  const int A = m + r - 1;
  if (dim < 1 || dim > 2 || A < 2 || A > ORC_MAX_ALPHA || n_sets < 0 || trials < 1) return -1;
  orc_size s = {dim, m, r, 1.0};
  size_data sd;
  memset(&sd, 0, sizeof(sd));
  int rc = build_size_data(&s, trials, seed, &sd);
  for (int q = 0; q < n_sets && rc == 0; ++q)
    err_out[q] = eval_instance(&s, &sd, points + (size_t)q * A, trials);
  free(sd.g); free(sd.d); free(sd.y);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Kronecker-product form of the 2D tile (Sec. 7): with row-major vec,       */
/*   vec(G g G^T) = (G (x) G) vec(g),  vec(B^T d B) = (B^T (x) B^T) vec(d),   */
/*   vec(A^T M A) = (A^T (x) A^T) vec(M).                                     */
/* Reading: the Kronecker entries are products of the FP64 matrix entries,  */
/* rounded once to FP32 ("multiply the transform matrices together before   */
/* the vector multiplication"); each product row is summed in FP32 with     */
/* fmaf, column index ascending, or (pairwise) as rounded products summed   */
/* pairwise: sum(x[0..n)) = sum(x[0..h)) + sum(x[h..n)), h = ceil(n / 2).   */
/* ------------------------------------------------------------------------ */

static float pairwise_sum(const float* x, int n) {
  if (n == 1) return x[0];
  const int h = (n + 1) / 2;
  return pairwise_sum(x, h) + pairwise_sum(x + h, n - h);
}

/* y[rows] = K[rows][cols] x[cols] in FP32, one of the two summation orders */
static void kron_matvec(const float* K, int rows, int cols, const float* x, float* y,
                        int pairwise) {
  float prod[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (int i = 0; i < rows; ++i) {
    const float* k = K + (size_t)i * cols;
    if (pairwise) {
      for (int c = 0; c < cols; ++c) prod[c] = k[c] * x[c];
      y[i] = pairwise_sum(prod, cols);
    } else {
      float acc = 0.0f;
      for (int c = 0; c < cols; ++c) acc = fmaf(k[c], x[c], acc);
      y[i] = acc;
    }
  }
}

/* The three Kronecker matrices of a point set, FP32. */
typedef struct {
  int m, r, A;
  float KG[ORC_MAX_ALPHA * ORC_MAX_ALPHA * 25];                       /* [A^2][r^2] */
  float KB[ORC_MAX_ALPHA * ORC_MAX_ALPHA * ORC_MAX_ALPHA * ORC_MAX_ALPHA]; /* [A^2][A^2] */
  float KA[ORC_MAX_ALPHA * ORC_MAX_ALPHA * ORC_MAX_ALPHA * ORC_MAX_ALPHA]; /* [m^2][A^2] */
} kron_mats;

static int build_kron(const double* points, int m, int r, kron_mats* K) {
  const int A = m + r - 1;
  if (r > 5 || A > ORC_MAX_ALPHA) return -1;
  double ATd[ORC_MAX_ALPHA * ORC_MAX_ALPHA], Gd[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  double BTd[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  int st = orc_make_matrices(points, m, r, ATd, Gd, BTd);
  if (st < 0) return st;
  K->m = m; K->r = r; K->A = A;
  for (int i = 0; i < A; ++i)
    for (int j = 0; j < A; ++j)
      for (int k = 0; k < r; ++k)
        for (int l = 0; l < r; ++l)
          K->KG[(i * A + j) * r * r + k * r + l] = (float)(Gd[i * r + k] * Gd[j * r + l]);
  for (int i = 0; i < A; ++i)
    for (int j = 0; j < A; ++j)
      for (int k = 0; k < A; ++k)
        for (int l = 0; l < A; ++l)
          K->KB[(i * A + j) * A * A + k * A + l] = (float)(BTd[i * A + k] * BTd[j * A + l]);
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b)
      for (int i = 0; i < A; ++i)
        for (int j = 0; j < A; ++j)
          K->KA[(a * m + b) * A * A + i * A + j] = (float)(ATd[a * A + i] * ATd[b * A + j]);
  return 0;
}

static void kron_tile(const kron_mats* K, const float* g, const float* d, float* y, int pairwise) {
  const int A2 = K->A * K->A;
  float u[ORC_MAX_ALPHA * ORC_MAX_ALPHA], v[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  float p[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  kron_matvec(K->KG, A2, K->r * K->r, g, u, pairwise);
  kron_matvec(K->KB, A2, A2, d, v, pairwise);
  for (int i = 0; i < A2; ++i) p[i] = u[i] * v[i];
  kron_matvec(K->KA, K->m * K->m, A2, p, y, pairwise);
}

int orc_tile2d_kron(const double* points, int m, int r, const float* g, const float* d,
                    float* y, int pairwise) {
  kron_mats* K = (kron_mats*)malloc(sizeof(kron_mats));
  if (!K) return -1;
  int st = build_kron(points, m, r, K);
  if (st == 0) kron_tile(K, g, d, y, pairwise);
  free(K);
  return st;
}

int orc_pointset_error_kron(int m, int r, const double* points, int n_sets, int trials,
                            uint64_t seed, int pairwise, double* err_out) {
  const int A = m + r - 1;
  if (A < 2 || A > ORC_MAX_ALPHA || r > 5 || n_sets < 0 || trials < 1) return -1;
  orc_size s = {2, m, r, 1.0};
  size_data sd;
  memset(&sd, 0, sizeof(sd));
  int rc = build_size_data(&s, trials, seed, &sd);
  kron_mats* K = (kron_mats*)malloc(sizeof(kron_mats));
  if (!K) rc = -1;
  for (int q = 0; q < n_sets && rc == 0; ++q) {
    int st = build_kron(points + (size_t)q * A, m, r, K);
    if (st == -2) { err_out[q] = INFINITY; continue; }
    if (st < 0) { err_out[q] = NAN; continue; }
    double num = 0.0;
    float yh[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
    for (int t = 0; t < trials; ++t) {
      kron_tile(K, sd.g + (size_t)t * sd.nin_g, sd.d + (size_t)t * sd.nin_d, yh, pairwise);
      for (int j = 0; j < sd.nout; ++j) num += fabs((double)yh[j] - sd.y[(size_t)t * sd.nout + j]);
    }
    err_out[q] = num / sd.ysum;
  }
  free(K);
  free(sd.g); free(sd.d); free(sd.y);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Summation-order variants of the single tile (Sec. 5): the Huffman        */
/* evaluation order of Barabasz et al. that the paper's error tables use,   */
/* alone in FP32, and with the transforms in FP64 and the Hadamard product  */
/* in FP32 ("mixed precision").  The paper names both and defines neither;  */
/* the reading taken here:                                                  */
/*  - every output of a transform is one dot product sum_k c_k x_k, c a row */
/*    of G, B^T or A^T (a 2D transform is two such passes, in the order of  */
/*    orc_tile2d_f32);                                                      */
/*  - terms with c_k == 0 are left out; the others are the rounded products */
/*    c_k * x_k (no fused multiply-add);                                    */
/*  - the terms are added along a Huffman tree with leaf weights |c_k| (the */
/*    FP32 entry): the two live nodes of least weight are replaced by their */
/*    sum, whose weight is the FP64 sum of theirs, until one node is left;  */
/*    ties go to the node created first (leaves in column order, then the   */
/*    merged nodes in order of creation);                                   */
/*  - ORC_ORDER_HUFFMAN: products and sums in FP32.                         */
/*    ORC_ORDER_HUFFMAN_MIXED: products and sums in FP64 on the FP64 matrix */
/*    entries and the widened inputs, with the same trees; U and V rounded  */
/*    to FP32, P = U .* V in FP32, the output transform in FP64 on P, and Y */
/*    rounded to FP32 once at the end.                                      */
/* ------------------------------------------------------------------------ */

/* Merge list of the Huffman tree over the leaves k < n with w[k] > 0: merge
 * s joins node ids first[s] and second[s] (leaf k has id k, merge s creates
 * id n + s).  Returns the number of merges (-1 when no weight is positive)
 * and the root's id in *root. */
static int huffman_merges(const double* w, int n, int* first, int* second, int* root) {
  double wt[2 * ORC_MAX_ALPHA];
  int live[2 * ORC_MAX_ALPHA];
  int n_live = 0, nodes = n, s = 0, last = -1;
  for (int k = 0; k < n; ++k) {
    wt[k] = w[k];
    live[k] = w[k] > 0.0;
    if (live[k]) { ++n_live; last = k; }
  }
  if (n_live == 0) return -1;
  while (n_live > 1) {
    int f = -1, g = -1;
    for (int id = 0; id < nodes; ++id) /* least weight, earliest id on ties */
      if (live[id] && (f < 0 || wt[id] < wt[f])) f = id;
    for (int id = 0; id < nodes; ++id) /* the same among the rest */
      if (live[id] && id != f && (g < 0 || wt[id] < wt[g])) g = id;
    first[s] = f;
    second[s] = g;
    wt[nodes] = wt[f] + wt[g];
    live[nodes] = 1;
    live[f] = live[g] = 0;
    ++nodes;
    ++s;
    --n_live;
  }
  *root = s == 0 ? last : nodes - 1;
  return s;
}

int orc_huffman_merges(const double* w, int n, int* first, int* second) {
  int root;
  if (n < 1 || n > ORC_MAX_ALPHA) return -1;
  return huffman_merges(w, n, first, second, &root);
}

/* sum_k c[k] x[k] in FP32 along the Huffman tree of |c| */
static float huff_dot_f32(const float* c, const float* x, int n) {
  double w[ORC_MAX_ALPHA];
  int f[ORC_MAX_ALPHA], g[ORC_MAX_ALPHA], root;
  for (int k = 0; k < n; ++k) w[k] = fabs((double)c[k]);
  const int ns = huffman_merges(w, n, f, g, &root);
  if (ns < 0) return 0.0f;
  float v[2 * ORC_MAX_ALPHA];
  for (int k = 0; k < n; ++k) v[k] = c[k] * x[k];
  for (int s = 0; s < ns; ++s) v[n + s] = v[f[s]] + v[g[s]];
  return v[root];
}

/* the same in FP64 (coefficients FP64, tree of the |FP32-rounded| entries) */
static double huff_dot_f64(const double* c, const double* x, int n) {
  double w[ORC_MAX_ALPHA];
  int f[ORC_MAX_ALPHA], g[ORC_MAX_ALPHA], root;
  for (int k = 0; k < n; ++k) w[k] = fabs((double)(float)c[k]);
  const int ns = huffman_merges(w, n, f, g, &root);
  if (ns < 0) return 0.0;
  double v[2 * ORC_MAX_ALPHA];
  for (int k = 0; k < n; ++k) v[k] = c[k] * x[k];
  for (int s = 0; s < ns; ++s) v[n + s] = v[f[s]] + v[g[s]];
  return v[root];
}

float orc_huffman_dot_f32(const float* c, const float* x, int n) {
  if (n < 1 || n > ORC_MAX_ALPHA) return NAN;
  return huff_dot_f32(c, x, n);
}

typedef struct {
  int m, r, A;
  double ATd[ORC_MAX_ALPHA * ORC_MAX_ALPHA], Gd[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  double BTd[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  float AT[ORC_MAX_ALPHA * ORC_MAX_ALPHA], G[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  float BT[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
} ord_mats;

static int build_ord(const double* points, int m, int r, ord_mats* M) {
  const int st = orc_make_matrices(points, m, r, M->ATd, M->Gd, M->BTd);
  if (st < 0) return st;
  M->m = m; M->r = r; M->A = st;
  for (int i = 0; i < m * st; ++i) M->AT[i] = (float)M->ATd[i];
  for (int i = 0; i < st * r; ++i) M->G[i] = (float)M->Gd[i];
  for (int i = 0; i < st * st; ++i) M->BT[i] = (float)M->BTd[i];
  return 0;
}

/* One tile in ORC_ORDER_HUFFMAN (mixed = 0) or ORC_ORDER_HUFFMAN_MIXED. */
static void tile_order(const ord_mats* M, int dim, const float* g, const float* d, float* y,
                       int mixed) {
  const int m = M->m, r = M->r, A = M->A;
  float xs[ORC_MAX_ALPHA];
  double xd[ORC_MAX_ALPHA];
  if (dim == 1) {
    float p[ORC_MAX_ALPHA];
    for (int i = 0; i < A; ++i) {
      float u, v;
      if (mixed) {
        for (int k = 0; k < r; ++k) xd[k] = g[k];
        u = (float)huff_dot_f64(&M->Gd[i * r], xd, r);
        for (int l = 0; l < A; ++l) xd[l] = d[l];
        v = (float)huff_dot_f64(&M->BTd[i * A], xd, A);
      } else {
        u = huff_dot_f32(&M->G[i * r], g, r);
        v = huff_dot_f32(&M->BT[i * A], d, A);
      }
      p[i] = u * v;
    }
    for (int j = 0; j < m; ++j) {
      if (mixed) {
        for (int i = 0; i < A; ++i) xd[i] = p[i];
        y[j] = (float)huff_dot_f64(&M->ATd[j * A], xd, A);
      } else {
        y[j] = huff_dot_f32(&M->AT[j * A], p, A);
      }
    }
    return;
  }
  /* 2D: W = G g, U = W G^T, T = B^T d, V = T B, P = U .* V, Z = A^T P,
   * Y = Z A; each entry one Huffman dot product over a matrix row. */
  float Wf[ORC_MAX_ALPHA * 5], U[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  float Tf[ORC_MAX_ALPHA * ORC_MAX_ALPHA], V[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  float P[ORC_MAX_ALPHA * ORC_MAX_ALPHA], Zf[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  double Wd[ORC_MAX_ALPHA * 5], Td[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  double Zd[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (int i = 0; i < A; ++i) /* W[i][k] = sum_l G[i][l] g[l][k] */
    for (int k = 0; k < r; ++k) {
      if (mixed) {
        for (int l = 0; l < r; ++l) xd[l] = g[l * r + k];
        Wd[i * r + k] = huff_dot_f64(&M->Gd[i * r], xd, r);
      } else {
        for (int l = 0; l < r; ++l) xs[l] = g[l * r + k];
        Wf[i * r + k] = huff_dot_f32(&M->G[i * r], xs, r);
      }
    }
  for (int i = 0; i < A; ++i) /* U[i][j] = sum_k W[i][k] G[j][k] */
    for (int j = 0; j < A; ++j)
      U[i * A + j] = mixed ? (float)huff_dot_f64(&M->Gd[j * r], &Wd[i * r], r)
                           : huff_dot_f32(&M->G[j * r], &Wf[i * r], r);
  for (int i = 0; i < A; ++i) /* T[i][l] = sum_k BT[i][k] d[k][l] */
    for (int l = 0; l < A; ++l) {
      if (mixed) {
        for (int k = 0; k < A; ++k) xd[k] = d[k * A + l];
        Td[i * A + l] = huff_dot_f64(&M->BTd[i * A], xd, A);
      } else {
        for (int k = 0; k < A; ++k) xs[k] = d[k * A + l];
        Tf[i * A + l] = huff_dot_f32(&M->BT[i * A], xs, A);
      }
    }
  for (int i = 0; i < A; ++i) /* V[i][j] = sum_l T[i][l] BT[j][l] */
    for (int j = 0; j < A; ++j)
      V[i * A + j] = mixed ? (float)huff_dot_f64(&M->BTd[j * A], &Td[i * A], A)
                           : huff_dot_f32(&M->BT[j * A], &Tf[i * A], A);
  for (int i = 0; i < A * A; ++i) P[i] = U[i] * V[i]; /* Hadamard, FP32 */
  for (int a = 0; a < m; ++a) /* Z[a][j] = sum_i AT[a][i] P[i][j] */
    for (int j = 0; j < A; ++j) {
      if (mixed) {
        for (int i = 0; i < A; ++i) xd[i] = P[i * A + j];
        Zd[a * A + j] = huff_dot_f64(&M->ATd[a * A], xd, A);
      } else {
        for (int i = 0; i < A; ++i) xs[i] = P[i * A + j];
        Zf[a * A + j] = huff_dot_f32(&M->AT[a * A], xs, A);
      }
    }
  for (int a = 0; a < m; ++a) /* Y[a][b] = sum_j Z[a][j] AT[b][j] */
    for (int b = 0; b < m; ++b)
      y[a * m + b] = mixed ? (float)huff_dot_f64(&M->ATd[b * A], &Zd[a * A], A)
                           : huff_dot_f32(&M->AT[b * A], &Zf[a * A], A);
}

int orc_tile_order(int dim, const double* points, int m, int r, const float* g,
                   const float* d, float* y, int order) {
  if (dim < 1 || dim > 2 || r > 5 || order < ORC_ORDER_HUFFMAN || order > ORC_ORDER_HUFFMAN_MIXED)
    return -1;
  ord_mats M;
  const int st = build_ord(points, m, r, &M);
  if (st < 0) return st;
  tile_order(&M, dim, g, d, y, order == ORC_ORDER_HUFFMAN_MIXED);
  return 0;
}

int orc_pointset_error_order(int dim, int m, int r, const double* points, int n_sets,
                             int trials, uint64_t seed, int order, double* err_out) {
  if (order == ORC_ORDER_FMA)
    return orc_pointset_error(dim, m, r, points, n_sets, trials, seed, err_out);
  const int A = m + r - 1;
  if (dim < 1 || dim > 2 || A < 2 || A > ORC_MAX_ALPHA || r > 5 || n_sets < 0 || trials < 1 ||
      order < ORC_ORDER_HUFFMAN || order > ORC_ORDER_HUFFMAN_MIXED)
    return -1;
  orc_size s = {dim, m, r, 1.0};
  size_data sd;
  memset(&sd, 0, sizeof(sd));
  int rc = build_size_data(&s, trials, seed, &sd);
  for (int q = 0; q < n_sets && rc == 0; ++q) {
    ord_mats M;
    const int st = build_ord(points + (size_t)q * A, m, r, &M);
    if (st == -2) { err_out[q] = INFINITY; continue; }
    if (st < 0) { err_out[q] = NAN; continue; }
    double num = 0.0;
    float yh[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
    for (int t = 0; t < trials; ++t) {
      tile_order(&M, dim, sd.g + (size_t)t * sd.nin_g, sd.d + (size_t)t * sd.nin_d, yh,
                 order == ORC_ORDER_HUFFMAN_MIXED);
      for (int j = 0; j < sd.nout; ++j) num += fabs((double)yh[j] - sd.y[(size_t)t * sd.nout + j]);
    }
    err_out[q] = num / sd.ysum;
  }
  free(sd.g); free(sd.d); free(sd.y);
  return rc;
}

double orc_direct_error(int dim, int m, int r, int trials, uint64_t seed) {
  orc_size s = {dim, m, r, 1.0};
  size_data sd;
  memset(&sd, 0, sizeof(sd));
  if (build_size_data(&s, trials, seed, &sd) != 0) return NAN;
  double num = 0.0;
  float yh[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (int t = 0; t < trials; ++t) {
    orc_tile_direct_f32(dim, m, r, sd.g + (size_t)t * sd.nin_g, sd.d + (size_t)t * sd.nin_d, yh);
    for (int j = 0; j < sd.nout; ++j) num += fabs((double)yh[j] - sd.y[(size_t)t * sd.nout + j]);
  }
  double e = num / sd.ysum;
  free(sd.g); free(sd.d); free(sd.y);
  return e;
}

/* ------------------------------------------------------------------------ */
/* Selected tiles of the FP32 Winograd layer (for full-size spot checks).   */
/* Same operation order as orc_wino_layer (f32 contraction only).           */
/* ------------------------------------------------------------------------ */

static void filter_one(int dim, int A, int r, const float* G, const float* g, float* out) {
  if (dim == 1) {
    for (int i = 0; i < A; ++i) {
      float acc = 0.0f;
      for (int q = 0; q < r; ++q) acc = fmaf(G[i * r + q], g[q], acc);
      out[i] = acc;
    }
    return;
  }
  float Wk[ORC_MAX_ALPHA * 5];
  for (int i = 0; i < A; ++i)
    for (int q = 0; q < r; ++q) {
      float acc = 0.0f;
      for (int l = 0; l < r; ++l) acc = fmaf(G[i * r + l], g[l * r + q], acc);
      Wk[i * r + q] = acc;
    }
  for (int i = 0; i < A; ++i)
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
      for (int q = 0; q < r; ++q) acc = fmaf(Wk[i * r + q], G[j * r + q], acc);
      out[i * A + j] = acc;
    }
}

static void input_one(int dim, int A, const float* BT, const float* d, float* out) {
  if (dim == 1) {
    for (int i = 0; i < A; ++i) {
      float acc = 0.0f;
      for (int l = 0; l < A; ++l) acc = fmaf(BT[i * A + l], d[l], acc);
      out[i] = acc;
    }
    return;
  }
  float Tm[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (int i = 0; i < A; ++i)
    for (int l = 0; l < A; ++l) {
      float acc = 0.0f;
      for (int q = 0; q < A; ++q) acc = fmaf(BT[i * A + q], d[q * A + l], acc);
      Tm[i * A + l] = acc;
    }
  for (int i = 0; i < A; ++i)
    for (int j = 0; j < A; ++j) {
      float acc = 0.0f;
      for (int l = 0; l < A; ++l) acc = fmaf(Tm[i * A + l], BT[j * A + l], acc);
      out[i * A + j] = acc;
    }
}

int orc_wino_layer_tiles(const float* x, const float* w, int dim, int N, int C, int K, int H,
                         int W, int pad, const double* points, int m, int r, int n_sel,
                         const int64_t* sel, float* out, int lowp) {
  const int A = m + r - 1;
  double ATd[ORC_MAX_ALPHA * ORC_MAX_ALPHA], Gd[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  double BTd[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  int st = orc_make_matrices(points, m, r, ATd, Gd, BTd);
  if (st < 0) return st;
  float AT[ORC_MAX_ALPHA * ORC_MAX_ALPHA], G[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  float BT[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (int i = 0; i < m * A; ++i) AT[i] = (float)ATd[i];
  for (int i = 0; i < A * r; ++i) G[i] = (float)Gd[i];
  for (int i = 0; i < A * A; ++i) BT[i] = (float)BTd[i];
  const int Hin = (dim == 1) ? 1 : H;
  const int Ho = (dim == 1) ? 1 : H + 2 * pad - r + 1;
  const int Wo = W + 2 * pad - r + 1;
  const int padh = (dim == 1) ? 0 : pad;
  const int th = (dim == 1) ? 1 : (Ho + m - 1) / m;
  const int tw = (Wo + m - 1) / m;
  const int F = (dim == 1) ? A : A * A;
  const int rw = (dim == 1) ? r : r * r;
  const int no = (dim == 1) ? m : m * m;
  float d[ORC_MAX_ALPHA * ORC_MAX_ALPHA], U[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  float Vf[ORC_MAX_ALPHA * ORC_MAX_ALPHA], Mf[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  /* precision form: the scales of orc_wino_layer -- U's from the B^T row
     norms, V's from max |V[f]| over every (c, k) of the layer */
  float sU[ORC_MAX_ALPHA * ORC_MAX_ALPHA], sV[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (int f = 0; f < F; ++f) { sU[f] = 1.0f; sV[f] = 1.0f; }
  if (lowp != 0) {
    double rown[ORC_MAX_ALPHA], vmax[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
    for (int i = 0; i < A; ++i) {
      double sr = 0.0;
      for (int l = 0; l < A; ++l) sr += fabs((double)BT[i * A + l]);
      rown[i] = sr;
    }
    for (int f = 0; f < F; ++f) vmax[f] = 0.0;
    for (int k = 0; k < K; ++k)
      for (int c = 0; c < C; ++c) {
        filter_one(dim, A, r, G, w + ((size_t)k * C + c) * rw, Vf);
        for (int f = 0; f < F; ++f)
          if (fabs((double)Vf[f]) > vmax[f]) vmax[f] = fabs((double)Vf[f]);
      }
    for (int f = 0; f < F; ++f) {
      sU[f] = pow2_normaliser((dim == 1) ? rown[f] : rown[f / A] * rown[f % A]);
      sV[f] = pow2_normaliser(vmax[f]);
    }
  }
  float Ml[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
  for (int s = 0; s < n_sel; ++s) {
    const int64_t t = sel[2 * s];
    const int k = (int)sel[2 * s + 1];
    const int n = (int)(t / ((int64_t)th * tw));
    const int ti = (int)((t / tw) % th), tj = (int)(t % tw);
    if (n < 0 || n >= N || k < 0 || k >= K) return -1;
    for (int f = 0; f < F; ++f) Mf[f] = Ml[f] = 0.0f;
    for (int c = 0; c < C; ++c) {
      const int pr = (dim == 1) ? 1 : A;
      for (int i = 0; i < pr; ++i)
        for (int j = 0; j < A; ++j) {
          int hh = ti * m - padh + i, ww = tj * m - pad + j;
          float v = 0.0f;
          if (hh >= 0 && hh < Hin && ww >= 0 && ww < W)
            v = x[(((size_t)n * C + c) * Hin + hh) * W + ww];
          d[i * A + j] = v;
        }
      input_one(dim, A, BT, d, U);
      filter_one(dim, A, r, G, w + ((size_t)k * C + c) * rw, Vf);
      for (int f = 0; f < F; ++f) mac_lowp(lowp, U[f], Vf[f], sU[f], sV[f], &Mf[f], &Ml[f]);
    }
    for (int f = 0; f < F; ++f) Mf[f] = finish_lowp(lowp, Mf[f], Ml[f], sU[f], sV[f]);
    float* o = out + (size_t)s * no;
    if (dim == 1) {
      for (int j = 0; j < m; ++j) {
        float acc = 0.0f;
        for (int i = 0; i < A; ++i) acc = fmaf(AT[j * A + i], Mf[i], acc);
        o[j] = acc;
      }
    } else {
      float Z[ORC_MAX_ALPHA * ORC_MAX_ALPHA];
      for (int a = 0; a < m; ++a)
        for (int j = 0; j < A; ++j) {
          float acc = 0.0f;
          for (int i = 0; i < A; ++i) acc = fmaf(AT[a * A + i], Mf[i * A + j], acc);
          Z[a * A + j] = acc;
        }
      for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
          float acc = 0.0f;
          for (int j = 0; j < A; ++j) acc = fmaf(Z[a * A + j], AT[b * A + j], acc);
          o[a * m + b] = acc;
        }
    }
  }
  return 0;
}
