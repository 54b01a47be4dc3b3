/*
 * wino_oracle.h -- plain CPU oracle for Winograd point selection.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct statement
 * of what the GPU library computes.  Only tests/, __graft_entry__.smoke()
 * and bench.py's CPU-baseline leg may load it.  It shares no code, header,
 * table or helper with the library under paper_2201_10369_gb300/.
 *
 * Parity status of every function is given beside it ("pinned by" names the
 * independent checks in tests/).
 */
#ifndef WINO_ORACLE_H
#define WINO_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_ALPHA 12

/* Modified Toom-Cook matrices in FP64 (Sec. 4.1 Eqs. (10)-(11), Sec. 4.2
 * Eq. (19)).  `points` holds alpha = m+r-1 values, exactly one +INFINITY.
 * Returns alpha, -1 on bad input, -2 on equal finite points.
 * Pinned by: exactness tensor, Eqs. (26)-(30) symbolic matrices, Lavin's
 * F(2,3), rational build (tests/test_oracle_matrices.py).                 */
int orc_make_matrices(const double* points, int m, int r,
                      double* AT, double* G, double* BT);

/* Canonical order: finite points ascending, infinity last.  Returns alpha
 * or -1 when the count of infinities is not one or a value is NaN.         */
int orc_canonical_points(const double* points, int alpha, double* out);

/* FP64 direct correlation, Eq. (1) (dim 2) and Eq. (2) read as correlation
 * (dim 1, H = 1).  x[N][C][H][W], w[K][C][r(^2)], y[N][K][Ho][Wo] (FP64).
 * Pinned by: exact rational brute force, delta kernel.                     */
void orc_direct_f64(const float* x, const float* w, double* y, int dim,
                    int N, int C, int K, int H, int W, int pad, int r);

/* FP32 single-tile Winograd, Eq. (8) (1D) and Eq. (9) (2D), in the fixed
 * FP32 operation order documented in the .c file.  Matrices are FP32.
 * g: r (1D) or r*r (2D); d: alpha or alpha*alpha; y: m or m*m.
 * Pinned by: rational exactness of the same algebra, error bound vs FP64. */
void orc_tile1d_f32(const float* AT, const float* G, const float* BT,
                    int m, int r, const float* g, const float* d, float* y);
void orc_tile2d_f32(const float* AT, const float* G, const float* BT,
                    int m, int r, const float* g, const float* d, float* y);

/* FP32 direct correlation of one tile (the "n = 0" rows of Tables 7-8). */
void orc_tile_direct_f32(int dim, int m, int r, const float* g,
                         const float* d, float* y);

/* FP32 Winograd layer (Eq. (9) per m x m tile, alpha^2 Hadamard products
 * summed over C in ascending c with fmaf).  dim = 1 uses H = 1 and w[K][C][r].
 * `lowp` selects the contraction operands: 0 FP32, 1 BF16, 2 FP16 (with the
 * per-frequency power-of-two scales of the precision form), 3 split BF16x3,
 * 4 split BF16x6 (hi, mid, lo; hh summed in one accumulator, hm, mh, hl, lh,
 * mm in a second, the two added at the end).
 * Returns 0, or -1 / -2 like orc_make_matrices.
 * Pinned by: FP64 direct within the FP32 Winograd error scale; equals the
 * tile function bit for bit when C = K = 1.                                */
int orc_wino_layer(const float* x, const float* w, float* y, int dim,
                   int N, int C, int K, int H, int W, int pad,
                   const double* points, int m, int r, int lowp);

/* The same layer evaluated only for selected (tile, k) pairs:
 * sel[2s] = linear tile index (n, tile row, tile column), sel[2s+1] = k;
 * out[s] receives the tile's m (1D) or m*m (2D) outputs, including those a
 * ragged tile crops; `lowp` is orc_wino_layer's (the scales are the whole
 * layer's).  Pinned by: equals orc_wino_layer bit for bit on every tile of
 * small layers, in every lowp mode.                                        */
int orc_wino_layer_tiles(const float* x, const float* w, int dim, int N, int C, int K,
                         int H, int W, int pad, const double* points, int m, int r,
                         int n_sel, const int64_t* sel, float* out, int lowp);

/* SplitMix64 (Steele, Lea, Flood 2014): the n-th output of the generator
 * whose state starts at `seed`.  Pinned by published output values.        */
uint64_t orc_splitmix64(uint64_t seed, uint64_t n);

/* Uniform [-1, 1) FP32 value of trial input `idx` (idx < 256: kernel g,
 * idx >= 256: data d) of trial `trial` of size (dim, m, r).                */
float orc_trial_value(uint64_t seed, int dim, int m, int r, int trial,
                      int idx);

/* Point set of (size, mask, c): {0, inf} plus the mask's slots of
 * [-1/c, -c, c, 1/c, -1/d, -d, d, 1/d].  Writes alpha points and returns
 * alpha, or -1 when the mask is invalid for the size.                      */
int orc_mask_points(int dim, int m, int r, double d, unsigned mask,
                    double c, double* points);

typedef struct {
  int dim, m, r;
  double d;
} orc_size;

/* The batched error sweep (Sec. 6): err_out[n_sizes][n_masks][n_c] =
 *   sum_t ||yhat_t - y_t||_1 / sum_t ||y_t||_1   (FP64, exact widening),
 * NaN for invalid masks, +INF for coinciding points.  `c_stride` > 1
 * evaluates only every c_stride-th c (the rest are left untouched).
 * `n_threads` >= 1 splits instances over POSIX threads.  Returns 0.        */
int orc_error_sweep(const double* c_grid, int n_c, const orc_size* sizes,
                    int n_sizes, const unsigned char* masks, int n_masks,
                    int trials, uint64_t seed, double* err_out,
                    int c_stride, int n_threads);

/* The same metric for explicit point sets (the comparison sets of Tables
 * 7-8, Chebyshev nodes): err_out[q] for points[q * alpha .. + alpha)
 * (alpha = m + r - 1 values, one +INFINITY, any order), on the trials the
 * sweep draws for size (dim, m, r).  +INF for coinciding points, NaN for an
 * invalid set.  Returns 0, -1 on bad arguments.                           */
int orc_pointset_error(int dim, int m, int r, const double* points, int n_sets, int trials,
                       uint64_t seed, double* err_out);

/* Kronecker-product form of the 2D Winograd tile (Sec. 7):
 *   u = (G (x) G) vec(g), v = (B^T (x) B^T) vec(d), y = (A^T (x) A^T)(u .* v),
 * row-major vec; Kronecker entries = FP64 products of the FP64 matrix entries
 * rounded once to FP32; each row summed with fmaf (column ascending), or
 * with pairwise = 1 as rounded products summed pairwise (split at ceil(n/2)).
 * orc_tile2d_kron: one tile (g r x r, d alpha x alpha, y m x m, row-major);
 * returns 0 or -1 / -2 like orc_make_matrices.  orc_pointset_error_kron: the
 * sweep metric on the sweep's 2D trials of size (m, r), like
 * orc_pointset_error.                                                      */
int orc_tile2d_kron(const double* points, int m, int r, const float* g, const float* d,
                    float* y, int pairwise);
int orc_pointset_error_kron(int m, int r, const double* points, int n_sets, int trials,
                            uint64_t seed, int pairwise, double* err_out);

/* Summation-order variants (Sec. 5; the order the paper's tables use, from
 * Barabasz et al., which the paper does not define -- the reading is stated
 * at the definitions in the .c file):
 *   ORC_ORDER_FMA            the order of orc_tile1d_f32 / orc_tile2d_f32;
 *   ORC_ORDER_HUFFMAN        every transform dot product summed in FP32
 *                            along the Huffman tree of its |coefficients|;
 *   ORC_ORDER_HUFFMAN_MIXED  the same trees, transforms in FP64, Hadamard
 *                            product in FP32.
 * orc_huffman_merges: the tree over the leaves k with w[k] > 0 as a merge
 * list (leaf k = id k, merge s creates id n + s); returns the merge count or
 * -1.  Pinned by: optimal weighted path length against brute force, the
 * tie rule on equal weights.
 * orc_huffman_dot_f32: sum c[k] x[k] along that tree, FP32.  Pinned by: a
 * worked example whose FP32 result differs from every sequential order,
 * and sequential ascending-magnitude summation when every weight exceeds
 * the sum of the smaller ones.
 * orc_tile_order: one tile (layout of orc_tile2d_kron; 1D: g r, d alpha,
 * y m) in ORC_ORDER_HUFFMAN or ORC_ORDER_HUFFMAN_MIXED; returns 0 or -1 /
 * -2 like orc_make_matrices.  Pinned by: exact correlation on inputs where
 * no operation rounds (both orders); MIXED equals the rational transforms
 * of the FP64 matrices rounded to FP32 at U, V, P and Y.
 * orc_pointset_error_order: the sweep metric of orc_pointset_error in one of
 * the three orders.                                                        */
#define ORC_ORDER_FMA 0
#define ORC_ORDER_HUFFMAN 1
#define ORC_ORDER_HUFFMAN_MIXED 2
int orc_huffman_merges(const double* w, int n, int* first, int* second);
float orc_huffman_dot_f32(const float* c, const float* x, int n);
int orc_tile_order(int dim, const double* points, int m, int r, const float* g,
                   const float* d, float* y, int order);
int orc_pointset_error_order(int dim, int m, int r, const double* points, int n_sets,
                             int trials, uint64_t seed, int order, double* err_out);

/* The same metric for FP32 direct correlation (the "n = 0" row).         */
double orc_direct_error(int dim, int m, int r, int trials, uint64_t seed);

/* BF16 / FP16 round-to-nearest-even of an FP32 value, returned as FP32. */
float orc_round_bf16(float v);
float orc_round_fp16(float v);

#ifdef __cplusplus
}
#endif
#endif
