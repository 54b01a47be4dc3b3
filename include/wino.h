/*
 * wino.h -- C ABI of the GB300 Winograd point-selection library.
 *
 * The library computes Toom-Cook / Winograd convolution F(m, r) and
 * F(m x m, r x r) with transform matrices built from a caller-chosen point
 * set (Alam, Anderson, Barabasz, Gregg, "Winograd Convolution for Deep Neural
 * Networks: Efficient Point Selection"), and the batched FP32-versus-FP64
 * error sweep over the point parameter c that the paper uses to pick points
 * (Sec. 6).
 *
 * Conventions shared by every entry point
 *  - Every call returns a wino_status; nothing is thrown across the ABI.
 *    wino_last_error() returns a thread-local text for the last failure.
 *  - Device pointers are plain CUDA device addresses (for example a torch
 *    tensor's data_ptr()), contiguous, row-major, owned by the caller.
 *  - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  The device work of a call is ordered on that stream: it starts
 *    after the work already enqueued there, and work enqueued there later
 *    starts after it.  Parts of it may run on the library's internal streams
 *    (the layers' filter transforms, the sweep's sizes), forked from and
 *    joined back to that stream by events, so the ordering holds for them
 *    too.  The call returns without synchronising, unless stated otherwise.
 *    Calls that run at the same time from several host threads share those
 *    internal streams and the library's scratch.
 *  - The library keeps internal scratch (allocated on first use and grown
 *    when needed, or caller-provided through wino_set_workspace) and releases
 *    it in wino_shutdown().  It never frees caller memory.
 *  - There is no CPU fallback: when no sm_103 device is present the GPU
 *    entry points return WINO_EUNSUPPORTED.
 *  - Point sets: alpha = m + r - 1 doubles holding alpha-1 distinct finite
 *    points and exactly one +INFINITY, in any order.  The library sorts the
 *    finite points ascending and puts infinity last (the modified Toom-Cook
 *    construction of Sec. 4.2 treats infinity as the extra point).
 */
#ifndef WINO_H
#define WINO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WINO_OK = 0,
  WINO_EINVAL = -1,        /* bad argument: size, null pointer, dtype      */
  WINO_ESINGULAR = -2,     /* two finite points equal (Vandermonde singular) */
  WINO_ENOMEM = -3,        /* scratch could not be allocated / is too small */
  WINO_ECUDA = -4,         /* a CUDA runtime call failed                    */
  WINO_ETIMEOUT = -5,      /* a bounded device wait gave up                 */
  WINO_EUNSUPPORTED = -6   /* no sm_103 device, or unsupported combination  */
} wino_status;

/* Arithmetic of the Winograd-domain contraction (the alpha^2 GEMMs).
 * Transforms are FP32 in every form; only the contraction changes.        */
typedef enum {
  WINO_F32 = 0,            /* FP32 SIMT fused multiply-add                  */
  WINO_BF16_TC = 1,        /* BF16 operands on tcgen05, FP32 accumulate     */
  WINO_FP16_TC = 2,        /* FP16 operands on tcgen05, FP32 accumulate     */
  WINO_SPLIT_BF16X3 = 3,   /* hi/lo BF16 split, 3 tcgen05 products, FP32 acc */
  WINO_SPLIT_BF16X6 = 4    /* hi/mid/lo BF16 split (all 24 bits of an FP32
                              operand), the 6 tcgen05 products down to 2^-16
                              relative: hh into one FP32 accumulator, hm, mh,
                              hl, lh, mm into a second, added at the end    */
} wino_dtype;

/* Largest alpha = m + r - 1 the library accepts. */
#define WINO_MAX_ALPHA 12

/* ---------------------------------------------------------------------- */
/* Transform matrices (host, FP64).                                        */
/* ---------------------------------------------------------------------- */

/* Builds the modified Toom-Cook matrices for F(m, r) from `points`
 * (Sec. 4.1 Eqs. (10)-(11) with N_i folded into G; Sec. 4.2 Eq. (19) for the
 * point at infinity):
 *   G [alpha][r]    : G[i][k]  = a_i^k / N_i,  N_i = prod_{j != i}(a_i - a_j);
 *                     last row e_{r-1}
 *   AT[m][alpha]    : AT[j][i] = a_i^j; last column e_{m-1}
 *   BT[alpha][alpha]: row i < alpha-1 = ascending coefficients of
 *                     prod_{j != i}(x - a_j); last row = coefficients of
 *                     M'(x) = prod_j (x - a_j)
 * so that Y = AT [(G g) .* (BT d)] (Eq. (8)) is the correlation
 * Y_j = sum_k g_k d_{j+k}.  Rows/columns follow the canonical point order
 * (finite ascending, infinity last).  Outputs are caller-owned host arrays,
 * row-major FP64.  Returns WINO_ESINGULAR on equal finite points, WINO_EINVAL
 * on non-finite points other than one +INFINITY, on m < 1, r < 1 or
 * alpha > WINO_MAX_ALPHA.  Pure host code; needs no GPU.                   */
int wino_make_matrices(const double* points, int m, int r,
                       double* AT, double* G, double* BT);

/* ---------------------------------------------------------------------- */
/* Winograd convolution layer (device).                                     */
/* ---------------------------------------------------------------------- */

/* 1D layer, Eq. (8) applied per tile of m outputs (tiles overlap by r-1,
 * stride m, zero padding `pad`, ragged last tile zero-filled):
 *   x[N][C][L], w[K][C][r], y[N][K][Lo], Lo = L + 2*pad - r + 1,
 *   y[n][k][o] = sum_c sum_u x[n][c][o+u-pad] * w[k][c][u]   (stride 1).
 * x, w, y are FP32 device arrays; `dtype` selects the contraction.        */
int wino_conv1d(const void* x, const void* w, void* y,
                int N, int C, int K, int L, int pad,
                const double* points, int m, int r, int dtype,
                void* cuda_stream);

/* 2D layer, Eq. (9) per m x m output tile; the per-tile Hadamard products
 * summed over C_in form alpha^2 independent GEMMs (Sec. 4.1):
 *   x[N][C][H][W], w[K][C][r][r], y[N][K][Ho][Wo], Ho = H+2pad-r+1,
 *   Wo = W+2pad-r+1, y[n][k][p][q] = sum_{c,u,v} x[n][c][p+u-pad][q+v-pad]
 *   * w[k][c][u][v]   (Eq. (1), stride 1).  FP32 device arrays.            */
int wino_conv2d(const void* x, const void* w, void* y,
                int N, int C, int K, int H, int W, int pad,
                const double* points, int m, int r, int dtype,
                void* cuda_stream);

/* Scratch the layer needs for this shape (bytes); 0 on invalid input.     */
size_t wino_workspace_bytes(int N, int C, int K, int H, int W,
                            int m, int r, int dtype);

/* Hands the library caller-owned device scratch of `bytes` bytes, used by
 * later layer calls instead of an internal allocation (NULL, 0 = go back to
 * internal scratch).  A call whose need exceeds it returns WINO_ENOMEM.
 * The caller keeps ownership and must keep it alive while calls using it
 * are in flight.                                                           */
int wino_set_workspace(void* dev_ptr, size_t bytes);

/* FP64 direct correlation, Eq. (1), the reference the paper measures FP32
 * Winograd against (Sec. 6: "normal convolution using double precision").
 * x[N][C][H][W] and w[K][C][r][r] are FP32 device arrays (widened exactly),
 * y64[N][K][Ho][Wo] is an FP64 device array.  dim = 1 treats H as 1 and
 * w as [K][C][r].                                                          */
int wino_direct_conv_f64(const void* x, const void* w, void* y64,
                         int dim, int N, int C, int K, int H, int W,
                         int pad, int r, void* cuda_stream);

/* Error statistics of an FP32 result against its FP64 reference, reduced on
 * the device in FP64 (warp shuffles): out4 (host, FP64) receives
 *   { sum |yhat - y|, sum |y|, max |yhat - y|, max |y| }.
 * A NaN anywhere in yhat (or y) makes the sums and the matching maximum NaN
 * (the maxima propagate NaN rather than skip it).
 * Synchronises `cuda_stream` because the result is a host array.          */
int wino_error_stats(const void* yhat_f32, const void* y_f64, int64_t n,
                     double* out4, void* cuda_stream);

/* ---------------------------------------------------------------------- */
/* Batched point sweep (device), Sec. 6.1-6.3.                              */
/* ---------------------------------------------------------------------- */

/* One problem size of the sweep: 1D F(m, r) (dim = 1) or 2D F(m x m, r x r)
 * (dim = 2); `d` is the fixed second group parameter of Eq. (22).          */
typedef struct {
  int dim, m, r;
  double d;
} wino_size;

/* Subset masks: bit b selects slot b of
 *   [-1/c, -c, c, 1/c, -1/d, -d, d, 1/d]
 * (Eqs. (21)-(25)); the point set is {0, inf} plus the selected slots.  A
 * mask is valid for a size when popcount(mask) = alpha - 2, and, when
 * |d| == 1 (the d-group collapses to {-1, 1}), bits 4 and 7 are clear (bits
 * 5 and 6 stand for -1 and 1).  Invalid (size, mask) pairs are skipped and
 * get NaN.  A c for which two points coincide exactly gets +INFINITY.
 *
 * For every valid (size, mask, c): `trials` single-tile problems with g, d
 * uniform in [-1, 1) drawn from the counter-based SplitMix64 stream of
 * `seed` (the same trials for every mask and c of a size), evaluated with
 * FP32 Winograd (transforms and Hadamard product in FP32, matrices built in
 * FP64 and rounded once) and scored against the FP64 direct correlation:
 *   err = sum_t ||yhat_t - y_t||_1 / sum_t ||y_t||_1.
 * Summation order (the same in wino_error_sweep and every planned-sweep
 * mode, so all return the same bits): per trial the terms in FP32; trials
 * in chunks of 128, each chunk's trial sums accumulated in trial order as a
 * compensated FP32 pair (hi, lo) -- per term (s, r) = TwoSum(hi, e) with
 * s = hi + e, b = s - hi, r = (hi - (s - b)) + (e - b), then hi = s and
 * lo = lo + r, every operation rounded to nearest -- and the chunk's value
 * (double)hi + (double)lo; chunk values added in FP64 in ascending order.
 * The result is within ~1e-10 relative of the exact sum.
 * err_out is a caller-owned HOST array [n_sizes][n_subsets][n_c] (FP64).
 * c_grid, sizes, subsets are host arrays.  Synchronises `cuda_stream`.     */
int wino_error_sweep(const double* c_grid, int n_c,
                     const wino_size* sizes, int n_sizes,
                     const unsigned char* subsets, int n_subsets,
                     int trials, unsigned long long seed,
                     double* err_out, void* cuda_stream);

/* The sweep's metric for explicit point sets (the comparison sets of
 * Tables 7-8, Chebyshev nodes): for each set q, points[q * alpha ..
 * + alpha) (alpha = m + r - 1 values holding one +INFINITY, any order;
 * sorted like wino_make_matrices), err_out[q] = the error of wino_error_sweep
 * on the same trials of size (dim, m, r), in the same summation order (a set
 * that is also a mask instance gets the same bits).  +INFINITY when two
 * points coincide.  Sizes as compiled for the sweep (1D r = 3 m = 2..8, 1D
 * r = 5 m = 2..6, 2D r = 3 m = 2..8, 2D r = 5 m = 2..4), else
 * WINO_EUNSUPPORTED; WINO_EINVAL
 * for a set without exactly one +INFINITY.  points, err_out: host arrays.
 * Synchronises `cuda_stream`.                                              */
int wino_pointset_error(int dim, int m, int r, const double* points, int n_sets,
                        int trials, unsigned long long seed, double* err_out,
                        void* cuda_stream);

/* Summation-order variants of the sweep (Sec. 5: the paper's tables use the
 * Huffman evaluation order of Barabasz et al., and its curves also show that
 * order with the transforms in FP64).  The paper defines neither; the reading
 * implemented:
 *   WINO_ORDER_FMA           the order of wino_error_sweep (fmaf, inner
 *                            index ascending);
 *   WINO_ORDER_HUFFMAN       every output of a transform (one dot product
 *                            over a row of G, B^T or A^T; a 2D transform is
 *                            two passes, left factor first) is the sum of
 *                            its non-zero terms, each a rounded FP32
 *                            product, added along the Huffman tree of the
 *                            terms' |FP32 coefficients|: the two live nodes
 *                            of least weight are replaced by their sum, of
 *                            weight the FP64 sum of theirs; ties go to the
 *                            node created first (leaves in column order,
 *                            then merged nodes in creation order);
 *   WINO_ORDER_HUFFMAN_MIXED the same trees with the FP64 matrices, FP64
 *                            products and sums, the FP32 inputs widened; U
 *                            and V rounded to FP32, the Hadamard product in
 *                            FP32, the output transform in FP64 and Y
 *                            rounded to FP32 once.
 * Error sums of orders 1 and 2: per trial the outputs' errors in FP32
 * (row-major), the trials t = l, l + 32, l + 64, ... summed in FP64 in trial
 * order for each l < 32, and the 32 sums combined by a fixed butterfly
 * (pairs 16 apart, then 8, 4, 2, 1); wino_pointset_error_order uses the
 * same, so a set that is also a mask instance gets the same bits.         */
typedef enum {
  WINO_ORDER_FMA = 0,
  WINO_ORDER_HUFFMAN = 1,
  WINO_ORDER_HUFFMAN_MIXED = 2
} wino_order;

/* wino_error_sweep in one of the summation orders; order WINO_ORDER_FMA is
 * wino_error_sweep itself.  Other order values: WINO_EINVAL.             */
int wino_error_sweep_order(const double* c_grid, int n_c,
                           const wino_size* sizes, int n_sizes,
                           const unsigned char* subsets, int n_subsets,
                           int trials, unsigned long long seed, int order,
                           double* err_out, void* cuda_stream);

/* wino_pointset_error in one of the summation orders.                     */
int wino_pointset_error_order(int dim, int m, int r, const double* points,
                              int n_sets, int trials, unsigned long long seed,
                              int order, double* err_out, void* cuda_stream);

/* The same metric for the Kronecker-product form of the 2D tile (Sec. 7):
 *   u = (G (x) G) vec(g), v = (B^T (x) B^T) vec(d), y = (A^T (x) A^T)(u .* v)
 * (row-major vec), Kronecker entries = FP64 products of the FP64 matrix
 * entries rounded once to FP32, each row summed with fmaf (column ascending)
 * or, pairwise != 0, as rounded products summed pairwise (a sum of n terms
 * splits at ceil(n / 2)).  2D F(m x m, 3 x 3), m = 2..6, on the sweep's 2D
 * trials of that size; points and err_out as for wino_pointset_error; trial
 * errors summed in FP64 in a fixed order.  Synchronises `cuda_stream`.     */
int wino_pointset_error_kron(int m, int r, const double* points, int n_sets,
                             int trials, unsigned long long seed, int pairwise,
                             double* err_out, void* cuda_stream);

/* The FP64 transform matrices the sweep builds on the device for the
 * instances (size, mask, c_k), k < n_c -- the same construction as
 * wino_make_matrices (Sec. 4.1-4.2), run by the sweep's own device code.
 * AT[n_c][m][alpha], G[n_c][alpha][r], BT[n_c][alpha][alpha] are caller-owned
 * HOST arrays; `singular` (host, n_c bytes, may be NULL) receives 1 where two
 * points coincide.  Returns WINO_EINVAL when the mask is invalid for the size.
 * Synchronises `cuda_stream`.                                               */
int wino_instance_matrices(const double* c_grid, int n_c, wino_size size,
                           unsigned mask, double* AT, double* G, double* BT,
                           unsigned char* singular, void* cuda_stream);

/* ---------------------------------------------------------------------- */
/* Subset patterns (Sec. 6.2, Tables 2-6): fixed base points besides 0 and  */
/* infinity joined to a subset of {-1/c, -c, c, 1/c}.                       */
/* ---------------------------------------------------------------------- */

/* One candidate subset of a base, ranked by the query below.              */
typedef struct {
  unsigned char mask;  /* the sweep mask: base bits | subset bits (0-3)     */
  int best_k;          /* grid index of its least error in the window, -1
                          when it has no finite error there                 */
  double best_c;       /* c_grid[best_k] (NaN when best_k < 0)             */
  double best_err;     /* that error (NaN when best_k < 0)                 */
  double win_frac;     /* share of the window's c, among those where every
                          candidate's error is finite, at which this
                          candidate has the least error (ties to the
                          smaller mask); 0 when there are none              */
} wino_pattern_cand;

/* The query behind Tables 2-6 of Sec. 6.2, over one size's sweep errors
 * err[n_masks][n_c] (host; the [size] slice of wino_error_sweep's output for
 * `size`, whose d fixes the d-group values).  A base is a set of d-group
 * slots, base_mask (bits 4-7 only: e.g. d = 3 with bit 6 is the base point
 * 3, with bit 5 the point -3; d = 2 with bit 7 is 1/2; d = 1 with bits 5 and
 * 6 is the pair -1, 1; 0 is no base point besides 0 and infinity).  The
 * candidates are the masks of `masks` whose bits 4-7 equal base_mask and
 * that are valid for the size (popcount alpha - 2; bits 4 and 7 clear when
 * |d| = 1).  Only grid points with c_lo <= c <= c_hi count (c > 1 covers
 * every point set once: a subset at c is its mirror, -c <-> -1/c and
 * c <-> 1/c, at 1/c).  Per candidate: its least finite error in the window
 * (the first grid index on ties) and its win fraction.  cand_out (host,
 * max_cand entries) receives the candidates ordered by best error, then
 * mask, those with no finite error last; *n_cand = the number of
 * candidates (entries beyond max_cand are not written).  The first entry is
 * the base's pattern.  The paper states no procedure; this is the reading
 * that reproduces its tables' layout.  Host code; needs no GPU.
 * WINO_EINVAL for NULL arrays, n_masks or n_c < 1, base_mask bits 0-3 set
 * or a bad size.                                                           */
int wino_subset_pattern(const double* err, const unsigned char* masks, int n_masks,
                        const double* c_grid, int n_c, wino_size size,
                        unsigned char base_mask, double c_lo, double c_hi,
                        wino_pattern_cand* cand_out, int max_cand, int* n_cand);

/* ---------------------------------------------------------------------- */
/* FP32 layer without allocation.                                           */
/* ---------------------------------------------------------------------- */

/* Size (floats) of the fixed scratch array wino_conv2d_f32_noalloc uses:
 * 4 Mi floats = 16 MiB of device memory, held by every device that loads
 * the library until the process exits.                                     */
#define WINO_NOALLOC_SCRATCH_FLOATS (1 << 22)

/* wino_conv2d with dtype WINO_F32, for callers that cannot allocate device
 * memory: code running while a stream is captured into a CUDA graph in
 * global mode (cudaMalloc is refused there), plug-ins inside a framework
 * whose allocator has already reserved the device's memory, and loops whose
 * rules forbid allocation after start-up.  It allocates nothing: its only
 * scratch (the transformed filters, alpha^2 * C * K floats) lives in a fixed
 * array compiled into the library.  The paper has no counterpart; this is
 * a deployment convenience around the same fused kernel.
 * Arguments and results are those of wino_conv2d.  Supported: r = 3,
 * m in {2, 4, 6}, K a multiple of 64, alpha^2 * C * K <=
 * WINO_NOALLOC_SCRATCH_FLOATS; anything else returns WINO_EINVAL with the
 * reason in wino_last_error().  The first call on each device looks up the
 * array's device address and prepares the kernel, so make it before any
 * stream capture.  All calls share the array: calls whose GPU work may
 * overlap (other streams, other host threads) race on it and must be
 * ordered by the caller.                                                   */
int wino_conv2d_f32_noalloc(const void* x, const void* w, void* y,
                            int N, int C, int K, int H, int W, int pad,
                            const double* points, int m, int r,
                            void* cuda_stream);

/* ---------------------------------------------------------------------- */
/* Planned sweep: one persistent launch in a CUDA graph (Sec. 6.2-6.3      */
/* searches run as explicit instance lists).                               */
/* ---------------------------------------------------------------------- */

/* One instance: sizes[size] with the point set of `mask` at parameter c
 * (same point rule as wino_error_sweep).                                    */
typedef struct {
  int size;
  unsigned char mask;
  double c;
} wino_instance;

enum {
  WINO_SWEEP_AUTO = 0,         /* time the modes below once, keep the best */
  WINO_SWEEP_PERSISTENT = 1,   /* one persistent launch, LPT work queue    */
  WINO_SWEEP_PERSISTENT3 = 2,  /* same, 3 CTAs/SM (register-capped)        */
  WINO_SWEEP_PER_SIZE = 3      /* one launch per size, sizes on 3 streams  */
};

/* Builds a plan evaluating every instance with `trials` trials of `seed`
 * (the same trial inputs and metric as wino_error_sweep), captures it in a
 * CUDA graph on the current device and returns an opaque handle in *plan.
 * Instances whose mask is invalid for their size are not evaluated (NaN).
 * With mode WINO_SWEEP_AUTO the call first times each mode on this plan
 * (cached per plan shape for the process).  Allocates device and pinned host
 * memory owned by the plan.                                                */
int wino_sweep_plan_create(const wino_size* sizes, int n_sizes,
                           const wino_instance* inst, int64_t n_inst,
                           int trials, unsigned long long seed, int mode,
                           void** plan);

/* Optional watchdog: a later run stops taking work `max_ms` milliseconds of
 * device time after its launch and returns WINO_ETIMEOUT (instances not
 * reached are NaN).  0 disables it.                                         */
int wino_sweep_plan_set_deadline(void* plan, double max_ms);

/* Launches the plan's graph on `cuda_stream` (NULL = the plan's own stream),
 * waits for it and writes err_out[n_inst] (host, FP64) in the caller's
 * instance order.                                                          */
int wino_sweep_plan_run(void* plan, double* err_out, void* cuda_stream);

/* Replaces the c of every instance (c[n_inst], host, the caller's instance
 * order) keeping sizes and masks, so the plan and its graph are reused;
 * synchronises the plan's stream.                                          */
int wino_sweep_plan_set_c(void* plan, const double* c, int64_t n);

/* The mode the plan runs, its persistent grid size and its work items.    */
int wino_sweep_plan_info(void* plan, int* mode, int* grid, int* n_items);

void wino_sweep_plan_destroy(void* plan);

/* ---------------------------------------------------------------------- */
/* Learned surrogate of the sweep.  The paper has no surrogate; its         */
/* observation that the error curve over c is roughly smooth (Sec. 6.1)     */
/* motivates ranking a dense c grid with a small network and evaluating     */
/* only the best candidates exactly.                                        */
/* ---------------------------------------------------------------------- */

#define WINO_MLP_INPUTS 16
#define WINO_MLP_HIDDEN 64
#define WINO_MLP_PARAMS 1153 /* W1 64x16 | b1 64 | w2 64 | b2 1 */

/* f(x) = w2 . gelu(W1 x + b1) + b2, gelu(z) = z (1 + erf(z / sqrt 2)) / 2,
 * predicting log10 of an instance's sweep error.  FP32 master parameters,
 * BF16-rounded working copy used by the forward and backward passes; MSE
 * loss; Adam (beta1 0.9, beta2 0.999, eps 1e-8).  Creates a network with
 * uniform(-sqrt(6/fan_in), +) weights and zero biases from `seed`.       */
int wino_mlp_create(unsigned long long seed, void** mlp);
/* Host arrays of WINO_MLP_PARAMS floats; set resets the Adam state.      */
int wino_mlp_set_params(void* mlp, const float* params);
int wino_mlp_get_params(void* mlp, float* params, int working);
/* Features X[n][16] (device) of instances (host array):
 * [m/8, (r-3)/2, mask bits 0..7, u, dim - 1, u^2, |u|, u^3, 0] with
 * u = ln c / ln 20.
 * Synchronises `cuda_stream`.                                              */
int wino_mlp_features(const wino_size* sizes, int n_sizes,
                      const wino_instance* inst, int64_t n, float* X,
                      void* cuda_stream);
/* Features of a grid (device X[n_rows * n_c][16], row-major): row q is
 * (sizes[row_size[q]], row_mask[q]) at every c of c_grid.  Host inputs;
 * synchronises `cuda_stream`.                                              */
int wino_mlp_grid_features(const wino_size* sizes, int n_sizes,
                           const int* row_size, const unsigned char* row_mask,
                           int n_rows, const double* c_grid, int n_c, float* X,
                           void* cuda_stream);
/* Mean squared error of the batch (X[B][16], y[B] device) at the working
 * weights and its gradient (host, WINO_MLP_PARAMS floats).               */
int wino_mlp_loss_grad(void* mlp, const float* X, const float* y, int B,
                       float* grad, double* loss, void* cuda_stream);
/* `epochs` passes over n samples (device) in whole batches of `batch`, in
 * order; one epoch is captured as a CUDA graph and replayed.  The batch
 * gradient is summed over blocks of 64 samples in a fixed order (no
 * atomics), so a run is deterministic: the same data, seed and schedule
 * give the same weights.  Grows a per-model buffer of partial gradients
 * (batch / 64 rows of WINO_MLP_PARAMS + 1 floats) on first use.            */
int wino_mlp_train(void* mlp, const float* X, const float* y, int64_t n,
                   int batch, int epochs, float lr, void* cuda_stream);
/* out[n] (device) = f(X[n][16]) at the working weights.                  */
int wino_mlp_predict(void* mlp, const float* X, int64_t n, float* out,
                     void* cuda_stream);
/* Indices of the k smallest values of each row of vals[rows][cols]
 * (device, ascending, ties by index, NaN last) into idx[rows][k] (device);
 * cols <= 8192.                                                            */
int wino_topk_rows(const float* vals, int rows, int cols, int k, int* idx,
                   void* cuda_stream);
void wino_mlp_destroy(void* mlp);

/* Surrogate-guided search of a c grid.  For every (size, mask) pair valid
 * under the rule of wino_error_sweep (a "row"):
 *   1. the network `mlp` ranks every c of c_grid (predict kernel); its `top`
 *      best predictions (top-k kernel) and `probe` random grid points
 *      (SplitMix64 draws of the search's seed and run count) are evaluated
 *      exactly in one planned launch;
 *   2. the 2 refine + 1 grid points centred on the network's best verified
 *      proposal are evaluated in a second planned launch (the error over c
 *      is smooth at large scale but noisy between neighbours, Sec. 6.1);
 *   3. a row whose network region (proposals and refinement) has a least
 *      error above guard x the best random probe is swept exhaustively
 *      (wino_error_sweep): the plain sweep is the fallback and the judge;
 *   4. the row's result is the least error evaluated and its c.
 * The paper has no surrogate; its observation that the error curve is
 * roughly smooth (Sec. 6.1) motivates ranking a dense grid with a network
 * and evaluating only the best candidates exactly.                         */
typedef struct {
  int top;       /* network proposals per row, 1 <= top <= n_c            */
  int probe;     /* random grid points per row, >= 1                      */
  int refine;    /* neighbours on each side of the refined point, >= 0     */
  double guard;  /* fallback threshold factor, >= 1                        */
} wino_guided_params;

typedef struct {
  int64_t evaluated;    /* instances evaluated (fallback rows count n_c)  */
  int rows;             /* valid (size, mask) rows                        */
  int fallback_rows;    /* rows swept exhaustively                        */
  double phase_ms[4];   /* host wall time: rank, verify, refine, fallback */
} wino_guided_stats;

/* Builds a search over sizes x masks x c_grid (host arrays, copied; n_c <=
 * 8192) with `trials` trials of `seed` (the sweep's trials and metric): the
 * grid's features on the device and the two planned launches (their graphs
 * captured once).  `mlp` (a wino_mlp_create handle) is borrowed and must
 * outlive the search.  Allocates device memory owned by the search.        */
int wino_guided_create(void* mlp, const wino_size* sizes, int n_sizes,
                       const unsigned char* masks, int n_masks,
                       const double* c_grid, int n_c, int trials,
                       unsigned long long seed, const wino_guided_params* prm,
                       void** search);
/* One search with the network's present weights.  best_err and best_c are
 * caller-owned host arrays [n_sizes][n_masks] (NaN where the mask is invalid
 * for the size); stats may be NULL.  Every run draws new random probes.
 * Synchronises cuda_stream.                                                */
int wino_guided_run(void* search, double* best_err, double* best_c,
                    wino_guided_stats* stats, void* cuda_stream);
void wino_guided_destroy(void* search);

/* The search without the network, for comparison: `budget` random grid
 * points per valid (size, mask) row (SplitMix64 draws of `seed`) evaluated
 * in one planned launch; best_err (host [n_sizes][n_masks], NaN where
 * invalid) = the least error found per row.  Synchronises cuda_stream.    */
int wino_random_search(const wino_size* sizes, int n_sizes, const unsigned char* masks,
                       int n_masks, const double* c_grid, int n_c, int trials, int budget,
                       unsigned long long seed, double* best_err, void* cuda_stream);

/* The two-parameter sweep (Sec. 4: the group {-1/c, -c, c, 1/c} with a
 * subset of {-1/d, -d, d, 1/d} for larger sizes): err_out (host,
 * [n_d][n_masks][n_c]) = the sweep error of every mask at every (d, c) on
 * the trials of size (dim, m, r) -- the same values as wino_error_sweep with
 * sizes {dim, m, r, d_i} -- NaN where a mask is invalid for that d.  Runs as
 * planned persistent launches of at most 64 d values each (the wide 2D
 * sizes F(7x7,3x3), F(8x8,3x3) as wino_error_sweep calls).  d > 0.
 * Synchronises cuda_stream.                                                */
int wino_cd_sweep(int dim, int m, int r, const double* c_grid, int n_c, const double* d_grid,
                  int n_d, const unsigned char* masks, int n_masks, int trials,
                  unsigned long long seed, double* err_out, void* cuda_stream);

/* ---------------------------------------------------------------------- */
/* Library state.                                                           */
/* ---------------------------------------------------------------------- */

/* Optional CUDA-event timing of the library's kernels: while enabled, every
 * launch records a start/stop event pair on its own stream (skipped during
 * graph capture).  wino_profile_read sums, then forgets, the recorded
 * launches of one kernel ("filter_transform", "input_transform",
 * "wino_gemm", "output_transform", "fused_layer", "tc_gemm", "tc_transform",
 * "sweep_eval", "sweep_prepare", "direct_f64", "error_stats", "mlp",
 * "sweep_order"); it waits for the recorded events.                       */
int wino_profile_enable(int on);
int wino_profile_read(const char* kernel, double* total_ms, int* launches);

/* Number of kernels this library has launched in this process (all
 * devices); a diagnostic for counting launches inside a timed region.      */
unsigned long long wino_kernel_launches(void);

/* Measured arithmetic peak of one pipe of the current device, the
 * denominator of the ALU-bound rooflines (the FP32 layer's contraction, the
 * sweep, the FP64 reference).  The paper has no counterpart; it is a
 * measurement aid.  One launch of blocks_per_sm x (SM count) CTAs of 256
 * threads, each thread running 16 independent chains of `iters` fused
 * multiply-adds on registers only:
 *   WINO_PIPE_FP32    fma.rn.f32     (2 flops per lane and instruction)
 *   WINO_PIPE_FP32X2  fma.rn.f32x2   (4 flops per lane and instruction)
 *   WINO_PIPE_FP64    fma.rn.f64     (2 flops per lane and instruction)
 * *tflops = flops / the launch's CUDA-event duration, *ms = that duration
 * (host outputs).  Synchronises cuda_stream.  WINO_EINVAL for another kind,
 * iters < 1, blocks_per_sm outside 1..8 or a NULL output.                 */
enum { WINO_PIPE_FP32 = 0, WINO_PIPE_FP32X2 = 1, WINO_PIPE_FP64 = 2 };
int wino_pipe_peak(int kind, int iters, int blocks_per_sm, double* tflops, double* ms,
                   void* cuda_stream);

/* Device-side failure detection.  Layer kernels that wait on hardware
 * completion (the tensor-core contraction's mbarrier, the FP32 layer's bulk
 * copies) bound every wait; a wait that gives up sets a per-device flag and
 * the kernel abandons its tile (its output is then incomplete) instead of
 * hanging.  Because layer calls return before their kernels run, the flag
 * is reported here: *flag = 1 when any wait gave up on the current device
 * since the last call, else 0; the flag is cleared.  Synchronises the
 * device.                                                                  */
int wino_wait_error(int* flag);

/* The give-up path of those waits, run on purpose for tests: one warp waits
 * on an mbarrier that nothing arrives at with the layer kernels' bounded
 * wait, limited to `polls` polls (>= 1), gives up, sets the flag read by
 * wino_wait_error and returns; *elapsed_ns = device time of the polls
 * (%globaltimer).  Synchronises cuda_stream (NULL: the default stream).
 * WINO_EINVAL for elapsed_ns NULL or polls < 1.  The layer kernels poll at
 * most WINO_WAIT_POLLS times per wait: about a second on a GB300, where a
 * poll of an incomplete phase suspends ~3.75 us.                          */
#define WINO_WAIT_POLLS (1 << 18)
int wino_wait_probe(int polls, long long* elapsed_ns, void* cuda_stream);

const char* wino_last_error(void);  /* thread-local message, never NULL  */
int wino_device_ok(void);           /* 1 when an sm_103 device is usable  */
void wino_shutdown(void);           /* frees internal scratch and graphs  */

#ifdef __cplusplus
}
#endif

#endif /* WINO_H */
