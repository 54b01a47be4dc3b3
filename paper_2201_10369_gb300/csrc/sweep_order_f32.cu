// sweep_order_f32.cu -- the warp-per-instance sweep kernels in FP32: the
// Huffman order (Sec. 5) and the plain fmaf order of the wide sizes, and the
// order dispatch.
#include "sweep_order.cuh"

namespace wino {

int order_sweep_launch_f64(const SweepSize& s, const float* rec, int trials,
                           const double* c_grid, int n_c, const MaskList& masks,
                           const double* ysum, double* err, cudaStream_t st);  // _f64.cu
int order_pointset_launch_f64(int dim, int m, int r, const float* rec, int trials,
                              const double* pts, int n_sets, const double* ysum, double* err,
                              cudaStream_t st);  // _f64.cu

int order_sweep_launch(int order, const SweepSize& s, const float* rec, int trials,
                       const double* c_grid, int n_c, const MaskList& masks, const double* ysum,
                       double* err, cudaStream_t st) {
  if (order == 0)
    return order_sweep_launch_t<float, false>(s, rec, trials, c_grid, n_c, masks, ysum, err, st);
  if (order == 1)
    return order_sweep_launch_t<float, true>(s, rec, trials, c_grid, n_c, masks, ysum, err, st);
  if (order == 2)
    return order_sweep_launch_f64(s, rec, trials, c_grid, n_c, masks, ysum, err, st);
  return WINO_EINVAL;
}

int order_pointset_launch(int order, int dim, int m, int r, const float* rec, int trials,
                          const double* pts, int n_sets, const double* ysum, double* err,
                          cudaStream_t st) {
  if (order == 0)
    return order_pointset_launch_t<float, false>(dim, m, r, rec, trials, pts, n_sets, ysum, err,
                                                 st);
  if (order == 1)
    return order_pointset_launch_t<float, true>(dim, m, r, rec, trials, pts, n_sets, ysum, err,
                                                st);
  if (order == 2)
    return order_pointset_launch_f64(dim, m, r, rec, trials, pts, n_sets, ysum, err, st);
  return WINO_EINVAL;
}

}  // namespace wino
