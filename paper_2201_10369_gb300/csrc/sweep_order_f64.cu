// sweep_order_f64.cu -- the Huffman-order sweep kernels with FP64
// transforms and the FP32 Hadamard product (Sec. 5, "mixed precision").
#include "sweep_order.cuh"

namespace wino {

int order_sweep_launch_f64(const SweepSize& s, const float* rec, int trials,
                           const double* c_grid, int n_c, const MaskList& masks,
                           const double* ysum, double* err, cudaStream_t st) {
  return order_sweep_launch_t<double, true>(s, rec, trials, c_grid, n_c, masks, ysum, err, st);
}

int order_pointset_launch_f64(int dim, int m, int r, const float* rec, int trials,
                              const double* pts, int n_sets, const double* ysum, double* err,
                              cudaStream_t st) {
  return order_pointset_launch_t<double, true>(dim, m, r, rec, trials, pts, n_sets, ysum, err, st);
}

}  // namespace wino
