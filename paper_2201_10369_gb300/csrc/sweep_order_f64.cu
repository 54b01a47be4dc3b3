// sweep_order_f64.cu -- the Huffman-order sweep kernels with FP64
// transforms and the FP32 Hadamard product (Sec. 5, "mixed precision").
#include "sweep_order.cuh"

namespace wino {

EvalFn order_sweep_kernel_f64(int dim, int m, int r) {
  return order_sweep_kernel_t<double>(dim, m, r);
}

PointsetFn order_pointset_kernel_f64(int dim, int m, int r) {
  return order_pointset_kernel_t<double>(dim, m, r);
}

}  // namespace wino
