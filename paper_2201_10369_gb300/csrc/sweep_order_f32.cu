// sweep_order_f32.cu -- the Huffman-order sweep kernels in FP32 (Sec. 5),
// and the order dispatch.
#include "sweep_order.cuh"

namespace wino {

EvalFn order_sweep_kernel_f64(int dim, int m, int r);        // sweep_order_f64.cu
PointsetFn order_pointset_kernel_f64(int dim, int m, int r);  // sweep_order_f64.cu

EvalFn order_sweep_kernel(int order, int dim, int m, int r) {
  if (order == 1) return order_sweep_kernel_t<float>(dim, m, r);
  if (order == 2) return order_sweep_kernel_f64(dim, m, r);
  return nullptr;
}

PointsetFn order_pointset_kernel(int order, int dim, int m, int r) {
  if (order == 1) return order_pointset_kernel_t<float>(dim, m, r);
  if (order == 2) return order_pointset_kernel_f64(dim, m, r);
  return nullptr;
}

size_t order_smem_bytes(int order, int m, int r) {
  if (order == 1) return order_smem_bytes_t<float>(m, r);
  if (order == 2) return order_smem_bytes_t<double>(m, r);
  return 0;
}

}  // namespace wino
