// Column-form predictor kernels (tckc.cuh), double, n = 6..8, reduction
// every 0, 1, 2 or 3 derivatives, curved and affine elements.
#include "tckc.cuh"

namespace dg {
void register_tckc_f64_hi(KernelTable* t) {
  register_tckc_one<6, double>(t);
  register_tckc_one<7, double>(t);
  register_tckc_one<8, double>(t);
}
int upload_tckc_f64_hi(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = tckc_allow_smem<6, double>()) != cudaSuccess) return (int)e;
  if ((e = tckc_allow_smem<7, double>()) != cudaSuccess) return (int)e;
  if ((e = tckc_allow_smem<8, double>()) != cudaSuccess) return (int)e;
  return 0;
}
}  // namespace dg
