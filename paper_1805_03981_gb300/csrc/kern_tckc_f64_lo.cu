// Column-form predictor kernels (tckc.cuh), double, n = 2..5, reduction
// every 0, 1, 2 or 3 derivatives, curved and affine elements.
#include "tckc.cuh"

namespace dg {
void register_tckc_f64_lo(KernelTable* t) {
  register_tckc_one<2, double>(t);
  register_tckc_one<3, double>(t);
  register_tckc_one<4, double>(t);
  register_tckc_one<5, double>(t);
}
int upload_tckc_f64_lo(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = tckc_allow_smem<2, double>()) != cudaSuccess) return (int)e;
  if ((e = tckc_allow_smem<3, double>()) != cudaSuccess) return (int)e;
  if ((e = tckc_allow_smem<4, double>()) != cudaSuccess) return (int)e;
  if ((e = tckc_allow_smem<5, double>()) != cudaSuccess) return (int)e;
  return 0;
}
}  // namespace dg
