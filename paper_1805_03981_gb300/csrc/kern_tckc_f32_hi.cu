// Column-form predictor kernels (tckc.cuh), float, n = 6..8, reduction
// every 0, 1, 2 or 3 derivatives, curved and affine elements.
#include "tckc.cuh"

namespace dg {
void register_tckc_f32_hi(KernelTable* t) {
  register_tckc_one<6, float>(t);
  register_tckc_one<7, float>(t);
  register_tckc_one<8, float>(t);
}
int upload_tckc_f32_hi(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = tckc_allow_smem<6, float>()) != cudaSuccess) return (int)e;
  if ((e = tckc_allow_smem<7, float>()) != cudaSuccess) return (int)e;
  if ((e = tckc_allow_smem<8, float>()) != cudaSuccess) return (int)e;
  return 0;
}
}  // namespace dg
