// Predictor kernels with reduction every 1 or 3 derivatives, float, n = 2..8
// (the variants of Sec. 3.3 that Fig. reduc-comp compares).
#include "kern_inst.cuh"

namespace dg {
void register_tck_odd_f32(KernelTable* t) {
  register_tck_odd_one<2, float>(t);
  register_tck_odd_one<3, float>(t);
  register_tck_odd_one<4, float>(t);
  register_tck_odd_one<5, float>(t);
  register_tck_odd_one<6, float>(t);
  register_tck_odd_one<7, float>(t);
  register_tck_odd_one<8, float>(t);
}
int upload_tck_odd_f32(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = tck_odd_allow_smem<2, float>()) != cudaSuccess) return (int)e;
  if ((e = tck_odd_allow_smem<3, float>()) != cudaSuccess) return (int)e;
  if ((e = tck_odd_allow_smem<4, float>()) != cudaSuccess) return (int)e;
  if ((e = tck_odd_allow_smem<5, float>()) != cudaSuccess) return (int)e;
  if ((e = tck_odd_allow_smem<6, float>()) != cudaSuccess) return (int)e;
  if ((e = tck_odd_allow_smem<7, float>()) != cudaSuccess) return (int)e;
  if ((e = tck_odd_allow_smem<8, float>()) != cudaSuccess) return (int)e;
  return 0;
}
}  // namespace dg
