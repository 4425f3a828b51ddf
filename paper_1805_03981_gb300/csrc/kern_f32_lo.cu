// Kernel instantiations: float, degrees k = 1..4 (n = 2..5).
#include "kern_inst.cuh"

namespace dg {
void register_f32_lo(KernelTable* t) {
  register_one<2, float>(t);
  register_one<3, float>(t);
  register_one<4, float>(t);
  register_one<5, float>(t);
}
int upload_f32_lo(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<2, float>()) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<3, float>()) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<4, float>()) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<5, float>()) != cudaSuccess) return (int)e;
  return 0;
}
}  // namespace dg
