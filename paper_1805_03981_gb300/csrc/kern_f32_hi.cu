// Kernel instantiations: float, degrees k = 5..7 (n = 6..8).
#include "kern_inst.cuh"

namespace dg {
void register_f32_hi(KernelTable* t) {
  register_one<6, float>(t);
  register_one<7, float>(t);
  register_one<8, float>(t);
}
int upload_f32_hi(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<6, float>()) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<7, float>()) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<8, float>()) != cudaSuccess) return (int)e;
  return 0;
}
}  // namespace dg
