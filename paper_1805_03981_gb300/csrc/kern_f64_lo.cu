// Kernel instantiations: double, degrees k = 1..4 (n = 2..5).
#include "kern_inst.cuh"

namespace dg {
void register_f64_lo(KernelTable* t) {
  register_one<2, double>(t);
  register_one<3, double>(t);
  register_one<4, double>(t);
  register_one<5, double>(t);
}
int upload_f64_lo(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<2, double>()) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<3, double>()) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<4, double>()) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<5, double>()) != cudaSuccess) return (int)e;
  return 0;
}
}  // namespace dg
