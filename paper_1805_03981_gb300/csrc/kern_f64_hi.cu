// Kernel instantiations: double, degrees k = 5..7 (n = 6..8).
#include "kern_inst.cuh"

namespace dg {
void register_f64_hi(KernelTable* t) {
  register_one<6, double>(t);
  register_one<7, double>(t);
  register_one<8, double>(t);
}
int upload_f64_hi(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<6, double>()) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<7, double>()) != cudaSuccess) return (int)e;
  if ((e = set_max_smem<8, double>()) != cudaSuccess) return (int)e;
  return 0;
}
}  // namespace dg
