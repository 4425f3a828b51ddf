// Operator kernels with the two-register LSRK stage epilogue (Sec. 2.2,
// LSRK4(5) and LSRK5(9)), double, n = 2..8: GL storage, Gauss-point states and
// the affine compact form.
#include "kern_inst.cuh"

namespace dg {
void register_lsrk2r_f64(KernelTable* t) {
  register_2r_one<2, double>(t);
  register_2r_one<3, double>(t);
  register_2r_one<4, double>(t);
  register_2r_one<5, double>(t);
  register_2r_one<6, double>(t);
  register_2r_one<7, double>(t);
  register_2r_one<8, double>(t);
}
int upload_lsrk2r_f64(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = op2r_allow_smem<2, double>()) != cudaSuccess) return (int)e;
  if ((e = op2r_allow_smem<3, double>()) != cudaSuccess) return (int)e;
  if ((e = op2r_allow_smem<4, double>()) != cudaSuccess) return (int)e;
  if ((e = op2r_allow_smem<5, double>()) != cudaSuccess) return (int)e;
  if ((e = op2r_allow_smem<6, double>()) != cudaSuccess) return (int)e;
  if ((e = op2r_allow_smem<7, double>()) != cudaSuccess) return (int)e;
  if ((e = op2r_allow_smem<8, double>()) != cudaSuccess) return (int)e;
  return 0;
}
}  // namespace dg
