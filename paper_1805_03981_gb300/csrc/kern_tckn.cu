// Predictor without the basis change (Alg. 1, tckn.cuh), double and float,
// n = 2..8.
#include "tckn.cuh"

namespace dg {
void register_tckn(KernelTable* t) {
  register_tckn_one<2, double>(t);
  register_tckn_one<3, double>(t);
  register_tckn_one<4, double>(t);
  register_tckn_one<5, double>(t);
  register_tckn_one<6, double>(t);
  register_tckn_one<7, double>(t);
  register_tckn_one<8, double>(t);
  register_tckn_one<2, float>(t);
  register_tckn_one<3, float>(t);
  register_tckn_one<4, float>(t);
  register_tckn_one<5, float>(t);
  register_tckn_one<6, float>(t);
  register_tckn_one<7, float>(t);
  register_tckn_one<8, float>(t);
}
int upload_tckn(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<2, double>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<3, double>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<4, double>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<5, double>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<6, double>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<7, double>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<8, double>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<2, float>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<3, float>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<4, float>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<5, float>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<6, float>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<7, float>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(tckn_kernel<8, float>)) != cudaSuccess) return (int)e;
  return 0;
}
}  // namespace dg
