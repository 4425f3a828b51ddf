// Interleaved column-form predictor kernels (tcki.cuh), float, n = 2..8,
// reduction every 0 or 2 derivatives, affine elements with constant
// coefficients.
#include "tcki.cuh"

namespace dg {
void register_tcki_f32(KernelTable* t) {
  register_tcki_one<2, float>(t);
  register_tcki_one<3, float>(t);
  register_tcki_one<4, float>(t);
  register_tcki_one<5, float>(t);
  register_tcki_one<6, float>(t);
  register_tcki_one<7, float>(t);
  register_tcki_one<8, float>(t);
}
int upload_tcki_f32(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = tcki_allow_smem<2, float>()) != cudaSuccess) return (int)e;
  if ((e = tcki_allow_smem<3, float>()) != cudaSuccess) return (int)e;
  if ((e = tcki_allow_smem<4, float>()) != cudaSuccess) return (int)e;
  if ((e = tcki_allow_smem<5, float>()) != cudaSuccess) return (int)e;
  if ((e = tcki_allow_smem<6, float>()) != cudaSuccess) return (int)e;
  if ((e = tcki_allow_smem<7, float>()) != cudaSuccess) return (int)e;
  if ((e = tcki_allow_smem<8, float>()) != cudaSuccess) return (int)e;
  return 0;
}
}  // namespace dg
