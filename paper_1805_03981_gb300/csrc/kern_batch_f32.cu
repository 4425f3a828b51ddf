// Batched persistent kernels (one launch per degree), float.  The predictor
// of Gauss-point states takes the column form (tckc.cuh).
#include "tckc.cuh"

namespace dg {
namespace {

template <int N, int MODE>
cudaError_t op_nm(const BatchItem* items, int nitems, const BatchInst* inst, int phase, int* counter,
                  int grid, int block, size_t smem, cudaStream_t st) {
  if (phase < 5)
    batch_op_kernel<N, float, EPI_LSRK, MODE><<<grid, block, smem, st>>>(items, nitems, inst, phase, counter);
  else
    batch_op_kernel<N, float, EPI_ADD, MODE><<<grid, block, smem, st>>>(items, nitems, inst, phase, counter);
  return cudaGetLastError();
}
template <int N>
cudaError_t op_n(const BatchItem* items, int nitems, const BatchInst* inst, int phase, int* counter,
                 int grid, int block, size_t smem, cudaStream_t st, int mode) {
  if (mode == 1) return op_nm<N, 1>(items, nitems, inst, phase, counter, grid, block, smem, st);
  if (mode == 2) return op_nm<N, 2>(items, nitems, inst, phase, counter, grid, block, smem, st);
  return op_nm<N, 0>(items, nitems, inst, phase, counter, grid, block, smem, st);
}
template <int N>
cudaError_t basis_n(const BatchItem* items, int nitems, const BatchInst* inst, int to_g, int* counter,
                    int grid, int block, size_t smem, cudaStream_t st) {
  batch_basis_kernel<N, float><<<grid, block, smem, st>>>(items, nitems, inst, to_g, counter);
  return cudaGetLastError();
}
// mode: 0 GL states (line form), 1 Gauss-point states (column form), 2 the
// same on affine elements with constant coefficients
template <int N, int RED>
cudaError_t tck_nr(const BatchItem* items, int nitems, const BatchInst* inst, int* counter, int grid,
                   int block, size_t smem, cudaStream_t st, int mode) {
  if (mode == 2)  // items are slices, one block each
    batch_tckc_kernel<N, float, RED, true><<<nitems, block, smem, st>>>(items, inst);
  else if (mode == 1)
    batch_tckc_kernel<N, float, RED, false><<<nitems, block, smem, st>>>(items, inst);
  else
    batch_tck_kernel<N, float, RED><<<grid, block, smem, st>>>(items, nitems, inst, counter);
  return cudaGetLastError();
}
template <int N>
cudaError_t tck_n(const BatchItem* items, int nitems, const BatchInst* inst, int red, int* counter,
                  int grid, int block, size_t smem, cudaStream_t st, int mode) {
  if (red == 2) return tck_nr<N, 2>(items, nitems, inst, counter, grid, block, smem, st, mode);
  return tck_nr<N, 0>(items, nitems, inst, counter, grid, block, smem, st, mode);
}
template <int N>
int occ_n(int which, int block, size_t smem) {
  int nb = 0;
  if (which == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_op_kernel<N, float, EPI_LSRK, 1>, block, smem);
  else if (which == 1)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_tck_kernel<N, float, 2>, block, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_tck_kernel<N, float, 0>, block, smem);
  cudaGetLastError();
  return nb;
}
template <int N>
int maxthr_n(int which) {
  if (which == 0)
    return min(min(min(kernel_max_threads(batch_op_kernel<N, float, EPI_LSRK, 0>),
                       kernel_max_threads(batch_op_kernel<N, float, EPI_ADD, 0>)),
                   min(kernel_max_threads(batch_op_kernel<N, float, EPI_LSRK, 1>),
                       kernel_max_threads(batch_op_kernel<N, float, EPI_ADD, 1>))),
               min(min(kernel_max_threads(batch_op_kernel<N, float, EPI_LSRK, 2>),
                       kernel_max_threads(batch_op_kernel<N, float, EPI_ADD, 2>)),
                   kernel_max_threads(batch_basis_kernel<N, float>)));
  return min(min(kernel_max_threads(batch_tck_kernel<N, float, 2>), kernel_max_threads(batch_tck_kernel<N, float, 0>)),
             min(min(kernel_max_threads(batch_tckc_kernel<N, float, 2, false>),
                     kernel_max_threads(batch_tckc_kernel<N, float, 0, false>)),
                 min(kernel_max_threads(batch_tckc_kernel<N, float, 2, true>),
                     kernel_max_threads(batch_tckc_kernel<N, float, 0, true>))));
}
template <int N>
cudaError_t allow_n() {
  cudaError_t e;
  for (cudaError_t r : {allow_smem(batch_op_kernel<N, float, EPI_LSRK, 0>), allow_smem(batch_op_kernel<N, float, EPI_ADD, 0>),
                        allow_smem(batch_op_kernel<N, float, EPI_LSRK, 1>), allow_smem(batch_op_kernel<N, float, EPI_ADD, 1>),
                        allow_smem(batch_op_kernel<N, float, EPI_LSRK, 2>), allow_smem(batch_op_kernel<N, float, EPI_ADD, 2>)})
    if (r != cudaSuccess) return r;
  if ((e = allow_smem(batch_basis_kernel<N, float>)) != cudaSuccess) return e;
  if ((e = allow_smem(batch_tck_kernel<N, float, 2>)) != cudaSuccess) return e;
  if ((e = allow_smem(batch_tckc_kernel<N, float, 2, false>)) != cudaSuccess) return e;
  if ((e = allow_smem(batch_tckc_kernel<N, float, 0, false>)) != cudaSuccess) return e;
  if ((e = allow_smem(batch_tckc_kernel<N, float, 2, true>)) != cudaSuccess) return e;
  if ((e = allow_smem(batch_tckc_kernel<N, float, 0, true>)) != cudaSuccess) return e;
  return allow_smem(batch_tck_kernel<N, float, 0>);
}

}  // namespace

#define DG_SWITCH_N(n, CALL) \
  switch (n) {              \
    case 2: return CALL(2);  \
    case 3: return CALL(3);  \
    case 4: return CALL(4);  \
    case 5: return CALL(5);  \
    case 6: return CALL(6);  \
    case 7: return CALL(7);  \
    case 8: return CALL(8);  \
    default: break;          \
  }

cudaError_t launch_batch_op_f32(int n, const BatchItem* items, int nitems, const BatchInst* inst, int phase,
                                    int* counter, int grid, int block, size_t smem, cudaStream_t st, int mode) {
#define C_(N) op_n<N>(items, nitems, inst, phase, counter, grid, block, smem, st, mode)
  DG_SWITCH_N(n, C_)
#undef C_
  return cudaErrorInvalidValue;
}
cudaError_t launch_batch_tck_f32(int n, const BatchItem* items, int nitems, const BatchInst* inst, int red,
                                     int* counter, int grid, int block, size_t smem, cudaStream_t st, int mode) {
#define C_(N) tck_n<N>(items, nitems, inst, red, counter, grid, block, smem, st, mode)
  DG_SWITCH_N(n, C_)
#undef C_
  return cudaErrorInvalidValue;
}
cudaError_t launch_batch_basis_f32(int n, const BatchItem* items, int nitems, const BatchInst* inst,
                                       int to_g, int* counter, int grid, int block, size_t smem,
                                       cudaStream_t st) {
#define C_(N) basis_n<N>(items, nitems, inst, to_g, counter, grid, block, smem, st)
  DG_SWITCH_N(n, C_)
#undef C_
  return cudaErrorInvalidValue;
}
// blocks per SM (which: 0 operator, 1 predictor red=2, 2 predictor red=0)
int batch_occupancy_f32(int n, int which, int block, size_t smem) {
#define C_(N) occ_n<N>(which, block, smem)
  DG_SWITCH_N(n, C_)
#undef C_
  return 0;
}
int batch_max_threads_f32(int n, int which) {
#define C_(N) maxthr_n<N>(which)
  DG_SWITCH_N(n, C_)
#undef C_
  return 0;
}
int upload_batch_f32(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  for (int n = 2; n <= DG_NMAX; ++n) {
    cudaError_t r = cudaErrorInvalidValue;
    switch (n) {
      case 2: r = allow_n<2>(); break;
      case 3: r = allow_n<3>(); break;
      case 4: r = allow_n<4>(); break;
      case 5: r = allow_n<5>(); break;
      case 6: r = allow_n<6>(); break;
      case 7: r = allow_n<7>(); break;
      case 8: r = allow_n<8>(); break;
    }
    if (r != cudaSuccess) return (int)r;
  }
  return 0;
}
}  // namespace dg
