// Batched persistent kernels (all degrees in one launch), double.
#include "kern_inst.cuh"

namespace dg {
cudaError_t launch_batch_op_f64(const BatchItem* items, int nitems, const BatchInst* inst, int phase,
                                    int* counter, int grid, int block, size_t smem, cudaStream_t st) {
  batch_op_kernel<double><<<grid, block, smem, st>>>(items, nitems, inst, phase, counter);
  return cudaGetLastError();
}
cudaError_t launch_batch_tck_f64(const BatchItem* items, int nitems, const BatchInst* inst, int red,
                                     int* counter, int grid, int block, size_t smem, cudaStream_t st) {
  if (red == 2)
    batch_tck_kernel<double, 2><<<grid, block, smem, st>>>(items, nitems, inst, counter);
  else
    batch_tck_kernel<double, 0><<<grid, block, smem, st>>>(items, nitems, inst, counter);
  return cudaGetLastError();
}
// blocks per SM of the batched kernels (which: 0 operator, 1 predictor red=2, 2 predictor red=0)
int batch_occupancy_f64(int which, int block, size_t smem) {
  int nb = 0;
  if (which == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_op_kernel<double>, block, smem);
  else if (which == 1)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_tck_kernel<double, 2>, block, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_tck_kernel<double, 0>, block, smem);
  cudaGetLastError();
  return nb;
}
int upload_batch_f64(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(batch_op_kernel<double>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(batch_tck_kernel<double, 2>)) != cudaSuccess) return (int)e;
  if ((e = allow_smem(batch_tck_kernel<double, 0>)) != cudaSuccess) return (int)e;
  return 0;
}
}  // namespace dg
