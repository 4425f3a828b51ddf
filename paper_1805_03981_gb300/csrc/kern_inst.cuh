// Explicit instantiation helpers for one precision and a range of degrees.
// Included by kern_f64_lo.cu, kern_f64_hi.cu, kern_f32_lo.cu, kern_f32_hi.cu.
#pragma once

#include "dg_internal.h"
#include "dg_kernels.cuh"

namespace dg {

template <int N, typename Real>
cudaError_t launch_op(const OpParams& p, int epi, int epb, cudaStream_t st) {
  const int threads = epb * N * N;
  const size_t smem = (size_t)epb * op_smem_per_elem<N>() * sizeof(Real);
  const int blocks = (p.E + epb - 1) / epb;
  if (epi == EPI_WRITE)
    op_kernel<N, Real, EPI_WRITE><<<blocks, threads, smem, st>>>(p);
  else if (epi == EPI_LSRK)
    op_kernel<N, Real, EPI_LSRK><<<blocks, threads, smem, st>>>(p);
  else
    op_kernel<N, Real, EPI_ADD><<<blocks, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int N, typename Real>
constexpr int opg_smem_per_elem() {
  return sizeof(Real) == 4 ? opgs_smem_per_elem<N>() : op_smem_per_elem<N>();
}

template <int N, typename Real>
cudaError_t launch_opg(const OpParams& p, int epi, int epb, cudaStream_t st) {
  const int threads = epb * N * N;
  const size_t smem = (size_t)epb * opg_smem_per_elem<N, Real>() * sizeof(Real);
  const int blocks = (p.E + epb - 1) / epb;
  if (epi == EPI_WRITE)
    opg_kernel<N, Real, EPI_WRITE><<<blocks, threads, smem, st>>>(p);
  else if (epi == EPI_LSRK)
    opg_kernel<N, Real, EPI_LSRK><<<blocks, threads, smem, st>>>(p);
  else
    opg_kernel<N, Real, EPI_ADD><<<blocks, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int N, typename Real>
cudaError_t launch_opga(const OpParams& p, int epi, int epb, cudaStream_t st) {
  const int threads = epb * N * N;
  const size_t smem = (size_t)epb * opga_smem_per_elem<N>(sizeof(Real) == 4) * sizeof(Real);
  const int blocks = (p.E + epb - 1) / epb;
  if (epi == EPI_WRITE)
    opga_kernel<N, Real, EPI_WRITE><<<blocks, threads, smem, st>>>(p);
  else if (epi == EPI_LSRK)
    opga_kernel<N, Real, EPI_LSRK><<<blocks, threads, smem, st>>>(p);
  else
    opga_kernel<N, Real, EPI_ADD><<<blocks, threads, smem, st>>>(p);
  return cudaGetLastError();
}

// Stages of the two-register LSRK schemes (EPI_LSRK2R), in their own units
// (kern_lsrk2r_*.cu).  which: 0 GL storage (op_kernel), 1 Gauss-point states
// (opg_kernel), 2 Gauss-point states on affine elements (opga_kernel).
template <int N, typename Real>
cudaError_t launch_op2r(const OpParams& p, int which, int epb, cudaStream_t st) {
  const int threads = epb * N * N;
  const int blocks = (p.E + epb - 1) / epb;
  if (which == 0) {
    op_kernel<N, Real, EPI_LSRK2R>
        <<<blocks, threads, (size_t)epb * op_smem_per_elem<N>() * sizeof(Real), st>>>(p);
  } else if (which == 1) {
    opg_kernel<N, Real, EPI_LSRK2R>
        <<<blocks, threads, (size_t)epb * opg_smem_per_elem<N, Real>() * sizeof(Real), st>>>(p);
  } else {
    opga_kernel<N, Real, EPI_LSRK2R>
        <<<blocks, threads, (size_t)epb * opga_smem_per_elem<N>(sizeof(Real) == 4) * sizeof(Real), st>>>(p);
  }
  return cudaGetLastError();
}

template <int N, typename Real>
cudaError_t launch_basis(const void* src, void* dst, int E, int to_g, int epb, cudaStream_t st) {
  const int threads = epb * N * N;
  const size_t smem = (size_t)epb * 4 * N * N * N * sizeof(Real);
  basis_kernel<N, Real><<<(E + epb - 1) / epb, threads, smem, st>>>(src, dst, E, to_g);
  return cudaGetLastError();
}

template <int N, typename Real, int RED>
cudaError_t launch_tck_red(const TckParams& p, int epb, cudaStream_t st) {
  const int threads = epb * N * N;
  const int blocks = (p.E + epb - 1) / epb;
  const size_t smem = (size_t)epb * tck_smem_per_elem<N, RED>() * sizeof(Real);
  tck_kernel<N, Real, RED><<<blocks, threads, smem, st>>>(p);
  return cudaGetLastError();
}

// Reduction every 0 or 2 derivatives; 1 and 3 live in their own units
// (kern_tck_odd_*.cu, launch_tck_odd).
template <int N, typename Real>
cudaError_t launch_tck(const TckParams& p, int red, int epb, cudaStream_t st) {
  if (red == 2) return launch_tck_red<N, Real, 2>(p, epb, st);
  if (red == 0) return launch_tck_red<N, Real, 0>(p, epb, st);
  return cudaErrorInvalidValue;
}

template <int N, typename Real>
cudaError_t launch_tck_odd(const TckParams& p, int red, int epb, cudaStream_t st) {
  if (red == 1) return launch_tck_red<N, Real, 1>(p, epb, st);
  if (red == 3) return launch_tck_red<N, Real, 3>(p, epb, st);
  return cudaErrorInvalidValue;
}

template <int N, typename Real>
cudaError_t launch_energy(const EnergyParams& p, int epb, cudaStream_t st) {
  const int threads = epb * N * N;
  const int blocks = (p.E + epb - 1) / epb;
  const size_t smem = (size_t)epb * 4 * N * N * N * sizeof(Real);
  energy_kernel<N, Real><<<blocks, threads, smem, st>>>(p);
  return cudaGetLastError();
}

// which: 0 operator, 1 predictor, 2 energy
template <int N, typename Real>
int smem_bytes(int which, int red) {
  if (which == 0)
    return max(max(op_smem_per_elem<N>(), opg_smem_per_elem<N, Real>()),
               opga_smem_per_elem<N>(sizeof(Real) == 4)) *
           (int)sizeof(Real);
  if (which == 1) {
    const int per = red == 1 ? tck_smem_per_elem<N, 1>()
                  : red == 2 ? tck_smem_per_elem<N, 2>()
                  : red == 3 ? tck_smem_per_elem<N, 3>()
                             : tck_smem_per_elem<N, 0>();
    return per * (int)sizeof(Real);
  }
  return 4 * N * N * N * (int)sizeof(Real);
}

// Allow each kernel the opt-in shared memory limit minus its static use.
template <typename K>
cudaError_t allow_smem(K kernel) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

template <int N, typename Real>
cudaError_t set_max_smem() {
  cudaError_t e;
  if ((e = allow_smem(op_kernel<N, Real, EPI_WRITE>)) != cudaSuccess) return e;
  if ((e = allow_smem(op_kernel<N, Real, EPI_LSRK>)) != cudaSuccess) return e;
  if ((e = allow_smem(op_kernel<N, Real, EPI_ADD>)) != cudaSuccess) return e;
  if ((e = allow_smem(opg_kernel<N, Real, EPI_WRITE>)) != cudaSuccess) return e;
  if ((e = allow_smem(opg_kernel<N, Real, EPI_LSRK>)) != cudaSuccess) return e;
  if ((e = allow_smem(opg_kernel<N, Real, EPI_ADD>)) != cudaSuccess) return e;
  if ((e = allow_smem(basis_kernel<N, Real>)) != cudaSuccess) return e;
  if ((e = allow_smem(opga_kernel<N, Real, EPI_WRITE>)) != cudaSuccess) return e;
  if ((e = allow_smem(opga_kernel<N, Real, EPI_LSRK>)) != cudaSuccess) return e;
  if ((e = allow_smem(opga_kernel<N, Real, EPI_ADD>)) != cudaSuccess) return e;
  if ((e = allow_smem(tck_kernel<N, Real, 0>)) != cudaSuccess) return e;
  if ((e = allow_smem(tck_kernel<N, Real, 2>)) != cudaSuccess) return e;
  return allow_smem(energy_kernel<N, Real>);
}

// Largest block the kernel can launch with (registers per thread included).
template <typename K>
int kernel_max_threads(K kernel) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return fa.maxThreadsPerBlock;
}

// which: 0 operator (all epilogues), 1 predictor (both reductions), 2 energy
template <int N, typename Real>
int max_threads(int which) {
  if (which == 0)
    return min(min(kernel_max_threads(op_kernel<N, Real, EPI_WRITE>),
                   min(kernel_max_threads(op_kernel<N, Real, EPI_LSRK>),
                       kernel_max_threads(op_kernel<N, Real, EPI_ADD>))),
               min(min(kernel_max_threads(opg_kernel<N, Real, EPI_WRITE>),
                       min(kernel_max_threads(opg_kernel<N, Real, EPI_LSRK>),
                           kernel_max_threads(opg_kernel<N, Real, EPI_ADD>))),
                   min(kernel_max_threads(opga_kernel<N, Real, EPI_LSRK>),
                       kernel_max_threads(opga_kernel<N, Real, EPI_ADD>))));
  if (which == 1)
    return min(kernel_max_threads(tck_kernel<N, Real, 0>), kernel_max_threads(tck_kernel<N, Real, 2>));
  return min(kernel_max_threads(energy_kernel<N, Real>), kernel_max_threads(basis_kernel<N, Real>));
}

// Largest block of the predictor with reduction every 1 or 3 derivatives.
template <int N, typename Real>
int tck_odd_max_threads() {
  return min(kernel_max_threads(tck_kernel<N, Real, 1>), kernel_max_threads(tck_kernel<N, Real, 3>));
}

template <int N, typename Real>
cudaError_t tck_odd_allow_smem() {
  cudaError_t e;
  if ((e = allow_smem(tck_kernel<N, Real, 1>)) != cudaSuccess) return e;
  return allow_smem(tck_kernel<N, Real, 3>);
}

template <int N, typename Real>
void register_tck_odd_one(KernelTable* t) {
  const int pi = sizeof(Real) == 8 ? 0 : 1;
  t->tck_odd[pi][N] = &launch_tck_odd<N, Real>;
  t->tck_odd_maxthr[pi][N] = &tck_odd_max_threads<N, Real>;
}

template <int N, typename Real>
cudaError_t op2r_allow_smem() {
  cudaError_t e;
  if ((e = allow_smem(op_kernel<N, Real, EPI_LSRK2R>)) != cudaSuccess) return e;
  if ((e = allow_smem(opg_kernel<N, Real, EPI_LSRK2R>)) != cudaSuccess) return e;
  return allow_smem(opga_kernel<N, Real, EPI_LSRK2R>);
}

template <int N, typename Real>
int op2r_max_threads() {
  return min(kernel_max_threads(op_kernel<N, Real, EPI_LSRK2R>),
             min(kernel_max_threads(opg_kernel<N, Real, EPI_LSRK2R>),
                 kernel_max_threads(opga_kernel<N, Real, EPI_LSRK2R>)));
}

template <int N, typename Real>
void register_2r_one(KernelTable* t) {
  const int pi = sizeof(Real) == 8 ? 0 : 1;
  t->op2r[pi][N] = &launch_op2r<N, Real>;
  t->op2r_maxthr[pi][N] = &op2r_max_threads<N, Real>;
}

template <int N, typename Real>
void register_one(KernelTable* t) {
  const int pi = sizeof(Real) == 8 ? 0 : 1;
  t->op[pi][N] = &launch_op<N, Real>;
  t->opg[pi][N] = &launch_opg<N, Real>;
  t->opga[pi][N] = &launch_opga<N, Real>;
  t->basis[pi][N] = &launch_basis<N, Real>;
  t->tck[pi][N] = &launch_tck<N, Real>;
  t->energy[pi][N] = &launch_energy<N, Real>;
  t->smem[pi][N] = &smem_bytes<N, Real>;
  t->maxthr[pi][N] = &max_threads<N, Real>;
}

}  // namespace dg
