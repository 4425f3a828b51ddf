// Internal declarations shared by the C ABI (capi.cu), the set-up kernel and
// the kernel instantiation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tables.h"

namespace dg {

struct OpParams;
struct TckParams;
struct EnergyParams;

struct SetupParams {
  int E, n, q;
  double alpha;
  const double* nodes;  // [E][(q+1)^3][3]
  const double* rho;    // [E][n^3]
  const double* c;      // [E][n^3]
  const int32_t* nbr;
  const int8_t* nbr_face;
  const int8_t* orient;
  const double* pts;  // [3][DG_PTS_LEN]: Gauss points, weights, GL points
  const double* xq;   // GL points of the geometry degree (q + 1 of them)
  void* geoA;
  void* geoM;
  void* geoF;
  void* geoT;
  void* geoK;   // compact affine operator data, or nullptr
  void* geoKT;  // compact affine predictor data, or nullptr
  int tstride;
  int tstep;  // predictor geometry at Gauss sets m = n, n - tstep, ... (1 or 2)
  int prec;  // 0 double, 1 float
  int* bad;  // set to 1 if det J <= 0 anywhere
};

cudaError_t launch_setup(const SetupParams& P, cudaStream_t st);

// 2D (quadrilateral) set-up: as SetupParams with 4 faces and n^2 points.
struct Setup2Params {
  int E, n, q;
  double alpha;
  const double* nodes;  // [E][(q+1)^2][2]
  const double* rho;    // [E][n^2]
  const double* c;      // [E][n^2]
  const int32_t* nbr;   // [E][4]
  const int8_t* nbr_face;
  const int8_t* orient;  // [E][4]: 1 = the neighbour's face coordinate runs opposite
  const double* pts;
  const double* xq;
  void* geoA;
  void* geoM;
  void* geoF;
  void* geoT;
  int tstride;
  int tstep;
  int prec;
  int* bad;
};
cudaError_t launch_setup2d(const Setup2Params& P, cudaStream_t st);

typedef cudaError_t (*OpFn)(const OpParams& p, int epi, int epb, cudaStream_t st);
typedef cudaError_t (*TckFn)(const TckParams& p, int red, int epb, cudaStream_t st);
typedef cudaError_t (*EnergyFn)(const EnergyParams& p, int epb, cudaStream_t st);
typedef cudaError_t (*BasisFn)(const void* src, void* dst, int E, int to_g, int epb, cudaStream_t st);
typedef int (*SmemFn)(int which, int red);  // bytes per element
typedef int (*MaxThrFn)(int which);          // largest launchable block
typedef int (*MaxThr0Fn)();

struct KernelTable {
  OpFn op[2][DG_NMAX + 1];
  OpFn opg[2][DG_NMAX + 1];   // operator on Gauss-basis states
  OpFn opga[2][DG_NMAX + 1];  // same, affine elements with constant coefficients
  BasisFn basis[2][DG_NMAX + 1];
  TckFn tck[2][DG_NMAX + 1];      // reduction every 0 or 2 derivatives
  TckFn tck_odd[2][DG_NMAX + 1];  // reduction every 1 or 3 derivatives
  MaxThr0Fn tck_odd_maxthr[2][DG_NMAX + 1];
  TckFn tckc[2][DG_NMAX + 1];     // column form, Gauss-basis states, every reduction
  int (*tckc_smem[2][DG_NMAX + 1])(int red);  // bytes per element
  MaxThr0Fn tckc_maxthr[2][DG_NMAX + 1];
  TckFn tcki[2][DG_NMAX + 1];     // column form, interleaved: affine Gauss-point states, reduction 0 or 2
  TckFn tckn[2][DG_NMAX + 1];     // without the basis change (Alg. 1), GL states, no reduction
  int (*tckn_smem[2][DG_NMAX + 1])(int red);
  MaxThr0Fn tckn_maxthr[2][DG_NMAX + 1];
  // two-register LSRK stages; which: 0 GL, 1 Gauss-point states, 2 affine
  cudaError_t (*op2r[2][DG_NMAX + 1])(const OpParams& p, int which, int epb, cudaStream_t st);
  MaxThr0Fn op2r_maxthr[2][DG_NMAX + 1];
  EnergyFn energy[2][DG_NMAX + 1];
  SmemFn smem[2][DG_NMAX + 1];
  MaxThrFn maxthr[2][DG_NMAX + 1];
};

struct Op2Params;
struct Tck2Params;
struct Energy2Params;
struct KernelTable2D {
  cudaError_t (*op[2][DG_NMAX + 1])(const Op2Params& p, int epi, int epb, cudaStream_t st);
  cudaError_t (*tck[2][DG_NMAX + 1])(const Tck2Params& p, int red, int epb, cudaStream_t st);
  cudaError_t (*basis[2][DG_NMAX + 1])(void* U, int E, int to_g, int epb, cudaStream_t st);
  cudaError_t (*energy[2][DG_NMAX + 1])(const Energy2Params& p, int epb, cudaStream_t st);
  int (*smem[2][DG_NMAX + 1])(int which);
  int (*maxthr[2][DG_NMAX + 1])(int which);
};
void register_2d(KernelTable2D* t);
int upload_2d(const double* d, const float* f);

// Each kernel translation unit registers its instantiations and uploads the
// constant tables into its own copy (returns 0 or a cudaError_t value).
void register_f64_lo(KernelTable* t);
void register_f64_hi(KernelTable* t);
void register_f32_lo(KernelTable* t);
void register_f32_hi(KernelTable* t);
int upload_f64_lo(const double* d, const float* f);
int upload_f64_hi(const double* d, const float* f);
int upload_f32_lo(const double* d, const float* f);
int upload_f32_hi(const double* d, const float* f);
void register_tck_odd_f64(KernelTable* t);
void register_tck_odd_f32(KernelTable* t);
int upload_tck_odd_f64(const double* d, const float* f);
int upload_tck_odd_f32(const double* d, const float* f);
void register_tckc_f64_lo(KernelTable* t);
void register_tckc_f64_hi(KernelTable* t);
void register_tckc_f32_lo(KernelTable* t);
void register_tckc_f32_hi(KernelTable* t);
int upload_tckc_f64_lo(const double* d, const float* f);
int upload_tckc_f64_hi(const double* d, const float* f);
int upload_tckc_f32_lo(const double* d, const float* f);
int upload_tckc_f32_hi(const double* d, const float* f);
void register_tckn(KernelTable* t);
int upload_tckn(const double* d, const float* f);
void register_tcki_f32(KernelTable* t);
int upload_tcki_f32(const double* d, const float* f);
void register_lsrk2r_f64(KernelTable* t);
void register_lsrk2r_f32(KernelTable* t);
int upload_lsrk2r_f64(const double* d, const float* f);
int upload_lsrk2r_f32(const double* d, const float* f);

struct BatchItem;
struct BatchInst;
// Batched persistent kernels, one launch per degree n (all items of degree n).
cudaError_t launch_batch_op_f64(int n, const BatchItem* items, int nitems, const BatchInst* inst, int phase,
                                int* counter, int grid, int block, size_t smem, cudaStream_t st, int mode);
cudaError_t launch_batch_op_f32(int n, const BatchItem* items, int nitems, const BatchInst* inst, int phase,
                                int* counter, int grid, int block, size_t smem, cudaStream_t st, int mode);
cudaError_t launch_batch_basis_f64(int n, const BatchItem* items, int nitems, const BatchInst* inst, int to_g,
                                   int* counter, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_batch_basis_f32(int n, const BatchItem* items, int nitems, const BatchInst* inst, int to_g,
                                   int* counter, int grid, int block, size_t smem, cudaStream_t st);
// mode (FP32 only; FP64 always takes the line form): 0 line form, 1 column
// form, 2 column form on affine elements with constant coefficients.  The
// column form takes a list of slices (one block each; grid and counter
// unused) instead of persistent work items.
cudaError_t launch_batch_tck_f64(int n, const BatchItem* items, int nitems, const BatchInst* inst, int red,
                                 int* counter, int grid, int block, size_t smem, cudaStream_t st, int mode);
cudaError_t launch_batch_tck_f32(int n, const BatchItem* items, int nitems, const BatchInst* inst, int red,
                                 int* counter, int grid, int block, size_t smem, cudaStream_t st, int mode);
// which: 0 operator, 1 / 2 predictor (reduction 2 / 0)
int batch_occupancy_f64(int n, int which, int block, size_t smem);
int batch_occupancy_f32(int n, int which, int block, size_t smem);
int batch_max_threads_f64(int n, int which);  // which: 0 operator, 1 predictor
int batch_max_threads_f32(int n, int which);
int upload_batch_f64(const double* d, const float* f);
int upload_batch_f32(const double* d, const float* f);

}  // namespace dg
