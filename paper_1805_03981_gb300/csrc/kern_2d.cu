// The 2D path: geometry set-up and kernel instantiations (double and float,
// n = 2..8) of dg2d.cuh, with their launchers.
#include <cmath>

#include "dg2d.cuh"
#include "dg_internal.h"
#include "kern_inst.cuh"

namespace dg {
namespace {

constexpr int C2MAX = DG_NMAX + 2;

__device__ void lag1d2(const double* nodes, int c, double x, double* L, double* dL) {
  for (int a = 0; a < c; ++a) {
    double v = 1.0, d = 0.0;
    for (int b = 0; b < c; ++b) {
      if (b == a) continue;
      const double inv = 1.0 / (nodes[a] - nodes[b]);
      d = d * (x - nodes[b]) * inv + v * inv;
      v *= (x - nodes[b]) * inv;
    }
    L[a] = v;
    if (dL) dL[a] = d;
  }
}

// J[i][j] = d x_i / d xi_j of element e at reference point xi
__device__ void jacobian2(const Setup2Params& P, int e, const double xi[2], double J[2][2]) {
  const int c = P.q + 1;
  double L[2][C2MAX], dL[2][C2MAX];
  for (int d = 0; d < 2; ++d) lag1d2(P.xq, c, xi[d], L[d], dL[d]);
  J[0][0] = J[0][1] = J[1][0] = J[1][1] = 0.0;
  const double* X = P.nodes + (size_t)e * c * c * 2;
  for (int jj = 0; jj < c; ++jj)
    for (int ii = 0; ii < c; ++ii) {
      const int idx = ii + c * jj;
      const double w0 = dL[0][ii] * L[1][jj], w1 = L[0][ii] * dL[1][jj];
      for (int i = 0; i < 2; ++i) {
        J[i][0] += X[idx * 2 + i] * w0;
        J[i][1] += X[idx * 2 + i] * w1;
      }
    }
}

// adj(J) = det(J) J^-1; returns det(J)
__device__ double adjugate2(const double J[2][2], double A[2][2]) {
  A[0][0] = J[1][1];
  A[0][1] = -J[0][1];
  A[1][0] = -J[1][0];
  A[1][1] = J[0][0];
  return J[0][0] * J[1][1] - J[0][1] * J[1][0];
}

__device__ double nodal_at2(const double* f, const double* xgl, int n, const double xi[2]) {
  double L0[C2MAX], L1[C2MAX];
  lag1d2(xgl, n, xi[0], L0, nullptr);
  lag1d2(xgl, n, xi[1], L1, nullptr);
  double s = 0.0;
  for (int y = 0; y < n; ++y) {
    double row = 0.0;
    for (int x = 0; x < n; ++x) row += f[x + n * y] * L0[x];
    s += row * L1[y];
  }
  return s;
}

__device__ __forceinline__ void put2(void* base, size_t i, double v, int prec) {
  if (prec == 0)
    static_cast<double*>(base)[i] = v;
  else
    static_cast<float*>(base)[i] = (float)v;
}

// Per element (one block): w adj(J) line-major, the inverse-mass diagonals,
// the face normals and flux weights (Sec. 2.4; Nanson's formula in 2D), and
// the predictor's J^-1 and coefficients at every stored Gauss set.
__global__ void setup2d_kernel(const Setup2Params P) {
  const int e = blockIdx.x;
  const int n = P.n, n2 = n * n;
  const double* xg = P.pts + dg_pts_off(n);
  const double* wg = P.pts + DG_PTS_LEN + dg_pts_off(n);
  const double* xgl = P.pts + 2 * DG_PTS_LEN + dg_pts_off(n);
  const double* rho = P.rho + (size_t)e * n2;
  const double* cc = P.c + (size_t)e * n2;
  const int ts = P.tstep > 1 ? 2 : 1;
  int ntck = 0;
  for (int m = n; m >= 2; m -= ts) ntck += m * m;
  const int ncell = n2, nface = 4 * n, nitems = ncell + nface + ntck;
  for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
    double J[2][2], A[2][2], xi[2];
    if (it < ncell) {
      const int x = it % n, y = it / n;
      xi[0] = xg[x];
      xi[1] = xg[y];
      const double w = wg[x] * wg[y];
      jacobian2(P, e, xi, J);
      const double det = adjugate2(J, A);
      if (!(det > 0.0)) atomicExch(P.bad, 1);
      const double r = nodal_at2(rho, xgl, n, xi), c = nodal_at2(cc, xgl, n, xi);
      const size_t ga = (size_t)e * geo2_stride_A(n);
      for (int d = 0; d < 2; ++d) {
        const int lm = d == 0 ? y + n * x : x + n * y;  // line-major: (line, position)
        for (int i = 0; i < 2; ++i) put2(P.geoA, ga + (d * 2 + i) * n2 + lm, w * A[d][i], P.prec);
      }
      put2(P.geoM, (size_t)e * geo2_stride_M(n) + it, r * c * c / (w * det), P.prec);
      put2(P.geoM, (size_t)e * geo2_stride_M(n) + n2 + it, 1.0 / (r * w * det), P.prec);
    } else if (it < ncell + nface) {
      const int k = it - ncell, f = k / n, j = k - f * n;
      const int d = f >> 1;
      const double side = (f & 1) ? 1.0 : -1.0;
      xi[d] = side;
      xi[1 - d] = xg[j];
      jacobian2(P, e, xi, J);
      const double det = adjugate2(J, A);
      if (!(det > 0.0)) atomicExch(P.bad, 1);
      const double nw[2] = {wg[j] * side * A[d][0], wg[j] * side * A[d][1]};
      const double s = sqrt(nw[0] * nw[0] + nw[1] * nw[1]);
      const double zm = nodal_at2(rho, xgl, n, xi) * nodal_at2(cc, xgl, n, xi);
      double zp = zm;
      const int en = P.nbr[e * 4 + f];
      if (en >= 0) {
        const int fn = P.nbr_face[e * 4 + f];
        const int jp = P.orient[e * 4 + f] ? n - 1 - j : j;
        double xn[2];
        xn[fn >> 1] = (fn & 1) ? 1.0 : -1.0;
        xn[1 - (fn >> 1)] = xg[jp];
        zp = nodal_at2(P.rho + (size_t)en * n2, xgl, n, xn) * nodal_at2(P.c + (size_t)en * n2, xgl, n, xn);
      }
      const double zs = zm + zp;
      const size_t fb = (size_t)e * geo2_stride_F(n) + (size_t)f * 5 * n + j;
      put2(P.geoF, fb, nw[0], P.prec);
      put2(P.geoF, fb + n, nw[1], P.prec);
      put2(P.geoF, fb + 2 * n, zm / zs, P.prec);
      put2(P.geoF, fb + 3 * n, P.alpha * zm * zp / (zs * s), P.prec);
      put2(P.geoF, fb + 4 * n, P.alpha * s / zs, P.prec);
    } else {
      int k = it - ncell - nface, m = n, off = 0;
      while (k >= m * m) {
        k -= m * m;
        off += 6 * m * m;
        m -= ts;
      }
      const int m2 = m * m, x = k % m, y = k / m;
      const double* xm = P.pts + dg_pts_off(m);
      xi[0] = xm[x];
      xi[1] = xm[y];
      jacobian2(P, e, xi, J);
      const double det = adjugate2(J, A);
      if (!(det > 0.0)) atomicExch(P.bad, 1);
      const double r = nodal_at2(rho, xgl, n, xi), c = nodal_at2(cc, xgl, n, xi);
      const size_t tb = (size_t)e * P.tstride + off;
      for (int d = 0; d < 2; ++d) {
        const int lm = d == 0 ? y + m * x : x + m * y;
        for (int i = 0; i < 2; ++i) put2(P.geoT, tb + (d * 2 + i) * m2 + lm, A[d][i] / det, P.prec);
      }
      put2(P.geoT, tb + 4 * m2 + k, -r * c * c, P.prec);
      put2(P.geoT, tb + 5 * m2 + k, -1.0 / r, P.prec);
    }
  }
}

template <int N, typename Real>
cudaError_t launch_op2(const Op2Params& p, int epi, int epb, cudaStream_t st) {
  const int threads = epb * N, blocks = (p.E + epb - 1) / epb;
  const size_t smem = (size_t)epb * 6 * N * N * sizeof(Real);
  if (epi == EPI_WRITE)
    opg2d_kernel<N, Real, EPI_WRITE><<<blocks, threads, smem, st>>>(p);
  else if (epi == EPI_LSRK)
    opg2d_kernel<N, Real, EPI_LSRK><<<blocks, threads, smem, st>>>(p);
  else
    opg2d_kernel<N, Real, EPI_ADD><<<blocks, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int N, typename Real>
cudaError_t launch_tck2(const Tck2Params& p, int red, int epb, cudaStream_t st) {
  const int threads = epb * N, blocks = (p.E + epb - 1) / epb;
  if (red == 2) {
    tck2d_kernel<N, Real, 2><<<blocks, threads, (size_t)epb * tck2_smem_per_elem<N, 2>() * sizeof(Real), st>>>(p);
  } else if (red == 0) {
    tck2d_kernel<N, Real, 0><<<blocks, threads, (size_t)epb * tck2_smem_per_elem<N, 0>() * sizeof(Real), st>>>(p);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int N, typename Real>
cudaError_t launch_basis2(void* U, int E, int to_g, int epb, cudaStream_t st) {
  basis2d_kernel<N, Real><<<(E + epb - 1) / epb, epb * N, (size_t)epb * 3 * N * N * sizeof(Real), st>>>(U, E, to_g);
  return cudaGetLastError();
}

template <int N, typename Real>
cudaError_t launch_energy2(const Energy2Params& p, int epb, cudaStream_t st) {
  energy2d_kernel<N, Real><<<(p.E + epb - 1) / epb, epb * N, (size_t)epb * 3 * N * N * sizeof(Real), st>>>(p);
  return cudaGetLastError();
}

// shared memory per element (bytes): 0 operator, 1 predictor (reduction 2), 2 basis / energy
template <int N, typename Real>
int smem2_bytes(int which) {
  if (which == 0) return 6 * N * N * (int)sizeof(Real);
  if (which == 1) return tck2_smem_per_elem<N, 2>() * (int)sizeof(Real);
  return 3 * N * N * (int)sizeof(Real);
}

template <int N, typename Real>
int maxthr2(int which) {
  if (which == 0)
    return min(kernel_max_threads(opg2d_kernel<N, Real, EPI_WRITE>),
               min(kernel_max_threads(opg2d_kernel<N, Real, EPI_LSRK>), kernel_max_threads(opg2d_kernel<N, Real, EPI_ADD>)));
  if (which == 1) return min(kernel_max_threads(tck2d_kernel<N, Real, 0>), kernel_max_threads(tck2d_kernel<N, Real, 2>));
  return min(kernel_max_threads(basis2d_kernel<N, Real>), kernel_max_threads(energy2d_kernel<N, Real>));
}

template <int N, typename Real>
cudaError_t allow2() {
  cudaError_t e;
  if ((e = allow_smem(opg2d_kernel<N, Real, EPI_WRITE>)) != cudaSuccess) return e;
  if ((e = allow_smem(opg2d_kernel<N, Real, EPI_LSRK>)) != cudaSuccess) return e;
  if ((e = allow_smem(opg2d_kernel<N, Real, EPI_ADD>)) != cudaSuccess) return e;
  if ((e = allow_smem(tck2d_kernel<N, Real, 0>)) != cudaSuccess) return e;
  if ((e = allow_smem(tck2d_kernel<N, Real, 2>)) != cudaSuccess) return e;
  if ((e = allow_smem(basis2d_kernel<N, Real>)) != cudaSuccess) return e;
  return allow_smem(energy2d_kernel<N, Real>);
}

template <int N, typename Real>
void reg2(KernelTable2D* t) {
  const int pi = sizeof(Real) == 8 ? 0 : 1;
  t->op[pi][N] = &launch_op2<N, Real>;
  t->tck[pi][N] = &launch_tck2<N, Real>;
  t->basis[pi][N] = &launch_basis2<N, Real>;
  t->energy[pi][N] = &launch_energy2<N, Real>;
  t->smem[pi][N] = &smem2_bytes<N, Real>;
  t->maxthr[pi][N] = &maxthr2<N, Real>;
}

}  // namespace

cudaError_t launch_setup2d(const Setup2Params& P, cudaStream_t st) {
  setup2d_kernel<<<P.E, 128, 0, st>>>(P);
  return cudaGetLastError();
}

void register_2d(KernelTable2D* t) {
  reg2<2, double>(t);
  reg2<3, double>(t);
  reg2<4, double>(t);
  reg2<5, double>(t);
  reg2<6, double>(t);
  reg2<7, double>(t);
  reg2<8, double>(t);
  reg2<2, float>(t);
  reg2<3, float>(t);
  reg2<4, float>(t);
  reg2<5, float>(t);
  reg2<6, float>(t);
  reg2<7, float>(t);
  reg2<8, float>(t);
}

int upload_2d(const double* d, const float* f) {
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_tab_d, d, sizeof(double) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpyToSymbol(c_tab_f, f, sizeof(float) * DG_TAB_LEN)) != cudaSuccess) return (int)e;
  cudaError_t r[] = {allow2<2, double>(), allow2<3, double>(), allow2<4, double>(), allow2<5, double>(),
                     allow2<6, double>(), allow2<7, double>(), allow2<8, double>(), allow2<2, float>(),
                     allow2<3, float>(),  allow2<4, float>(),  allow2<5, float>(),  allow2<6, float>(),
                     allow2<7, float>(),  allow2<8, float>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) return (int)x;
  return 0;
}

}  // namespace dg
