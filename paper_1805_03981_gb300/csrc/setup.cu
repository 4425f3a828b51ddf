// Geometry and coefficient set-up in FP64 (one block per element).
//
// The paper pre-computes inverse Jacobians at each quadrature point and
// re-uses them (Sec. 3.3, Sec. 4.4); this kernel evaluates, from the degree-q
// geometry nodes and the degree-k nodal coefficients, everything the
// operator and the predictor read per point, and writes it in the precision
// of the context and in the layouts of dg_kernels.cuh:
//   geoA [3 d][3 i][n^3] line-major per d   w adj(J)_{d i} = w detJ (J^-1)_{d i}
//   geoM [2][n^3]                            rho c^2/(w detJ), 1/(rho w detJ)
//   geoF [6 f][6][n^2]                       nw = w_f adj(J)_{d .} (+-1),
//   (per-element strides geo_stride_A/M/F of tables.h: padded to 8 values)
//                                            Z-/(Z-+Z+), alpha Z- Z+/((Z-+Z+)|nw|),
//                                            alpha |nw|/(Z-+Z+)
//   geoT per Gauss set m = n, n-s, ... >= 2 (s = P.tstep, 1 or 2):
//                                        [3 d][3 i][m^3] J^-1_{d i} line-major,
//                                        [m^3] -rho c^2, [m^3] -1/rho
// with J_{i j} = d x_i / d xi_j, Nanson's formula for the face normal and
// Z = rho c (Sec. 2.4).
#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_internal.h"
#include "tables.h"

namespace dg {
namespace {

constexpr int CMAX = DG_NMAX + 2;

// inv[a c + b] = 1 / (nodes[a] - nodes[b]) (a != b), computed once per block
// into shared memory by fill_inv, so that no point evaluation divides.
__device__ void fill_inv(const double* nodes, int c, double* inv) {
  for (int i = threadIdx.x; i < c * c; i += blockDim.x) {
    const int a = i / c, b = i - a * c;
    inv[i] = a == b ? 0.0 : 1.0 / (nodes[a] - nodes[b]);
  }
}

// Lagrange polynomials of the c nodes (and their derivatives) at x.
__device__ void lag1d(const double* nodes, const double* inv, int c, double x, double* L, double* dL) {
  for (int a = 0; a < c; ++a) {
    double v = 1.0, d = 0.0;
    for (int b = 0; b < c; ++b) {
      if (b == a) continue;
      const double iv = inv[a * c + b];
      d = d * (x - nodes[b]) * iv + v * iv;
      v *= (x - nodes[b]) * iv;
    }
    L[a] = v;
    if (dL) dL[a] = d;
  }
}

// the node inverse-difference tables of the geometry (q+1 points) and of the
// solution (n points) nodes, in shared memory
struct InvTabs {
  double q[(DG_NMAX + 2) * (DG_NMAX + 2)];
  double gl[(DG_NMAX + 2) * (DG_NMAX + 2)];
};

__device__ void jacobian(const SetupParams& P, const InvTabs& T, int e, const double xi[3], double J[3][3]) {
  const int c = P.q + 1;
  double L[3][CMAX], dL[3][CMAX];
  for (int d = 0; d < 3; ++d) lag1d(P.xq, T.q, c, xi[d], L[d], dL[d]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) J[i][j] = 0.0;
  const double* X = P.nodes + (size_t)e * c * c * c * 3;
  for (int kk = 0; kk < c; ++kk)
    for (int jj = 0; jj < c; ++jj)
      for (int ii = 0; ii < c; ++ii) {
        const int idx = ii + c * jj + c * c * kk;
        const double w0 = dL[0][ii] * L[1][jj] * L[2][kk];
        const double w1 = L[0][ii] * dL[1][jj] * L[2][kk];
        const double w2 = L[0][ii] * L[1][jj] * dL[2][kk];
        for (int i = 0; i < 3; ++i) {
          const double x = X[idx * 3 + i];
          J[i][0] += x * w0;
          J[i][1] += x * w1;
          J[i][2] += x * w2;
        }
      }
}

// adj(J) = det(J) J^-1; returns det(J)
__device__ double adjugate(const double J[3][3], double A[3][3]) {
  A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
}

__device__ double nodal_at(const double* f, const double* xgl, const double* inv, int n, const double xi[3]) {
  double L[3][CMAX];
  for (int d = 0; d < 3; ++d) lag1d(xgl, inv, n, xi[d], L[d], nullptr);
  double s = 0.0;
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y) {
      double row = 0.0;
      for (int x = 0; x < n; ++x) row += f[x + n * y + n * n * z] * L[0][x];
      s += row * L[1][y] * L[2][z];
    }
  return s;
}

__device__ __forceinline__ void put(void* base, size_t i, double v, int prec) {
  if (prec == 0)
    static_cast<double*>(base)[i] = v;
  else
    static_cast<float*>(base)[i] = (float)v;
}

// position of point (x, y, z) of an m^3 tile in the line-major order of dir
__device__ __forceinline__ int line_major(int dir, int m, int x, int y, int z) {
  return dir == 0 ? (y + m * z) + m * m * x : (dir == 1 ? (x + m * z) + m * m * y : (x + m * y) + m * m * z);
}

__global__ void setup_kernel(const SetupParams P) {
  const int e = blockIdx.x;
  const int n = P.n, n2 = n * n, n3 = n2 * n;
  const double* xg = P.pts + dg_pts_off(n);
  const double* wg = P.pts + DG_PTS_LEN + dg_pts_off(n);
  const double* xgl = P.pts + 2 * DG_PTS_LEN + dg_pts_off(n);
  __shared__ InvTabs T;
  fill_inv(P.xq, P.q + 1, T.q);
  fill_inv(xgl, n, T.gl);
  __syncthreads();
  const double* rho = P.rho + (size_t)e * n3;
  const double* cc = P.c + (size_t)e * n3;
  const int ncell = n3, nface = 6 * n2;
  int ntck = 0;
  const int ts = P.tstep > 1 ? 2 : 1;
  for (int m = n; m >= 2; m -= ts) ntck += m * m * m;
  const int nitems = ncell + nface + ntck;
  for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
    double J[3][3], A[3][3], xi[3];
    if (it < ncell) {
      const int x = it % n, y = (it / n) % n, z = it / n2;
      xi[0] = xg[x];
      xi[1] = xg[y];
      xi[2] = xg[z];
      const double w = wg[x] * wg[y] * wg[z];
      jacobian(P, T, e, xi, J);
      const double det = adjugate(J, A);
      if (!(det > 0.0)) atomicExch(P.bad, 1);
      const double r = nodal_at(rho, xgl, T.gl, n, xi), c = nodal_at(cc, xgl, T.gl, n, xi);
      for (int d = 0; d < 3; ++d)
        for (int i = 0; i < 3; ++i)
          put(P.geoA, (size_t)e * geo_stride_A(n) + (d * 3 + i) * n3 + line_major(d, n, x, y, z), w * A[d][i],
              P.prec);
      put(P.geoM, (size_t)e * geo_stride_M(n) + it, r * c * c / (w * det), P.prec);
      put(P.geoM, (size_t)e * geo_stride_M(n) + n3 + it, 1.0 / (r * w * det), P.prec);
    } else if (it < ncell + nface) {
      const int k = it - ncell;
      const int f = k / n2, ij = k - f * n2, i = ij % n, j = ij / n;
      const int d = f >> 1;
      const double side = (f & 1) ? 1.0 : -1.0;
      const int t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
      xi[d] = side;
      xi[t0] = xg[i];
      xi[t1] = xg[j];
      jacobian(P, T, e, xi, J);
      const double det = adjugate(J, A);
      if (!(det > 0.0)) atomicExch(P.bad, 1);
      const double wf = wg[i] * wg[j];
      const double nw[3] = {wf * side * A[d][0], wf * side * A[d][1], wf * side * A[d][2]};
      const double s = sqrt(nw[0] * nw[0] + nw[1] * nw[1] + nw[2] * nw[2]);
      const double zm = nodal_at(rho, xgl, T.gl, n, xi) * nodal_at(cc, xgl, T.gl, n, xi);
      double zp = zm;
      const int en = P.nbr[e * 6 + f];
      if (en >= 0) {
        const int fn = P.nbr_face[e * 6 + f], o = P.orient[e * 6 + f];
        const int uu = (o & 1) ? j : i, vv = (o & 1) ? i : j;
        const int ip = (o & 2) ? n - 1 - uu : uu, jp = (o & 4) ? n - 1 - vv : vv;
        const int dn = fn >> 1;
        double xn[3];
        xn[dn] = (fn & 1) ? 1.0 : -1.0;
        xn[dn == 0 ? 1 : 0] = xg[ip];
        xn[dn == 2 ? 1 : 2] = xg[jp];
        zp = nodal_at(P.rho + (size_t)en * n3, xgl, T.gl, n, xn) * nodal_at(P.c + (size_t)en * n3, xgl, T.gl, n, xn);
      }
      const double zs = zm + zp;
      const size_t fb = (size_t)e * geo_stride_F(n) + (size_t)f * 6 * n2 + ij;
      put(P.geoF, fb, nw[0], P.prec);
      put(P.geoF, fb + n2, nw[1], P.prec);
      put(P.geoF, fb + 2 * n2, nw[2], P.prec);
      put(P.geoF, fb + 3 * n2, zm / zs, P.prec);
      put(P.geoF, fb + 4 * n2, P.alpha * zm * zp / (zs * s), P.prec);
      put(P.geoF, fb + 5 * n2, P.alpha * s / zs, P.prec);
    } else {
      int k = it - ncell - nface, m = n, off = 0;
      while (k >= m * m * m) {
        k -= m * m * m;
        off += 11 * m * m * m;
        m -= ts;
      }
      const int m2 = m * m, m3 = m2 * m;
      const int x = k % m, y = (k / m) % m, z = k / m2;
      const double* xm = P.pts + dg_pts_off(m);
      xi[0] = xm[x];
      xi[1] = xm[y];
      xi[2] = xm[z];
      jacobian(P, T, e, xi, J);
      const double det = adjugate(J, A);
      if (!(det > 0.0)) atomicExch(P.bad, 1);
      const double r = nodal_at(rho, xgl, T.gl, n, xi), c = nodal_at(cc, xgl, T.gl, n, xi);
      const size_t tb = (size_t)e * P.tstride + off;
      for (int d = 0; d < 3; ++d)
        for (int i = 0; i < 3; ++i)
          put(P.geoT, tb + (d * 3 + i) * m3 + line_major(d, m, x, y, z), A[d][i] / det, P.prec);
      put(P.geoT, tb + 9 * m3 + k, -r * c * c, P.prec);
      put(P.geoT, tb + 10 * m3 + k, -1.0 / r, P.prec);
    }
  }
}

// Compact data of an affine element with constant coefficients (one thread
// per element), in the context precision:
//   geoK  [48]: adj(J)_{d i} (9), rho c^2 / detJ, 1 / (rho detJ),
//               per face: nw0 = +-adj(J)_{d .} (3), Z-/(Z-+Z+),
//               alpha Z- Z+ / ((Z-+Z+) |nw0|), alpha |nw0| / (Z-+Z+)
//   geoKT [16]: J^-1_{d i} (9), -rho c^2, -1/rho
// At a point with Gauss weight w (face: w_f) the per-point values of the
// general layout are w adj(J), m / w, w_f nw0, b0 / w_f and c0 w_f.
__global__ void setup_affine_kernel(const SetupParams P) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n, n3 = n * n * n;
  const double* xgl = P.pts + 2 * DG_PTS_LEN + dg_pts_off(n);
  __shared__ InvTabs T;
  fill_inv(P.xq, P.q + 1, T.q);
  fill_inv(xgl, n, T.gl);
  __syncthreads();
  if (e >= P.E) return;
  const double ctr[3] = {0.0, 0.0, 0.0};
  double J[3][3], A[3][3];
  jacobian(P, T, e, ctr, J);
  const double det = adjugate(J, A);
  if (!(det > 0.0)) atomicExch(P.bad, 1);
  const double r = nodal_at(P.rho + (size_t)e * n3, xgl, T.gl, n, ctr);
  const double c = nodal_at(P.c + (size_t)e * n3, xgl, T.gl, n, ctr);
  const size_t kb = (size_t)e * DG_AFF_OP, tb = (size_t)e * DG_AFF_TCK;
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < 3; ++i) {
      put(P.geoK, kb + d * 3 + i, A[d][i], P.prec);
      put(P.geoKT, tb + d * 3 + i, A[d][i] / det, P.prec);
    }
  put(P.geoK, kb + 9, r * c * c / det, P.prec);
  put(P.geoK, kb + 10, 1.0 / (r * det), P.prec);
  put(P.geoKT, tb + 9, -r * c * c, P.prec);
  put(P.geoKT, tb + 10, -1.0 / r, P.prec);
  const double zm = r * c;
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1;
    const double side = (f & 1) ? 1.0 : -1.0;
    const double nw[3] = {side * A[d][0], side * A[d][1], side * A[d][2]};
    const double s = sqrt(nw[0] * nw[0] + nw[1] * nw[1] + nw[2] * nw[2]);
    double zp = zm;
    const int en = P.nbr[e * 6 + f];
    if (en >= 0)
      zp = nodal_at(P.rho + (size_t)en * n3, xgl, T.gl, n, ctr) * nodal_at(P.c + (size_t)en * n3, xgl, T.gl, n, ctr);
    const double zs = zm + zp;
    const size_t fb = kb + 11 + f * 6;
    put(P.geoK, fb, nw[0], P.prec);
    put(P.geoK, fb + 1, nw[1], P.prec);
    put(P.geoK, fb + 2, nw[2], P.prec);
    put(P.geoK, fb + 3, zm / zs, P.prec);
    put(P.geoK, fb + 4, P.alpha * zm * zp / (zs * s), P.prec);
    put(P.geoK, fb + 5, P.alpha * s / zs, P.prec);
  }
  put(P.geoK, kb + 47, 0.0, P.prec);
  for (int i = 11; i < DG_AFF_TCK; ++i) put(P.geoKT, tb + i, 0.0, P.prec);
}

}  // namespace

cudaError_t launch_setup(const SetupParams& P, cudaStream_t st) {
  setup_kernel<<<P.E, 128, 0, st>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && P.geoK) {
    setup_affine_kernel<<<(P.E + 127) / 128, 128, 0, st>>>(P);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace dg
