// Predictor of ADER without the basis change (Sec. 3.2, Alg. 1): the Taylor
// terms stay in the Gauss-Lobatto storage basis, and every derivative is an
// L2 projection in that basis,
//   evaluate grad T_{j-1} at the Gauss points (GL -> G interpolation and the
//   collocation derivative there, metric and coefficients as in Alg. 2),
//   multiply by the weights w_q det J_q and integrate against the GL shape
//   functions (transposed interpolation), and
//   apply the inverse GL mass matrix in sum-factorised form,
//   M_GL^-1 = V^-1 diag(1 / (w det J)) V^-T (Sec. 3.1).
// No degree reduction (the unoptimised variant of Sec. 4.1).  In exact
// arithmetic the result equals the collocated predictor's (Alg. 2): the
// n-point Gauss rule makes M_GL = V^T diag(w det J) V with V invertible, so
// projecting values known at the Gauss points returns their interpolant.
// The kernel exists to measure what the basis change saves.
//
// A block holds epb elements with n^2 threads each; a thread owns one line
// of its element per contraction pass (as in tck_block); the derivative
// spreads the lines of all the block's elements over all threads.
#pragma once

#include "kern_inst.cuh"

namespace dg {

template <int N>
__host__ __device__ constexpr int tckn_smem_per_elem() {
  return 13 * N * N * N;  // T, work, accumulator (4 fields each), w det J
}

// Every line along DIR of the element's 4-field tile, in place: out = M in
// (TR: out = M^T in), M the n x n table matrix at OFF.
template <int N, typename Real, int DIR, int OFF, bool TR>
__device__ __forceinline__ void tckn_pass(Real* s, int t) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const int a = t % N, b = t / N;
  const int base = DIR == 0 ? N * a + N2 * b : (DIR == 1 ? a + N2 * b : a + N * b);
  constexpr int st = DIR == 0 ? 1 : (DIR == 1 ? N : N2);
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    Real in[N], out[N];
#pragma unroll
    for (int q = 0; q < N; ++q) in[q] = s[f * N3 + base + st * q];
    if (TR)
      mtv<Real, OFF, N, N>(in, out);
    else
      mv<Real, OFF, N, N>(in, out);
#pragma unroll
    for (int q = 0; q < N; ++q) s[f * N3 + base + st * q] = out[q];
  }
}

// The three directions of one tensor-product operator (a sync after each).
template <int N, typename Real, int OFF, bool TR>
__device__ __forceinline__ void tckn_tensor(Real* s, int t, bool own) {
  if (own) tckn_pass<N, Real, 0, OFF, TR>(s, t);
  __syncthreads();
  if (own) tckn_pass<N, Real, 1, OFF, TR>(s, t);
  __syncthreads();
  if (own) tckn_pass<N, Real, 2, OFF, TR>(s, t);
  __syncthreads();
}

template <int N, typename Real>
__device__ __forceinline__ void tckn_block(const TckParams& p, const int e0, const int ne, const int epb,
                                           Real* sm) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int SE = tckn_smem_per_elem<N>();
  const int T = threadIdx.x, NT = blockDim.x;
  const int le0 = T / N2;
  const bool own = le0 < ne;
  const int le = own ? le0 : 0;
  const int t = T - le0 * N2;
  // per element: [0, 4n^3) current term (GL coefficients), [4n^3, 8n^3) work
  // tile, [8n^3, 12n^3) Taylor sum (GL coefficients), [12n^3, 13n^3) w det J
  Real* sT = sm + le * SE;
  Real* sW = sT + 4 * N3;
  const Real* __restrict__ U = static_cast<const Real*>(p.U);
  const Real* geo0 = static_cast<const Real*>(p.geoT) + (size_t)e0 * p.geoT_stride;
  const Real* geoK0 = p.aff ? static_cast<const Real*>(p.geoKT) + (size_t)e0 * DG_AFF_TCK : nullptr;
  const Real c0 = (Real)p.coef[0];
  for (int i = T; i < ne * 4 * N3; i += NT) {
    const int l = i / (4 * N3), r = i - l * 4 * N3;
    const Real v = U[(size_t)e0 * 4 * N3 + i];
    sm[l * SE + r] = v;
    sm[l * SE + 8 * N3 + r] = c0 * v;
  }
  // w_q det J_q from the inverse Jacobian at the n-point set (line-major per
  // direction: J^-1_{d i} of point (x, y, z) at (3 d + i) n^3 + line + n^2 pos)
  for (int i = T; i < ne * N3; i += NT) {
    const int l = i / N3, q = i - l * N3;
    const int x = q % N, y = (q / N) % N, z = q / N2;
    Real j[3][3];
    if (p.aff) {
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int c = 0; c < 3; ++c) j[d][c] = geoK0[l * DG_AFF_TCK + 3 * d + c];
    } else {
      const Real* g = geo0 + l * p.geoT_stride;
      const int pos[3] = {(y + N * z) + N2 * x, (x + N * z) + N2 * y, (x + N * y) + N2 * z};
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int c = 0; c < 3; ++c) j[d][c] = g[(3 * d + c) * N3 + pos[d]];
    }
    const Real dinv = j[0][0] * (j[1][1] * j[2][2] - j[1][2] * j[2][1]) -
                      j[0][1] * (j[1][0] * j[2][2] - j[1][2] * j[2][0]) +
                      j[0][2] * (j[1][0] * j[2][1] - j[1][1] * j[2][0]);
    const Real w = tab<Real>(OFF_W(N) + x) * tab<Real>(OFF_W(N) + y) * tab<Real>(OFF_W(N) + z);
    sm[l * SE + 12 * N3 + q] = w / dinv;
  }
  __syncthreads();
#pragma unroll 1
  for (int jj = 1; jj <= N; ++jj) {
    // gradient at the Gauss points: interpolate GL -> G into the work tile ...
    for (int i = T; i < ne * 4 * N3; i += NT) {
      const int l = i / (4 * N3), r = i - l * 4 * N3;
      sm[l * SE + 4 * N3 + r] = sm[l * SE + r];
    }
    __syncthreads();
    tckn_tensor<N, Real, OFF_V(N), false>(sW, t, own);
    // ... differentiate there with the metric and coefficients (into T) ...
    if (p.aff)
      tck_derivative_aff<N, Real, N3>(sm + 4 * N3, sm, SE, geoK0, ne, T, NT);
    else
      tck_derivative<N, Real, N3>(sm + 4 * N3, sm, SE, geo0, p.geoT_stride, ne, T, NT);
    // ... weight by w det J and integrate against the GL functions (V^T) ...
    for (int i = T; i < ne * 4 * N3; i += NT) {
      const int l = i / (4 * N3), r = i - l * 4 * N3;
      sm[l * SE + r] *= sm[l * SE + 12 * N3 + r % N3];
    }
    __syncthreads();
    tckn_tensor<N, Real, OFF_V(N), true>(sT, t, own);
    // ... and apply M_GL^-1 = V^-1 diag(1 / (w det J)) V^-T
    tckn_tensor<N, Real, OFF_VI(N), true>(sT, t, own);
    for (int i = T; i < ne * 4 * N3; i += NT) {
      const int l = i / (4 * N3), r = i - l * 4 * N3;
      sm[l * SE + r] /= sm[l * SE + 12 * N3 + r % N3];
    }
    __syncthreads();
    tckn_tensor<N, Real, OFF_VI(N), false>(sT, t, own);
    const Real cj = (Real)p.coef[jj];
    for (int i = T; i < ne * 4 * N3; i += NT) {
      const int l = i / (4 * N3), r = i - l * 4 * N3;
      sm[l * SE + 8 * N3 + r] = fma(cj, sm[l * SE + r], sm[l * SE + 8 * N3 + r]);
    }
    __syncthreads();
  }
  Real* __restrict__ out = static_cast<Real*>(p.Ubar);
  for (int i = T; i < ne * 4 * N3; i += NT) {
    const int l = i / (4 * N3);
    out[(size_t)e0 * 4 * N3 + i] = sm[l * SE + 8 * N3 + (i - l * 4 * N3)];
  }
}

template <int N, typename Real>
__global__ void tckn_kernel(const TckParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int epb = blockDim.x / (N * N);
  const int e0 = blockIdx.x * epb;
  tckn_block<N, Real>(p, e0, min(epb, p.E - e0), epb, reinterpret_cast<Real*>(smem_raw));
}

template <int N, typename Real>
cudaError_t launch_tckn(const TckParams& p, int red, int epb, cudaStream_t st) {
  if (red != 0 || p.gmode || p.W) return cudaErrorInvalidValue;
  const int threads = epb * N * N;
  const int blocks = (p.E + epb - 1) / epb;
  const size_t smem = (size_t)epb * tckn_smem_per_elem<N>() * sizeof(Real);
  tckn_kernel<N, Real><<<blocks, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int N, typename Real>
int tckn_smem(int) {
  return tckn_smem_per_elem<N>() * (int)sizeof(Real);
}

template <int N, typename Real>
int tckn_max_threads() {
  return kernel_max_threads(tckn_kernel<N, Real>);
}

template <int N, typename Real>
void register_tckn_one(KernelTable* t) {
  const int pi = sizeof(Real) == 8 ? 0 : 1;
  t->tckn[pi][N] = &launch_tckn<N, Real>;
  t->tckn_smem[pi][N] = &tckn_smem<N, Real>;
  t->tckn_maxthr[pi][N] = &tckn_max_threads<N, Real>;
}

}  // namespace dg
