// Device kernels of the 2D solver (quadrilaterals; the paper treats d = 2
// and d = 3 alike, Sec. 2): state (p, v_x, v_y), n^2 nodes per element, node
// (x, y) at x + n y.  The state is held at the Gauss points (values in the
// collocated basis G) inside the steppers, as the 3D Gauss-basis kernels do.
//
// Work decomposition: a block owns EPB consecutive elements, n threads each.
// A thread with in-element index t owns
//   direction 0 (x): the row y = t,
//   direction 1 (y): the column x = t,
// and t is also the face-point index of the two faces normal to that
// direction.  Per-point geometry of a direction-d phase is stored line-major:
// point (line t, position s) at t + n s.
#pragma once

#include "dg_kernels.cuh"

namespace dg {

// per-element strides (values) of the 2D geometry, padded to multiples of 8
DG_HD constexpr int geo2_stride_A(int n) { return dg_pad8(4 * n * n); }
DG_HD constexpr int geo2_stride_M(int n) { return dg_pad8(2 * n * n); }
DG_HD constexpr int geo2_stride_F(int n) { return dg_pad8(4 * 5 * n); }
// predictor data per Gauss set m = n, n-s, ... >= 2: [2 d][2 i][m^2] J^-1
// line-major, [m^2] -rho c^2, [m^2] -1/rho
DG_HD constexpr int geo2_stride_T(int n, int s) { return n < 2 ? 0 : 6 * n * n + geo2_stride_T(n - s, s); }

struct Op2Params {
  const void* U;
  void* out;
  const void* Uadd;
  void* dU;
  double cA, cB, dt;
  int first;
  const int32_t* nbr;
  const int8_t* nbr_face;
  const int8_t* orient;
  const void* geoA;  // [E][2 d][2 i][n^2] w adj(J)_{d i}, line-major per d
  const void* geoM;  // [E][2][n^2] rho c^2 / (w detJ), 1 / (rho w detJ)
  const void* geoF;  // [E][4 f][5][n] w_f adj(J)_{d .} (+-1) (2), Z-/(Z-+Z+), alpha Z-Z+/((Z-+Z+)|nw|), alpha |nw|/(Z-+Z+)
  int E;
};

struct Tck2Params {
  const void* U;  // Gauss-basis state
  void* Ubar;     // predictor output (Gauss basis)
  const void* geoT;
  long long geoT_stride;
  double coef[DG_NMAX + 2];  // dt^{j+1} / (j+1)!
  int E;
  int geo_step;
};

struct Energy2Params {
  const void* U;  // GL state
  const void* geoM;
  double* partial;
  int E;
};

// Contract line l of an X x Y tile of NF fields along DIR with the RO x RI
// matrix at OFF.  DIR 0: line l is the row y = l; DIR 1: the column x = l.
template <typename Real, int DIR, int X, int Y, int RO, int OFF, int FS_IN, int FS_OUT, bool ADD = false>
__device__ __forceinline__ void contract_line2(const Real* src, Real* dst, int l) {
  constexpr int RI = DIR == 0 ? X : Y;
  constexpr int OX = DIR == 0 ? RO : X;
  const int bi = DIR == 0 ? X * l : l, bo = DIR == 0 ? OX * l : l;
  constexpr int si = DIR == 0 ? 1 : X, so = DIR == 0 ? 1 : OX;
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    Real in[RI], out[RO];
#pragma unroll
    for (int s = 0; s < RI; ++s) in[s] = src[f * FS_IN + bi + si * s];
    mv<Real, OFF, RO, RI>(in, out);
#pragma unroll
    for (int s = 0; s < RO; ++s) {
      if (ADD)
        dst[f * FS_OUT + bo + so * s] += out[s];
      else
        dst[f * FS_OUT + bo + so * s] = out[s];
    }
  }
}

// all lines of ne tiles (element stride es) spread over the block's threads
template <typename Real, int DIR, int X, int Y, int RO, int OFF, int FS_IN, int FS_OUT, bool ADD = false>
__device__ __forceinline__ void contract_tile2(const Real* src0, Real* dst0, int es, int ne, int T, int nthr) {
  constexpr int L = DIR == 0 ? Y : X;  // lines per tile
  for (int i = T; i < ne * L; i += nthr) {
    const int le = i / L;
    contract_line2<Real, DIR, X, Y, RO, OFF, FS_IN, FS_OUT, ADD>(src0 + le * es, dst0 + le * es, i - le * L);
  }
}

// In-place change of basis of whole states: GL -> G (to_g) or G -> GL.
template <int N, typename Real>
__global__ void basis2d_kernel(void* Uv, int E, int to_g) {
  constexpr int N2 = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int epb = blockDim.x / N;
  const int e0 = blockIdx.x * epb, ne = min(epb, E - e0);
  Real* U = static_cast<Real*>(Uv) + (size_t)e0 * 3 * N2;
  for (int i = threadIdx.x; i < ne * 3 * N2; i += blockDim.x) sm[i] = U[i];
  __syncthreads();
  if (to_g) {
    contract_tile2<Real, 0, N, N, N, OFF_V(N), N2, N2>(sm, sm, 3 * N2, ne, threadIdx.x, blockDim.x);
    __syncthreads();
    contract_tile2<Real, 1, N, N, N, OFF_V(N), N2, N2>(sm, sm, 3 * N2, ne, threadIdx.x, blockDim.x);
  } else {
    contract_tile2<Real, 0, N, N, N, OFF_VI(N), N2, N2>(sm, sm, 3 * N2, ne, threadIdx.x, blockDim.x);
    __syncthreads();
    contract_tile2<Real, 1, N, N, N, OFF_VI(N), N2, N2>(sm, sm, 3 * N2, ne, threadIdx.x, blockDim.x);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ne * 3 * N2; i += blockDim.x) U[i] = sm[i];
}

// The neighbour's trace on face f at face point j (Gauss basis): the
// l(+-1) contraction of the neighbour's line through that point.
template <int N, typename Real>
__device__ __forceinline__ bool nbr_trace2(const Op2Params& p, const Real* __restrict__ U, int e, int f, int j,
                                           Real (&nb)[3]) {
  constexpr int N2 = N * N;
  const int en = p.nbr[e * 4 + f];
  if (en < 0) return false;
  const int fn = p.nbr_face[e * 4 + f];
  const int jp = p.orient[e * 4 + f] ? N - 1 - j : j;
  const int dn = fn >> 1, sdn = fn & 1;
  const Real* src = U + (size_t)en * 3 * N2 + (dn == 0 ? N * jp : jp);
  const int st = dn == 0 ? 1 : N;
  constexpr int LF = OFF_LF(N);
#pragma unroll
  for (int fl = 0; fl < 3; ++fl) {
    Real acc = tab<Real>(LF + sdn * N) * __ldg(src + fl * N2);
#pragma unroll
    for (int s = 1; s < N; ++s) acc = fma(tab<Real>(LF + sdn * N + s), __ldg(src + fl * N2 + s * st), acc);
    nb[fl] = acc;
  }
  return true;
}

// Cell and face contributions of the direction-DIR phase along the thread's
// line (Sec. 2.1 Eq. (2), Sec. 2.4): the transposed collocation derivative of
// the contravariant fluxes, and the lifting of the two faces normal to DIR.
template <int N, typename Real, int DIR, bool ACC>
__device__ __forceinline__ void cell_face_dir2(const Real (&u)[3][N], Real (&r)[3][N], const Real* __restrict__ gA,
                                               const Real* __restrict__ gF, const Op2Params& p,
                                               const Real* __restrict__ U, int e, int t) {
  constexpr int N2 = N * N;
  const Real* A0 = gA + (DIR * 2 + 0) * N2 + t;
  const Real* A1 = gA + (DIR * 2 + 1) * N2 + t;
  Real F[N];
#pragma unroll
  for (int s = 0; s < N; ++s) F[s] = fma(__ldg(A0 + N * s), u[1][s], __ldg(A1 + N * s) * u[2][s]);
  if (ACC)
    mtv_acc<Real, OFF_D(N), N, N>(F, r[0]);
  else
    mtv<Real, OFF_D(N), N, N>(F, r[0]);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const Real* Ai = i == 0 ? A0 : A1;
#pragma unroll
    for (int s = 0; s < N; ++s) F[s] = __ldg(Ai + N * s) * u[0][s];
    if (ACC)
      mtv_acc<Real, OFF_D(N), N, N>(F, r[1 + i]);
    else
      mtv<Real, OFF_D(N), N, N>(F, r[1 + i]);
  }
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const int f = 2 * DIR + sd;
    constexpr int LF = OFF_LF(N);
    Real um[3];
#pragma unroll
    for (int fl = 0; fl < 3; ++fl) {
      Real acc = tab<Real>(LF + sd * N) * u[fl][0];
#pragma unroll
      for (int s = 1; s < N; ++s) acc = fma(tab<Real>(LF + sd * N + s), u[fl][s], acc);
      um[fl] = acc;
    }
    const Real* fc = gF + f * 5 * N + t;
    const Real nw0 = __ldg(fc), nw1 = __ldg(fc + N);
    const Real a2 = __ldg(fc + 2 * N), bb = __ldg(fc + 3 * N), cc = __ldg(fc + 4 * N);
    const Real vnm = fma(nw0, um[1], nw1 * um[2]);
    Real nb[3], pp, vnp;
    if (nbr_trace2<N, Real>(p, U, e, f, t, nb)) {
      pp = nb[0];
      vnp = fma(nw0, nb[1], nw1 * nb[2]);
    } else {  // reflecting wall: mirror state
      pp = um[0];
      vnp = -vnm;
    }
    const Real dp = um[0] - pp, dvn = vnm - vnp;
    const Real pstar = fma(-a2, dp, fma(bb, dvn, um[0]));
    const Real flp = fma(a2, dvn, fma(cc, dp, vnp));
    const Real g0 = nw0 * pstar, g1 = nw1 * pstar;
#pragma unroll
    for (int s = 0; s < N; ++s) {
      const Real l = tab<Real>(LF + sd * N + s);
      r[0][s] = fma(-l, flp, r[0][s]);
      r[1][s] = fma(-l, g0, r[1][s]);
      r[2][s] = fma(-l, g1, r[2][s]);
    }
  }
}

// The 2D operator R = -M^-1 K U on Gauss-basis states, with the LSRK / ADER
// epilogues fused into the second (y) phase.
template <int N, typename Real, int EPI>
__global__ void opg2d_kernel(const Op2Params p) {
  constexpr int N2 = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int epb = blockDim.x / N;
  const int e0 = blockIdx.x * epb, ne = min(epb, p.E - e0);
  const int le = threadIdx.x / N, t = threadIdx.x - le * N;
  const int e = e0 + le;
  const bool act = le < ne;
  Real* su = sm + le * 6 * N2;
  Real* sr = su + 3 * N2;
  const Real* __restrict__ U = static_cast<const Real*>(p.U);
  for (int i = threadIdx.x; i < ne * 3 * N2; i += blockDim.x) {
    const int l = i / (3 * N2);
    sm[l * 6 * N2 + (i - l * 3 * N2)] = U[(size_t)e0 * 3 * N2 + i];
  }
  __syncthreads();
  const Real* gA = static_cast<const Real*>(p.geoA) + (size_t)(act ? e : 0) * geo2_stride_A(N);
  const Real* gF = static_cast<const Real*>(p.geoF) + (size_t)(act ? e : 0) * geo2_stride_F(N);
  const Real* gM = static_cast<const Real*>(p.geoM) + (size_t)(act ? e : 0) * geo2_stride_M(N);
  if (act) {  // x: row y = t
    Real u[3][N], r[3][N];
#pragma unroll
    for (int fl = 0; fl < 3; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) u[fl][s] = su[fl * N2 + s + N * t];
    cell_face_dir2<N, Real, 0, false>(u, r, gA, gF, p, U, e, t);
#pragma unroll
    for (int fl = 0; fl < 3; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) sr[fl * N2 + s + N * t] = r[fl][s];
  }
  __syncthreads();
  if (act) {  // y: column x = t, then the diagonal inverse mass and the epilogue
    Real u[3][N], r[3][N];
#pragma unroll
    for (int fl = 0; fl < 3; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) {
        u[fl][s] = su[fl * N2 + t + N * s];
        r[fl][s] = sr[fl * N2 + t + N * s];
      }
    cell_face_dir2<N, Real, 1, true>(u, r, gA, gF, p, U, e, t);
    Real* __restrict__ out = static_cast<Real*>(p.out);
    const Real* __restrict__ Uadd = static_cast<const Real*>(p.Uadd);
    Real* __restrict__ dU = static_cast<Real*>(p.dU);
    const Real cA = (Real)p.cA, cB = (Real)p.cB, dt = (Real)p.dt;
    const size_t g0 = (size_t)e * 3 * N2 + t;
#pragma unroll
    for (int s = 0; s < N; ++s) {
      const Real mp = __ldg(gM + t + N * s), mvv = __ldg(gM + N2 + t + N * s);
#pragma unroll
      for (int fl = 0; fl < 3; ++fl) {
        const Real R = r[fl][s] * (fl == 0 ? mp : mvv);
        const size_t g = g0 + fl * N2 + N * s;
        if (EPI == EPI_WRITE) {
          out[g] = R;
        } else if (EPI == EPI_ADD) {
          out[g] = Uadd[g] + R;
        } else {
          const Real d = p.first ? dt * R : fma(cA, dU[g], dt * R);
          dU[g] = d;
          out[g] = fma(cB, d, Uadd[g]);
        }
      }
    }
  }
}

// levels of the 2D predictor: m = N, N - RED, ... >= 1
template <int N, int RED>
__host__ __device__ constexpr int tck2_level_count() {
  return RED == 0 ? 1 : (N - 1) / RED + 1;
}
template <int N, int RED>
__host__ __device__ constexpr int tck2_acc_off(int l) {
  return l == 0 ? 0 : tck2_acc_off<N, RED>(l - 1) + 3 * (N - RED * (l - 1)) * (N - RED * (l - 1));
}
template <int N, int RED>
__host__ __device__ constexpr int tck2_smem_per_elem() {
  return 6 * N * N + tck2_acc_off<N, RED>(tck2_level_count<N, RED>());
}

// One derivative T_j = -S T_{j-1} at an M^2 Gauss set for ne elements (lines
// spread over the block); g0: element 0's geometry of the set, gs: stride.
template <int M, typename Real, int FS>
__device__ __forceinline__ void tck2_derivative(const Real* src0, Real* dst0, int es, const Real* __restrict__ g0,
                                                long long gs, int ne, int T, int nthr) {
  constexpr int M2 = M * M;
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    for (int L = T; L < ne * M; L += nthr) {
      const int le = L / M, l = L - le * M;
      const Real* src = src0 + le * es;
      Real* dst = dst0 + le * es;
      const Real* g = g0 + le * gs;
      const int base = dir == 0 ? M * l : l;
      const int st = dir == 0 ? 1 : M;
      Real q[3][M], d[3][M];
#pragma unroll
      for (int fl = 0; fl < 3; ++fl) {
#pragma unroll
        for (int s = 0; s < M; ++s) q[fl][s] = src[fl * FS + base + st * s];
        mv<Real, OFF_D(M), M, M>(q[fl], d[fl]);
      }
      const Real* J0 = g + (dir * 2 + 0) * M2 + l;
      const Real* J1 = g + (dir * 2 + 1) * M2 + l;
#pragma unroll
      for (int s = 0; s < M; ++s) {
        const Real j0 = __ldg(J0 + M * s), j1 = __ldg(J1 + M * s);
        const int idx = base + st * s;
        Real tp, tv0, tv1;
        if (dir > 0) {
          tp = fma(j0, d[1][s], fma(j1, d[2][s], dst[idx]));
          tv0 = fma(j0, d[0][s], dst[FS + idx]);
          tv1 = fma(j1, d[0][s], dst[2 * FS + idx]);
          const Real cp = __ldg(g + 4 * M2 + idx), cv = __ldg(g + 5 * M2 + idx);
          tp *= cp;
          tv0 *= cv;
          tv1 *= cv;
        } else {
          tp = fma(j0, d[1][s], j1 * d[2][s]);
          tv0 = j0 * d[0][s];
          tv1 = j1 * d[0][s];
        }
        dst[idx] = tp;
        dst[FS + idx] = tv0;
        dst[2 * FS + idx] = tv1;
      }
    }
    __syncthreads();
  }
}

template <int M, int RR, typename Real, int FS>
__device__ __forceinline__ void tck2_project(Real* src0, Real* tmp0, int es, int ne, int T, int nthr) {
  constexpr int R = M - RR;
  contract_tile2<Real, 0, M, M, R, OFF_PR(M, RR), FS, FS>(src0, tmp0, es, ne, T, nthr);
  __syncthreads();
  contract_tile2<Real, 1, R, M, R, OFF_PR(M, RR), FS, FS>(tmp0, src0, es, ne, T, nthr);
  __syncthreads();
}

// acc_big += I(M+RR <- M) acc_small in both directions (acc_small field stride M^2)
template <int M, int RR, typename Real, int FS>
__device__ __forceinline__ void tck2_fold(const Real* small0, Real* big0, Real* t10, int es, int ne, int T,
                                          int nthr) {
  constexpr int B = M + RR;
  contract_tile2<Real, 0, M, M, B, OFF_IR(B, RR), M * M, FS>(small0, t10, es, ne, T, nthr);
  __syncthreads();
  contract_tile2<Real, 1, B, M, B, OFF_IR(B, RR), FS, B * B, true>(t10, big0, es, ne, T, nthr);
  __syncthreads();
}

// The 2D predictor on Gauss-basis states (Sec. 2.3 Eq. (6), Sec. 3.2-3.3):
// lines, points and accumulator entries of all the block's elements are
// spread over every thread.
template <int N, typename Real, int RED>
__global__ void tck2d_kernel(const Tck2Params p) {
  constexpr int N2 = N * N;
  constexpr int SE = tck2_smem_per_elem<N, RED>();
  constexpr int NL = tck2_level_count<N, RED>();
  constexpr int ACC = 6 * N2;
  constexpr int NACC = tck2_acc_off<N, RED>(NL);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int epb = blockDim.x / N;
  const int e0 = blockIdx.x * epb, ne = min(epb, p.E - e0);
  const int T = threadIdx.x, NT = blockDim.x;
  const Real* __restrict__ U = static_cast<const Real*>(p.U);
  const Real* geo0 = static_cast<const Real*>(p.geoT) + (size_t)e0 * p.geoT_stride;
  for (int i = T; i < ne * 3 * N2; i += NT) {
    const int l = i / (3 * N2);
    sm[l * SE + (i - l * 3 * N2)] = U[(size_t)e0 * 3 * N2 + i];
  }
  for (int i = T; i < ne * NACC; i += NT) {
    const int l = i / NACC;
    sm[l * SE + ACC + (i - l * NACC)] = Real(0);
  }
  __syncthreads();
  // accumulate c T over the block (T field stride N2, acc field stride m^2)
  auto accumulate = [&](int aoff, const Real* T0, int m2, Real c) {
    for (int i = T; i < ne * 3 * m2; i += NT) {
      const int le = i / (3 * m2), r = i - le * 3 * m2;
      const int fl = r / m2, q = r - fl * m2;
      Real* acc = sm + le * SE + ACC + aoff;
      acc[r] = fma(c, T0[le * SE + fl * N2 + q], acc[r]);
    }
  };
  accumulate(0, sm, N2, (Real)p.coef[0]);
  Real* cur = sm;
  Real* nxt = sm + 3 * N2;
  int m = N, goff = 0, aoff = 0;
#pragma unroll 1
  for (int j = 1; j <= N; ++j) {
    switch (m) {
#define DG_TCK2_DERIV(MM)                                                                   \
  case MM:                                                                                  \
    if constexpr (MM <= N) tck2_derivative<MM, Real, N2>(cur, nxt, SE, geo0 + goff, p.geoT_stride, ne, T, NT); \
    break;
      DG_TCK2_DERIV(2) DG_TCK2_DERIV(3) DG_TCK2_DERIV(4) DG_TCK2_DERIV(5) DG_TCK2_DERIV(6)
      DG_TCK2_DERIV(7) DG_TCK2_DERIV(8)
#undef DG_TCK2_DERIV
      default:  // m == 1: the derivative of a constant vanishes
        for (int i = T; i < ne * 3 * N2; i += NT) {
          const int l = i / (3 * N2);
          nxt[l * SE + (i - l * 3 * N2)] = Real(0);
        }
        __syncthreads();
        break;
    }
    if (RED > 0 && (j % RED) == 0) {
      if (m - RED < 1) break;
      switch (m) {
#define DG_TCK2_PROJ(MM)                                                                               \
  case MM:                                                                                             \
    if constexpr (RED > 0 && MM <= N && MM - RED >= 1) tck2_project<MM, RED, Real, N2>(nxt, cur, SE, ne, T, NT); \
    break;
        DG_TCK2_PROJ(2) DG_TCK2_PROJ(3) DG_TCK2_PROJ(4) DG_TCK2_PROJ(5) DG_TCK2_PROJ(6) DG_TCK2_PROJ(7)
        DG_TCK2_PROJ(8)
#undef DG_TCK2_PROJ
        default:
          break;
      }
      // the projection leaves its result in nxt (two passes: nxt -> cur -> nxt)
      const int gs = p.geo_step > 1 ? 2 : 1;
      for (int mm = m; mm > m - RED; mm -= gs) goff += 6 * mm * mm;
      aoff += 3 * m * m;
      m -= RED;
    }
    accumulate(aoff, nxt, m * m, (Real)p.coef[j]);
    __syncthreads();
    Real* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  if (RED > 0) {
#pragma unroll
    for (int l = NL - 1; l >= 1; --l) {
      const int ms = N - RED * l;
      Real* small = sm + ACC + tck2_acc_off<N, RED>(l);
      Real* big = sm + ACC + tck2_acc_off<N, RED>(l - 1);
      switch (ms) {
#define DG_TCK2_FOLD(MM)                                                                           \
  case MM:                                                                                         \
    if constexpr (RED > 0 && MM + RED <= N) tck2_fold<MM, RED, Real, N2>(small, big, sm, SE, ne, T, NT); \
    break;
        DG_TCK2_FOLD(1) DG_TCK2_FOLD(2) DG_TCK2_FOLD(3) DG_TCK2_FOLD(4) DG_TCK2_FOLD(5) DG_TCK2_FOLD(6)
        DG_TCK2_FOLD(7)
#undef DG_TCK2_FOLD
        default:
          break;
      }
    }
  }
  Real* __restrict__ out = static_cast<Real*>(p.Ubar);
  __syncthreads();
  for (int i = T; i < ne * 3 * N2; i += NT) {
    const int l = i / (3 * N2);
    out[(size_t)e0 * 3 * N2 + i] = sm[l * SE + ACC + (i - l * 3 * N2)];
  }
}

// Discrete energy 1/2 U^T M U of GL states (partial sums per block, fixed order).
template <int N, typename Real>
__global__ void energy2d_kernel(const Energy2Params p) {
  constexpr int N2 = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int epb = blockDim.x / N;
  const int e0 = blockIdx.x * epb, ne = min(epb, p.E - e0);
  const Real* U = static_cast<const Real*>(p.U);
  for (int i = threadIdx.x; i < ne * 3 * N2; i += blockDim.x) sm[i] = U[(size_t)e0 * 3 * N2 + i];
  __syncthreads();
  contract_tile2<Real, 0, N, N, N, OFF_V(N), N2, N2>(sm, sm, 3 * N2, ne, threadIdx.x, blockDim.x);
  __syncthreads();
  contract_tile2<Real, 1, N, N, N, OFF_V(N), N2, N2>(sm, sm, 3 * N2, ne, threadIdx.x, blockDim.x);
  __syncthreads();
  double s = 0.0;
  for (int i = threadIdx.x; i < ne * N2; i += blockDim.x) {
    const int le = i / N2, q = i - le * N2;
    const Real* gM = static_cast<const Real*>(p.geoM) + (size_t)(e0 + le) * geo2_stride_M(N);
    const Real* su = sm + le * 3 * N2;
    const double pp = su[q], vx = su[N2 + q], vy = su[2 * N2 + q];
    s += pp * pp / (double)gM[q] + (vx * vx + vy * vy) / (double)gM[N2 + q];
  }
  __shared__ double red[1024];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) tot += red[i];
    p.partial[blockIdx.x] = 0.5 * tot;
  }
}

}  // namespace dg
