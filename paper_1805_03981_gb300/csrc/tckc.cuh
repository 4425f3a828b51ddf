// Predictor of ADER (the Taylor-Cauchy-Kowalevski sum, Sec. 2.3 Eq. (6),
// Sec. 3.2 Alg. 2, Sec. 3.3 Alg. 3) for Gauss-point states: the "column"
// form.  It computes what tck_block computes in gmode, with the work laid
// out for fewer shared-memory and index instructions:
//
// * Each phase spreads its work items (columns, x-lines or y-lines of the
//   current Gauss set) of all the block's elements over consecutive threads:
//   item i of element e goes to thread e * count + i, count being the items
//   per element.  At the full set (m = n, count n^2) thread e n^2 + t owns
//   the z-column (x, y) = (t % n, t / n) of element e; at a reduced set the
//   m^2 columns of every element are packed the same way, so the phase
//   occupies ne m^2 threads in whole warps instead of m^2 of every n^2 (the
//   idle threads skip it).  The owner of a column holds the current Taylor
//   term T_j on it for all four fields, in registers.
// * A derivative T_j = -S T_{j-1} (collocation at the m^3 Gauss points)
//   differentiates along z in registers.  For x and y the column owners
//   write their columns once to shared memory; thread t then owns the
//   x-line (y, z) = (t % m, t / m) and the y-line (x, z) = (t % m, t / m),
//   differentiates them, multiplies by the metric terms of that reference
//   direction and writes the partial sums, which the column owners read
//   back, add to their own z part and scale by the coefficients -rho c^2
//   and -1/rho.  On an affine element with constant coefficients the
//   pressure equation differentiates w_d = sum_i (J^-1)_{d i} v_i, so a line
//   carries two fields instead of four.
// * Degree reduction (reference L2 projection m -> m - RED) contracts z in
//   registers and x, y through shared memory; the prolongations that fold
//   the smaller levels' sums into the n-point one (Sec. 3.3) likewise.
// * The n-point accumulator stays in registers; the smaller levels'
//   accumulators sit in shared memory, each entry touched only by the
//   thread that owns its column at that level.
// * N and RED fix the level sequence at compile time, so every loop is
//   unrolled and every shared-memory offset is a constant plus the thread's
//   base.  Tiles are padded (node (x, y, z) of an m-point level at
//   x + tckc_P(m) y + tckc_Q(m) z) so that the columns, x-lines and y-lines
//   a warp touches at once fall into distinct banks, up to two-way
//   conflicts where a warp spans more than one element or m^2 > 32.
#pragma once

#include "kern_inst.cuh"

namespace dg {

__host__ __device__ constexpr int tckc_P(int m) { return m == 8 ? 9 : m; }
__host__ __device__ constexpr int tckc_Q(int m) {
  return m == 4 ? 19 : (m == 7 ? 52 : (m == 8 ? 72 : m * m));
}
// residue mod 32 of the per-element shared-memory stride (Reals) that keeps
// neighbouring elements' lines in different banks
__host__ __device__ constexpr int tckc_pad(int n) {
  return n == 2 ? 7 : (n == 3 ? 27 : (n == 4 ? 16 : (n == 5 ? 25 : (n == 6 ? 27 : (n == 7 ? 5 : 0)))));
}

template <int N, int RED, bool AFF>
struct TckcShape {
  static constexpr int FT = tckc_Q(N) * N;  // field stride of the line buffers
  static constexpr int NBUF = AFF ? 8 : 12;  // line buffers, in fields (the projection needs 8)
  static constexpr int NA = AFF ? 3 : 4;     // fields written by the column owners
  static constexpr int NB = AFF ? 2 : 4;     // partial sums per line direction
  static constexpr int NL = tck_level_count<N, RED>();
  static constexpr int ACC = NBUF * FT;      // accumulators of levels 1 .. NL-1, [4][m^3] each
  static constexpr int RAW = ACC + tck_acc_off<N, RED>(NL) - 4 * N * N * N;
  static constexpr int SE = RAW + (((tckc_pad(N) - RAW % 32) % 32) + 32) % 32;  // Reals per element
  static constexpr int acc_off(int l) { return ACC + tck_acc_off<N, RED>(l) - 4 * N * N * N; }
};

template <typename Real>
struct TckcCtx {
  Real* sm;             // the block's shared memory (element slots SE Reals apart)
  const Real* geoT;     // predictor geometry of the block's first element (curved)
  long long geoT_stride;
  const Real* geoKT;    // compact predictor data of the block's first element (affine)
  int ne;               // elements in the block
  int geo_step;         // stored Gauss sets m = n, n - geo_step, ...
};

// The work item of this thread in a phase with COUNT items per element:
// element slot le, item t; on = the item exists.
template <int COUNT>
struct TckcSlot {
  int le, t;
  bool on;
  template <typename Real>
  __device__ __forceinline__ explicit TckcSlot(const TckcCtx<Real>& x) {
    le = threadIdx.x / COUNT;
    t = threadIdx.x - le * COUNT;
    on = le < x.ne;
  }
};

// geometry of the m-point set: the stored sets above it come first
template <int N>
__device__ __forceinline__ int tckc_geo_off(int m, int geo_step) {
  const int st = geo_step > 1 ? 2 : 1;
  int off = 0;
  for (int mm = N; mm > m; mm -= st) off += 11 * mm * mm * mm;
  return off;
}

// T_j = -S T_{j-1} at the M-point set, column registers in and out.
template <int N, typename Real, int RED, bool AFF, int M>
__device__ __forceinline__ void tckc_derivative(Real (&c)[4][N], const TckcCtx<Real>& x) {
  using SH = TckcShape<N, RED, AFF>;
  constexpr int P = tckc_P(M), Q = tckc_Q(M), FT = SH::FT;
  constexpr int M2 = M * M, M3 = M2 * M;
  const TckcSlot<M2> w(x);  // column (a, b), x-line (y, z) = (a, b), y-line (x, z) = (a, b)
  Real* A = x.sm + w.le * SH::SE;
  Real* BX = A + SH::NA * FT;
  Real* BY = BX + SH::NB * FT;
  const bool on = w.on;
  const int a = w.t % M, b = w.t / M;
  const int cb = a + P * b;  // column (x, y) = (a, b)
  const Real* __restrict__ g =
      AFF ? nullptr : x.geoT + (size_t)(on ? w.le : 0) * x.geoT_stride + tckc_geo_off<N>(M, x.geo_step);
  Real gk[11];  // affine: (J^-1)_{d i} at gk[3 d + i], -rho c^2, -1/rho
  if constexpr (AFF) {
    const Real* k = x.geoKT + (size_t)(on ? w.le : 0) * DG_AFF_TCK;
#pragma unroll
    for (int i = 0; i < 11; ++i) gk[i] = __ldg(k + i);
  }
  Real zc[SH::NB][M];
  if (on) {
    if constexpr (AFF) {
      Real p[M], w2[M];
#pragma unroll
      for (int z = 0; z < M; ++z) {
        const Real v0 = c[1][z], v1 = c[2][z], v2 = c[3][z];
        p[z] = c[0][z];
        A[cb + Q * z] = p[z];
        A[FT + cb + Q * z] = fma(gk[0], v0, fma(gk[1], v1, gk[2] * v2));
        A[2 * FT + cb + Q * z] = fma(gk[3], v0, fma(gk[4], v1, gk[5] * v2));
        w2[z] = fma(gk[6], v0, fma(gk[7], v1, gk[8] * v2));
      }
      mv<Real, OFF_D(M), M, M>(p, zc[0]);
      mv<Real, OFF_D(M), M, M>(w2, zc[1]);
    } else {
      Real d[4][M];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
#pragma unroll
        for (int z = 0; z < M; ++z) A[f * FT + cb + Q * z] = c[f][z];
        mv<Real, OFF_D(M), M, M>(c[f], d[f]);
      }
#pragma unroll
      for (int z = 0; z < M; ++z) {
        const Real j0 = __ldg(g + 6 * M3 + w.t + M2 * z), j1 = __ldg(g + 7 * M3 + w.t + M2 * z),
                   j2 = __ldg(g + 8 * M3 + w.t + M2 * z);
        zc[0][z] = fma(j0, d[1][z], fma(j1, d[2][z], j2 * d[3][z]));
        zc[1][z] = j0 * d[0][z];
        zc[2][z] = j1 * d[0][z];
        zc[3][z] = j2 * d[0][z];
      }
    }
  }
  __syncthreads();
  if (on) {
    const int xb = P * a + Q * b;  // x-line (y, z) = (a, b)
    const int yb = a + Q * b;      // y-line (x, z) = (a, b)
    if constexpr (AFF) {
      Real q[2][M], d[2][M];
#pragma unroll
      for (int s = 0; s < M; ++s) {
        q[0][s] = A[xb + s];
        q[1][s] = A[FT + xb + s];
      }
      mv<Real, OFF_D(M), M, M>(q[0], d[0]);
      mv<Real, OFF_D(M), M, M>(q[1], d[1]);
#pragma unroll
      for (int s = 0; s < M; ++s) {
        BX[xb + s] = d[0][s];
        BX[FT + xb + s] = d[1][s];
      }
#pragma unroll
      for (int s = 0; s < M; ++s) {
        q[0][s] = A[yb + P * s];
        q[1][s] = A[2 * FT + yb + P * s];
      }
      mv<Real, OFF_D(M), M, M>(q[0], d[0]);
      mv<Real, OFF_D(M), M, M>(q[1], d[1]);
#pragma unroll
      for (int s = 0; s < M; ++s) {
        BY[yb + P * s] = d[0][s];
        BY[FT + yb + P * s] = d[1][s];
      }
    } else {
      Real q[4][M], d[4][M];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
#pragma unroll
        for (int s = 0; s < M; ++s) q[f][s] = A[f * FT + xb + s];
        mv<Real, OFF_D(M), M, M>(q[f], d[f]);
      }
#pragma unroll
      for (int s = 0; s < M; ++s) {
        const Real j0 = __ldg(g + 0 * M3 + w.t + M2 * s), j1 = __ldg(g + 1 * M3 + w.t + M2 * s),
                   j2 = __ldg(g + 2 * M3 + w.t + M2 * s);
        BX[xb + s] = fma(j0, d[1][s], fma(j1, d[2][s], j2 * d[3][s]));
        BX[FT + xb + s] = j0 * d[0][s];
        BX[2 * FT + xb + s] = j1 * d[0][s];
        BX[3 * FT + xb + s] = j2 * d[0][s];
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
#pragma unroll
        for (int s = 0; s < M; ++s) q[f][s] = A[f * FT + yb + P * s];
        mv<Real, OFF_D(M), M, M>(q[f], d[f]);
      }
#pragma unroll
      for (int s = 0; s < M; ++s) {
        const Real j0 = __ldg(g + 3 * M3 + w.t + M2 * s), j1 = __ldg(g + 4 * M3 + w.t + M2 * s),
                   j2 = __ldg(g + 5 * M3 + w.t + M2 * s);
        BY[yb + P * s] = fma(j0, d[1][s], fma(j1, d[2][s], j2 * d[3][s]));
        BY[FT + yb + P * s] = j0 * d[0][s];
        BY[2 * FT + yb + P * s] = j1 * d[0][s];
        BY[3 * FT + yb + P * s] = j2 * d[0][s];
      }
    }
  }
  __syncthreads();
  if (on) {
#pragma unroll
    for (int z = 0; z < M; ++z) {
      const int i = cb + Q * z;
      if constexpr (AFF) {
        const Real dxp = BX[i], dxw = BX[FT + i], dyp = BY[i], dyw = BY[FT + i];
        c[0][z] = gk[9] * (dxw + dyw + zc[1][z]);
        c[1][z] = gk[10] * fma(gk[0], dxp, fma(gk[3], dyp, gk[6] * zc[0][z]));
        c[2][z] = gk[10] * fma(gk[1], dxp, fma(gk[4], dyp, gk[7] * zc[0][z]));
        c[3][z] = gk[10] * fma(gk[2], dxp, fma(gk[5], dyp, gk[8] * zc[0][z]));
      } else {
        const Real cp = __ldg(g + 9 * M3 + w.t + M2 * z), cv = __ldg(g + 10 * M3 + w.t + M2 * z);
        c[0][z] = cp * (zc[0][z] + BX[i] + BY[i]);
#pragma unroll
        for (int f = 1; f < 4; ++f) c[f][z] = cv * (zc[f][z] + BX[f * FT + i] + BY[f * FT + i]);
      }
    }
  }
}

// Reference L2 projection M -> MR (Sec. 3.3) of the column registers; on
// return the owners of the MR-point columns (packed) hold them.
template <int N, typename Real, int RED, bool AFF, int M, int MR>
__device__ __forceinline__ void tckc_project(Real (&c)[4][N], const TckcCtx<Real>& x) {
  using SH = TckcShape<N, RED, AFF>;
  constexpr int P = tckc_P(M), Q = tckc_Q(M), PR = tckc_P(MR), QR = tckc_Q(MR), FT = SH::FT;
  constexpr int OFF = OFF_PR(M, M - MR);  // MR x M
  {  // z, in the registers of the M-point column owners
    const TckcSlot<M * M> w(x);
    if (w.on) {
      Real* S1 = x.sm + w.le * SH::SE;
      const int cb = w.t % M + P * (w.t / M);
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        Real o[MR];
        mv<Real, OFF, MR, M>(c[f], o);
#pragma unroll
        for (int z = 0; z < MR; ++z) S1[f * FT + cb + Q * z] = o[z];
      }
    }
  }
  __syncthreads();
  {  // x-lines (y, z), y < M, z < MR
    const TckcSlot<M * MR> w(x);
    if (w.on) {
      Real* S1 = x.sm + w.le * SH::SE;
      Real* S2 = S1 + 4 * FT;
      const int base = P * (w.t % M) + Q * (w.t / M);
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        Real in[M], o[MR];
#pragma unroll
        for (int s = 0; s < M; ++s) in[s] = S1[f * FT + base + s];
        mv<Real, OFF, MR, M>(in, o);
#pragma unroll
        for (int s = 0; s < MR; ++s) S2[f * FT + base + s] = o[s];
      }
    }
  }
  __syncthreads();
  {  // y-lines (x, z), x, z < MR; written in the MR-point layout
    const TckcSlot<MR * MR> w(x);
    if (w.on) {
      Real* S1 = x.sm + w.le * SH::SE;
      Real* S2 = S1 + 4 * FT;
      const int xx = w.t % MR, zz = w.t / MR;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        Real in[M], o[MR];
#pragma unroll
        for (int s = 0; s < M; ++s) in[s] = S2[f * FT + xx + P * s + Q * zz];
        mv<Real, OFF, MR, M>(in, o);
#pragma unroll
        for (int s = 0; s < MR; ++s) S1[f * FT + xx + PR * s + QR * zz] = o[s];
      }
    }
  }
  __syncthreads();
  {  // the new column owners read their columns
    const TckcSlot<MR * MR> w(x);
    if (w.on) {
      const Real* S1 = x.sm + w.le * SH::SE;
      const int cb = w.t % MR + PR * (w.t / MR);
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int z = 0; z < MR; ++z) c[f][z] = S1[f * FT + cb + QR * z];
    }
  }
}

// acc(level L) += cj T (or = cj T when FIRST), by the owners of the M-point columns
template <int N, typename Real, int RED, bool AFF, int L, int M, bool FIRST>
__device__ __forceinline__ void tckc_accumulate(const Real (&c)[4][N], Real (&acc)[4][N],
                                                const TckcCtx<Real>& x, Real cj) {
  const TckcSlot<M * M> w(x);
  if (!w.on) return;
  if constexpr (L == 0) {
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int z = 0; z < M; ++z) acc[f][z] = fma(cj, c[f][z], acc[f][z]);
  } else {
    constexpr int M3 = M * M * M;
    Real* a = x.sm + w.le * TckcShape<N, RED, AFF>::SE + TckcShape<N, RED, AFF>::acc_off(L);
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int z = 0; z < M; ++z) {
        Real* q = a + f * M3 + w.t + M * M * z;
        *q = FIRST ? cj * c[f][z] : fma(cj, c[f][z], *q);
      }
  }
}

// Taylor terms J .. N; M: points of the set T_{J-1} lives on
template <int N, typename Real, int RED, bool AFF, int J, int M>
__device__ __forceinline__ void tckc_steps(Real (&c)[4][N], Real (&acc)[4][N], const TckcCtx<Real>& x,
                                           const TckParams& p, const Real* __restrict__ W) {
  if constexpr (J <= N && M >= 2) {  // at M = 1 the derivative of a constant vanishes: so does every later term
    if (J == 1 && W) {  // HDG-ADER (Eq. hdg-ader): the DG derivative in place of -S U
      constexpr int N2 = N * N, N3 = N2 * N;
      const TckcSlot<N2> w(x);
      if (w.on)
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
          for (int z = 0; z < N; ++z) c[f][z] = __ldg(W + f * N3 + w.t + N2 * z);
    } else {
      tckc_derivative<N, Real, RED, AFF, M>(c, x);
    }
    const Real cj = (Real)p.coef[J];
    if constexpr (RED > 0 && J % RED == 0) {
      if constexpr (M - RED >= 1) {  // else projected to a negative degree: T_J = 0, stop
        tckc_project<N, Real, RED, AFF, M, M - RED>(c, x);
        tckc_accumulate<N, Real, RED, AFF, J / RED, M - RED, true>(c, acc, x, cj);
        tckc_steps<N, Real, RED, AFF, J + 1, M - RED>(c, acc, x, p, W);
      }
    } else {
      constexpr int L = RED > 0 ? (N - M) / RED : 0;
      tckc_accumulate<N, Real, RED, AFF, L, M, false>(c, acc, x, cj);
      tckc_steps<N, Real, RED, AFF, J + 1, M>(c, acc, x, p, W);
    }
  }
}

// acc(level L - 1) += I(M -> M + RED) acc(level L), in x, y through shared
// memory and z in the registers of the (M + RED)-point column owners.
template <int N, typename Real, int RED, bool AFF, int L>
__device__ __forceinline__ void tckc_fold(Real (&acc)[4][N], const TckcCtx<Real>& x) {
  using SH = TckcShape<N, RED, AFF>;
  constexpr int M = N - RED * L, B = M + RED;
  constexpr int M2 = M * M, M3 = M2 * M;
  constexpr int PB = tckc_P(B), QB = tckc_Q(B), FT = SH::FT;
  constexpr int OFF = OFF_IR(B, RED);  // B x M
  {  // x-lines (y, z) of the compact M^3 sums
    const TckcSlot<M2> w(x);
    if (w.on) {
      Real* sE = x.sm + w.le * SH::SE;
      const Real* src = sE + SH::acc_off(L);
      const int y = w.t % M, z = w.t / M;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        Real in[M], o[B];
#pragma unroll
        for (int s = 0; s < M; ++s) in[s] = src[f * M3 + s + M * y + M2 * z];
        mv<Real, OFF, B, M>(in, o);
#pragma unroll
        for (int s = 0; s < B; ++s) sE[f * FT + s + PB * y + QB * z] = o[s];
      }
    }
  }
  __syncthreads();
  {  // y-lines (x, z), x < B, z < M
    const TckcSlot<B * M> w(x);
    if (w.on) {
      Real* S1 = x.sm + w.le * SH::SE;
      Real* S2 = S1 + 4 * FT;
      const int xx = w.t % B, z = w.t / B;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        Real in[M], o[B];
#pragma unroll
        for (int s = 0; s < M; ++s) in[s] = S1[f * FT + xx + PB * s + QB * z];
        mv<Real, OFF, B, M>(in, o);
#pragma unroll
        for (int s = 0; s < B; ++s) S2[f * FT + xx + PB * s + QB * z] = o[s];
      }
    }
  }
  __syncthreads();
  {  // z, by the B-point column owners
    const TckcSlot<B * B> w(x);
    if (w.on) {
      Real* sE = x.sm + w.le * SH::SE;
      const Real* S2 = sE + 4 * FT;
      const int cb = w.t % B + PB * (w.t / B);
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        Real in[M], o[B];
#pragma unroll
        for (int s = 0; s < M; ++s) in[s] = S2[f * FT + cb + QB * s];
        mv<Real, OFF, B, M>(in, o);
        if constexpr (L == 1) {
#pragma unroll
          for (int z = 0; z < B; ++z) acc[f][z] += o[z];
        } else {
          Real* dst = sE + SH::acc_off(L - 1) + f * B * B * B + w.t;
#pragma unroll
          for (int z = 0; z < B; ++z) dst[B * B * z] += o[z];
        }
      }
    }
  }
  __syncthreads();
  if constexpr (L > 1) tckc_fold<N, Real, RED, AFF, L - 1>(acc, x);
}

// The predictor for elements e0 .. e0+ne-1 (ne <= the block's element slots).
template <int N, typename Real, int RED, bool AFF>
__device__ __forceinline__ void tckc_block(const TckParams& p, const int e0, const int ne, Real* sm) {
  using SH = TckcShape<N, RED, AFF>;
  constexpr int N2 = N * N, N3 = N2 * N;
  TckcCtx<Real> x;
  x.sm = sm;
  x.ne = ne;
  x.geo_step = p.geo_step;
  x.geoT_stride = p.geoT_stride;
  x.geoT = AFF ? nullptr : static_cast<const Real*>(p.geoT) + (size_t)e0 * (size_t)p.geoT_stride;
  x.geoKT = AFF ? static_cast<const Real*>(p.geoKT) + (size_t)e0 * DG_AFF_TCK : nullptr;
  const TckcSlot<N2> w(x);  // the n-point column owners: thread le n^2 + t
  const size_t e = (size_t)e0 + (w.on ? w.le : 0);
  const Real* __restrict__ U = static_cast<const Real*>(p.U) + e * 4 * N3;
  const Real* __restrict__ W = p.W ? static_cast<const Real*>(p.W) + e * 4 * N3 : nullptr;
  Real c[4][N], acc[4][N];
  const Real c0 = (Real)p.coef[0];
  if (w.on) {
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int z = 0; z < N; ++z) {
        c[f][z] = __ldg(U + f * N3 + w.t + N2 * z);
        acc[f][z] = c0 * c[f][z];
      }
  }
  tckc_steps<N, Real, RED, AFF, 1, N>(c, acc, x, p, W);
  if constexpr (SH::NL > 1) {
    __syncthreads();
    tckc_fold<N, Real, RED, AFF, SH::NL - 1>(acc, x);
  }
  if (w.on) {
    Real* __restrict__ out = static_cast<Real*>(p.Ubar) + e * 4 * N3;
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int z = 0; z < N; ++z) out[f * N3 + w.t + N2 * z] = acc[f][z];
  }
}

template <int N, typename Real, int RED, bool AFF>
__global__ void tckc_kernel(const TckParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int epb = blockDim.x / (N * N);
  const int e0 = blockIdx.x * epb;
  tckc_block<N, Real, RED, AFF>(p, e0, min(epb, p.E - e0), reinterpret_cast<Real*>(smem_raw));
}

// One slice of a work item, kept out of line: inlined into the persistent
// loop, the compiler hoists the slice's many loop-invariant addresses into
// registers (twice the registers of tckc_kernel, and spills from n = 7).
template <int N, typename Real, int RED, bool AFF>
__device__ __noinline__ void tckc_slice(const TckParams& p, int e0, int ne, Real* sm) {
  tckc_block<N, Real, RED, AFF>(p, e0, ne, sm);
}

// Batched form: one launch per degree over a list of slices (an instance
// and up to epb of its elements), one block per slice, in the order of the
// list.  The per-element code is tckc_block's, so a solve's result does not
// depend on the batch.  Unlike the other batched kernels it is not
// persistent: inside a persistent loop the compiler keeps twice the
// registers live (250 instead of 128 at n = 6) and spills from n = 7.
template <int N, typename Real, int RED, bool AFF>
__global__ void batch_tckc_kernel(const BatchItem* __restrict__ slices, const BatchInst* __restrict__ inst) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchItem w = slices[blockIdx.x];
  tckc_block<N, Real, RED, AFF>(inst[w.inst].tck, w.e0, w.ne, reinterpret_cast<Real*>(smem_raw));
}

template <int N, typename Real, int RED>
int tckc_smem_bytes(int aff) {
  return (aff ? TckcShape<N, RED, true>::SE : TckcShape<N, RED, false>::SE) * (int)sizeof(Real);
}

template <int N, typename Real, int RED>
cudaError_t launch_tckc_red(const TckParams& p, int epb, cudaStream_t st) {
  const int threads = epb * N * N;
  const int blocks = (p.E + epb - 1) / epb;
  const size_t smem = (size_t)epb * tckc_smem_bytes<N, Real, RED>(p.aff);
  if (p.aff)
    tckc_kernel<N, Real, RED, true><<<blocks, threads, smem, st>>>(p);
  else
    tckc_kernel<N, Real, RED, false><<<blocks, threads, smem, st>>>(p);
  return cudaGetLastError();
}

// Every reduction (0, 1, 2, 3); gmode states only.
template <int N, typename Real>
cudaError_t launch_tckc(const TckParams& p, int red, int epb, cudaStream_t st) {
  if (!p.gmode) return cudaErrorInvalidValue;
  switch (red) {
    case 0: return launch_tckc_red<N, Real, 0>(p, epb, st);
    case 1: return launch_tckc_red<N, Real, 1>(p, epb, st);
    case 2: return launch_tckc_red<N, Real, 2>(p, epb, st);
    case 3: return launch_tckc_red<N, Real, 3>(p, epb, st);
    default: return cudaErrorInvalidValue;
  }
}

// per-element shared memory (bytes) of the largest variant for this reduction
template <int N, typename Real>
int tckc_smem(int red) {
  switch (red) {
    case 0: return max(tckc_smem_bytes<N, Real, 0>(0), tckc_smem_bytes<N, Real, 0>(1));
    case 1: return max(tckc_smem_bytes<N, Real, 1>(0), tckc_smem_bytes<N, Real, 1>(1));
    case 2: return max(tckc_smem_bytes<N, Real, 2>(0), tckc_smem_bytes<N, Real, 2>(1));
    default: return max(tckc_smem_bytes<N, Real, 3>(0), tckc_smem_bytes<N, Real, 3>(1));
  }
}

template <int N, typename Real>
int tckc_max_threads() {
  int m = 1024;
  m = min(m, kernel_max_threads(tckc_kernel<N, Real, 0, false>));
  m = min(m, kernel_max_threads(tckc_kernel<N, Real, 0, true>));
  m = min(m, kernel_max_threads(tckc_kernel<N, Real, 1, false>));
  m = min(m, kernel_max_threads(tckc_kernel<N, Real, 1, true>));
  m = min(m, kernel_max_threads(tckc_kernel<N, Real, 2, false>));
  m = min(m, kernel_max_threads(tckc_kernel<N, Real, 2, true>));
  m = min(m, kernel_max_threads(tckc_kernel<N, Real, 3, false>));
  m = min(m, kernel_max_threads(tckc_kernel<N, Real, 3, true>));
  return m;
}

template <int N, typename Real>
cudaError_t tckc_allow_smem() {
  cudaError_t e;
  if ((e = allow_smem(tckc_kernel<N, Real, 0, false>)) != cudaSuccess) return e;
  if ((e = allow_smem(tckc_kernel<N, Real, 0, true>)) != cudaSuccess) return e;
  if ((e = allow_smem(tckc_kernel<N, Real, 1, false>)) != cudaSuccess) return e;
  if ((e = allow_smem(tckc_kernel<N, Real, 1, true>)) != cudaSuccess) return e;
  if ((e = allow_smem(tckc_kernel<N, Real, 2, false>)) != cudaSuccess) return e;
  if ((e = allow_smem(tckc_kernel<N, Real, 2, true>)) != cudaSuccess) return e;
  if ((e = allow_smem(tckc_kernel<N, Real, 3, false>)) != cudaSuccess) return e;
  return allow_smem(tckc_kernel<N, Real, 3, true>);
}

template <int N, typename Real>
void register_tckc_one(KernelTable* t) {
  const int pi = sizeof(Real) == 8 ? 0 : 1;
  t->tckc[pi][N] = &launch_tckc<N, Real>;
  t->tckc_smem[pi][N] = &tckc_smem<N, Real>;
  t->tckc_maxthr[pi][N] = &tckc_max_threads<N, Real>;
}

}  // namespace dg
