// Predictor of ADER (the Taylor-Cauchy-Kowalevski sum, Sec. 2.3 Eq. (6),
// Sec. 3.2 Alg. 2, Sec. 3.3 Alg. 3) for Gauss-point states on affine
// elements with element-wise constant coefficients: the "interleaved" column
// form.  It computes what tckc_block computes for such elements, with the
// block's shared memory and threads arranged for fewer shared-memory
// wavefronts, and with each reduced Taylor term projected as it is formed:
//
// * A block holds EPB elements and EPB n^2 threads.  Thread T works on
//   element le = T % EPB in every phase, on item t = T / EPB (a column, an
//   x-line or a y-line of the current Gauss set, or nothing when t is past
//   the phase's item count).  At a reduced set of m points only the first
//   EPB m^2 threads work, in whole warps.
// * Shared memory is element-interleaved: word o of element le sits at
//   o EPB + le.  The EPB threads that take the same item of the EPB elements
//   are consecutive lanes and touch consecutive words, and the tile strides
//   (x + P(m) y + Q(m) z) put the lines a warp touches at once into disjoint
//   banks.
// * The state comes in and Ubar goes out by bulk asynchronous copies between
//   global memory and an element-blocked staging area (one contiguous run
//   per element), with the per-element stride chosen so that the column
//   reads and writes of the staging area are conflict free.
// * The Taylor terms themselves follow the column form: the column owner
//   keeps T_j on its z-column in registers; the x- and y-derivatives of p and
//   w_d = sum_i (J^-1)_{d i} v_i go through shared memory; a term that is
//   reduced is formed directly on the smaller Gauss set with the projected
//   derivative P_2 D (tcki_derivative_project), the final prolongations
//   contract z in registers and x, y through shared memory; the n-point sum
//   stays in registers, the smaller levels' sums in shared memory.  The
//   rounding differs from the column form's (other products, other order),
//   the arithmetic is the same in exact arithmetic.
#pragma once

#include "tckc.cuh"

namespace dg {

// tile strides of an m-point set (interleaved words): odd row strides keep
// the EPB-word groups of consecutive lines in distinct banks
__host__ __device__ constexpr int tcki_P(int m) {
  return m == 4 ? 5 : (m == 6 ? 7 : (m == 8 ? 9 : m));
}
__host__ __device__ constexpr int tcki_Q(int m) {
  return m == 2 ? 6 : (m == 3 ? 11 : (m == 4 ? 22 : (m == 6 ? 42 : (m == 8 ? 73 : tcki_P(m) * m))));
}
// elements per block
__host__ __device__ constexpr int tcki_epb(int n) { return n <= 6 ? 8 : 4; }
// per-element stride of the staging area (Reals): the element's 4 n^3 values,
// padded so that the stride is an odd multiple of G = 32 / EPB banks (mod 32):
// the EPB elements' groups of G consecutive column words then fall in
// distinct banks.  A multiple of 4, so every slot starts 16-byte aligned.
__host__ __device__ constexpr int tcki_stage_from(int s, int g) { return s % (2 * g) == g ? s : tcki_stage_from(s + 4, g); }
__host__ __device__ constexpr int tcki_stage(int n) { return tcki_stage_from(4 * n * n * n, 32 / tcki_epb(n)); }

template <int N, int RED>
struct TckiShape {
  static constexpr int EPB = tcki_epb(N);
  static constexpr int FT = tcki_Q(N) * N;  // field stride of the line buffers (words)
  static constexpr int NL = tck_level_count<N, RED>();
  static constexpr int ACC = 10 * FT;        // accumulators of levels 1 .. NL-1, [4][m^3] each
  static constexpr int SEW = ACC + tck_acc_off<N, RED>(NL) - 4 * N * N * N;  // words per element
  static constexpr int SL = tcki_stage(N);
  static constexpr int WORDS = (SEW > SL ? SEW : SL) * EPB;  // Reals per block
  static constexpr int acc_off(int l) { return ACC + tck_acc_off<N, RED>(l) - 4 * N * N * N; }
};

// This thread's view of the block: element slot le, item t.
template <typename Real, int EPB>
struct TckiCtx {
  Real* sm;     // the block's shared memory
  int le, t;
  bool act;     // le < ne
  Real gk[11];  // (J^-1)_{d i} at gk[3 d + i], -rho c^2, -1/rho
  __device__ __forceinline__ Real& at(int o) const { return sm[o * EPB + le]; }
};

__device__ __forceinline__ void bulk_copy_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit_group() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// T_j = -S T_{j-1} at the M-point set (affine, constant coefficients).
template <int N, typename Real, int RED, int M>
__device__ __forceinline__ void tcki_derivative(Real (&c)[4][N], const TckiCtx<Real, TckiShape<N, RED>::EPB>& x) {
  using SH = TckiShape<N, RED>;
  constexpr int P = tcki_P(M), Q = tcki_Q(M), FT = SH::FT;
  constexpr int A = 0, BX = 3 * FT, BY = 5 * FT;  // p, w_x, w_y | d_x p, d_x w_x | d_y p, d_y w_y
  const bool on = x.act && x.t < M * M;
  const int a = x.t % M, b = x.t / M;
  const int cb = a + P * b;  // column (x, y) = (a, b)
  Real zc[2][M];
  if (on) {
    Real p[M], w2[M];
#pragma unroll
    for (int z = 0; z < M; ++z) {
      const Real v0 = c[1][z], v1 = c[2][z], v2 = c[3][z];
      p[z] = c[0][z];
      x.at(A + cb + Q * z) = p[z];
      x.at(A + FT + cb + Q * z) = fma(x.gk[0], v0, fma(x.gk[1], v1, x.gk[2] * v2));
      x.at(A + 2 * FT + cb + Q * z) = fma(x.gk[3], v0, fma(x.gk[4], v1, x.gk[5] * v2));
      w2[z] = fma(x.gk[6], v0, fma(x.gk[7], v1, x.gk[8] * v2));
    }
    mv<Real, OFF_D(M), M, M>(p, zc[0]);
    mv<Real, OFF_D(M), M, M>(w2, zc[1]);
  }
  __syncthreads();
  if (on) {
    const int xb = P * a + Q * b;  // x-line (y, z) = (a, b)
    const int yb = a + Q * b;      // y-line (x, z) = (a, b)
    Real q[2][M], d[2][M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
      q[0][s] = x.at(A + xb + s);
      q[1][s] = x.at(A + FT + xb + s);
    }
    mv<Real, OFF_D(M), M, M>(q[0], d[0]);
    mv<Real, OFF_D(M), M, M>(q[1], d[1]);
#pragma unroll
    for (int s = 0; s < M; ++s) {
      x.at(BX + xb + s) = d[0][s];
      x.at(BX + FT + xb + s) = d[1][s];
    }
#pragma unroll
    for (int s = 0; s < M; ++s) {
      q[0][s] = x.at(A + yb + P * s);
      q[1][s] = x.at(A + 2 * FT + yb + P * s);
    }
    mv<Real, OFF_D(M), M, M>(q[0], d[0]);
    mv<Real, OFF_D(M), M, M>(q[1], d[1]);
#pragma unroll
    for (int s = 0; s < M; ++s) {
      x.at(BY + yb + P * s) = d[0][s];
      x.at(BY + FT + yb + P * s) = d[1][s];
    }
  }
  __syncthreads();
  if (on) {
#pragma unroll
    for (int z = 0; z < M; ++z) {
      const int i = cb + Q * z;
      const Real dxp = x.at(BX + i), dxw = x.at(BX + FT + i), dyp = x.at(BY + i), dyw = x.at(BY + FT + i);
      c[0][z] = x.gk[9] * (dxw + dyw + zc[1][z]);
      c[1][z] = x.gk[10] * fma(x.gk[0], dxp, fma(x.gk[3], dyp, x.gk[6] * zc[0][z]));
      c[2][z] = x.gk[10] * fma(x.gk[1], dxp, fma(x.gk[4], dyp, x.gk[7] * zc[0][z]));
      c[3][z] = x.gk[10] * fma(x.gk[2], dxp, fma(x.gk[5], dyp, x.gk[8] * zc[0][z]));
    }
  }
}

// Reference L2 projection M -> MR (Sec. 3.3) of the column registers; on
// return the owners of the MR-point columns (t < MR^2) hold them.
template <int N, typename Real, int RED, int M, int MR>
__device__ __forceinline__ void tcki_project(Real (&c)[4][N], const TckiCtx<Real, TckiShape<N, RED>::EPB>& x) {
  using SH = TckiShape<N, RED>;
  constexpr int P = tcki_P(M), Q = tcki_Q(M), PR = tcki_P(MR), QR = tcki_Q(MR), FT = SH::FT;
  constexpr int OFF = OFF_PR(M, M - MR);  // MR x M
  constexpr int S1 = 0, S2 = 4 * FT;
  if (x.act && x.t < M * M) {  // z, in registers
    const int cb = x.t % M + P * (x.t / M);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      Real o[MR];
      mv<Real, OFF, MR, M>(c[f], o);
#pragma unroll
      for (int z = 0; z < MR; ++z) x.at(S1 + f * FT + cb + Q * z) = o[z];
    }
  }
  __syncthreads();
  if (x.act && x.t < M * MR) {  // x-lines (y, z), y < M, z < MR
    const int base = P * (x.t % M) + Q * (x.t / M);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      Real in[M], o[MR];
#pragma unroll
      for (int s = 0; s < M; ++s) in[s] = x.at(S1 + f * FT + base + s);
      mv<Real, OFF, MR, M>(in, o);
#pragma unroll
      for (int s = 0; s < MR; ++s) x.at(S2 + f * FT + base + s) = o[s];
    }
  }
  __syncthreads();
  if (x.act && x.t < MR * MR) {  // y-lines (x, z), x, z < MR; written in the MR-point layout
    const int xx = x.t % MR, zz = x.t / MR;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      Real in[M], o[MR];
#pragma unroll
      for (int s = 0; s < M; ++s) in[s] = x.at(S2 + f * FT + xx + P * s + Q * zz);
      mv<Real, OFF, MR, M>(in, o);
#pragma unroll
      for (int s = 0; s < MR; ++s) x.at(S1 + f * FT + xx + PR * s + QR * zz) = o[s];
    }
  }
  __syncthreads();
  if (x.act && x.t < MR * MR) {  // the new column owners read their columns
    const int cb = x.t % MR + PR * (x.t / MR);
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int z = 0; z < MR; ++z) c[f][z] = x.at(S1 + f * FT + cb + QR * z);
  }
}

// T_j = P (-S T_{j-1}) from the M-point set straight to the MR = M - 2
// point set, for a Taylor term that is reduced (Sec. 3.3): on an affine
// element with constant coefficients the projection P = P_x P_y P_z commutes
// with the coefficients, so every derivative term is one tensor product of
// the 1D matrices P_2 and P_2 D (the projected derivative, table PD2):
//   P grad p = ((P_2D)_x P_y P_z p, P_x (P_2D)_y P_z p, P_x P_y (P_2D)_z p),
//   P div_ref w = (P_2D)_x P_y P_z w_x + P_x (P_2D)_y P_z w_y + P_x P_y (P_2D)_z w_z.
// z is contracted by the M-point column owners in registers, x and y through
// shared memory, as in a derivative; the unreduced term at M points is never
// formed, and the separate projection pass goes away.
template <int N, typename Real, int RED, int M, int MR>
__device__ __forceinline__ void tcki_derivative_project(Real (&c)[4][N],
                                                        const TckiCtx<Real, TckiShape<N, RED>::EPB>& x) {
  using SH = TckiShape<N, RED>;
  constexpr int P = tcki_P(M), Q = tcki_Q(M), PR = tcki_P(MR), QR = tcki_Q(MR), FT = SH::FT;
  constexpr int PJ = OFF_PR(M, M - MR), PDJ = OFF_PD2(M);  // MR x M each
  constexpr int S = 0, T = 5 * FT, U = 0;  // S: 5 z-contracted fields; T: 5 after x; U: 4 results (S reused)
  static_assert(M - MR == 2, "the projected derivative is tabulated for reduction by 2");
  if (x.act && x.t < M * M) {  // z, by the M-point column owners
    const int cb = x.t % M + P * (x.t / M);
    Real p[M], wx[M], wy[M], wz[M];
#pragma unroll
    for (int z = 0; z < M; ++z) {
      const Real v0 = c[1][z], v1 = c[2][z], v2 = c[3][z];
      p[z] = c[0][z];
      wx[z] = fma(x.gk[0], v0, fma(x.gk[1], v1, x.gk[2] * v2));
      wy[z] = fma(x.gk[3], v0, fma(x.gk[4], v1, x.gk[5] * v2));
      wz[z] = fma(x.gk[6], v0, fma(x.gk[7], v1, x.gk[8] * v2));
    }
    Real o[5][MR];
    mv<Real, PJ, MR, M>(p, o[0]);    // P_z p
    mv<Real, PDJ, MR, M>(p, o[1]);   // (P_2D)_z p
    mv<Real, PJ, MR, M>(wx, o[2]);   // P_z w_x
    mv<Real, PJ, MR, M>(wy, o[3]);   // P_z w_y
    mv<Real, PDJ, MR, M>(wz, o[4]);  // (P_2D)_z w_z
#pragma unroll
    for (int f = 0; f < 5; ++f)
#pragma unroll
      for (int z = 0; z < MR; ++z) x.at(S + f * FT + cb + Q * z) = o[f][z];
  }
  __syncthreads();
  if (x.act && x.t < M * MR) {  // x-lines (y, z), y < M, z < MR
    const int base = P * (x.t % M) + Q * (x.t / M);
    Real in[M], a[MR], b[MR];
#pragma unroll
    for (int s = 0; s < M; ++s) in[s] = x.at(S + base + s);  // P_z p
    mv<Real, PJ, MR, M>(in, a);
    mv<Real, PDJ, MR, M>(in, b);
#pragma unroll
    for (int s = 0; s < MR; ++s) {
      x.at(T + base + s) = a[s];       // P_x P_z p
      x.at(T + FT + base + s) = b[s];  // (P_2D)_x P_z p
    }
#pragma unroll
    for (int s = 0; s < M; ++s) in[s] = x.at(S + FT + base + s);  // (P_2D)_z p
    mv<Real, PJ, MR, M>(in, a);
#pragma unroll
    for (int s = 0; s < MR; ++s) x.at(T + 2 * FT + base + s) = a[s];  // P_x (P_2D)_z p
#pragma unroll
    for (int s = 0; s < M; ++s) in[s] = x.at(S + 2 * FT + base + s);  // P_z w_x
    mv<Real, PDJ, MR, M>(in, a);
#pragma unroll
    for (int s = 0; s < M; ++s) in[s] = x.at(S + 4 * FT + base + s);  // (P_2D)_z w_z
    mv<Real, PJ, MR, M>(in, b);
#pragma unroll
    for (int s = 0; s < MR; ++s) x.at(T + 3 * FT + base + s) = a[s] + b[s];  // the x and z divergence terms
#pragma unroll
    for (int s = 0; s < M; ++s) in[s] = x.at(S + 3 * FT + base + s);  // P_z w_y
    mv<Real, PJ, MR, M>(in, a);
#pragma unroll
    for (int s = 0; s < MR; ++s) x.at(T + 4 * FT + base + s) = a[s];  // P_x P_z w_y
  }
  __syncthreads();
  if (x.act && x.t < MR * MR) {  // y-lines (x, z), x, z < MR; written in the MR-point layout
    const int xx = x.t % MR, zz = x.t / MR;
    const int base = xx + Q * zz;
    Real in[M], a[MR], b[MR], d[4][MR];
#pragma unroll
    for (int s = 0; s < M; ++s) in[s] = x.at(T + FT + base + P * s);
    mv<Real, PJ, MR, M>(in, d[0]);  // d/dx
#pragma unroll
    for (int s = 0; s < M; ++s) in[s] = x.at(T + base + P * s);
    mv<Real, PDJ, MR, M>(in, d[1]);  // d/dy
#pragma unroll
    for (int s = 0; s < M; ++s) in[s] = x.at(T + 2 * FT + base + P * s);
    mv<Real, PJ, MR, M>(in, d[2]);  // d/dz
#pragma unroll
    for (int s = 0; s < M; ++s) in[s] = x.at(T + 3 * FT + base + P * s);
    mv<Real, PJ, MR, M>(in, a);
#pragma unroll
    for (int s = 0; s < M; ++s) in[s] = x.at(T + 4 * FT + base + P * s);
    mv<Real, PDJ, MR, M>(in, b);
#pragma unroll
    for (int s = 0; s < MR; ++s) d[3][s] = a[s] + b[s];  // projected reference divergence
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int s = 0; s < MR; ++s) x.at(U + f * FT + xx + PR * s + QR * zz) = d[f][s];
  }
  __syncthreads();
  if (x.act && x.t < MR * MR) {  // the MR-point column owners apply the coefficients
    const int cb = x.t % MR + PR * (x.t / MR);
#pragma unroll
    for (int z = 0; z < MR; ++z) {
      const int i = cb + QR * z;
      const Real gx = x.at(U + i), gy = x.at(U + FT + i), gz = x.at(U + 2 * FT + i), q = x.at(U + 3 * FT + i);
      c[0][z] = x.gk[9] * q;
      c[1][z] = x.gk[10] * fma(x.gk[0], gx, fma(x.gk[3], gy, x.gk[6] * gz));
      c[2][z] = x.gk[10] * fma(x.gk[1], gx, fma(x.gk[4], gy, x.gk[7] * gz));
      c[3][z] = x.gk[10] * fma(x.gk[2], gx, fma(x.gk[5], gy, x.gk[8] * gz));
    }
  }
  __syncthreads();  // the next derivative writes the fields read above
}

// acc(level L) += cj T (or = cj T when FIRST), by the owners of the M-point columns
template <int N, typename Real, int RED, int L, int M, bool FIRST>
__device__ __forceinline__ void tcki_accumulate(const Real (&c)[4][N], Real (&acc)[4][N],
                                                const TckiCtx<Real, TckiShape<N, RED>::EPB>& x, Real cj) {
  if (!(x.act && x.t < M * M)) return;
  if constexpr (L == 0) {
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int z = 0; z < M; ++z) acc[f][z] = fma(cj, c[f][z], acc[f][z]);
  } else {
    constexpr int M3 = M * M * M;
    constexpr int AO = TckiShape<N, RED>::acc_off(L);
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int z = 0; z < M; ++z) {
        Real& q = x.at(AO + f * M3 + x.t + M * M * z);
        q = FIRST ? cj * c[f][z] : fma(cj, c[f][z], q);
      }
  }
}

// Taylor terms J .. N; M: points of the set T_{J-1} lives on
template <int N, typename Real, int RED, int J, int M>
__device__ __forceinline__ void tcki_steps(Real (&c)[4][N], Real (&acc)[4][N],
                                           const TckiCtx<Real, TckiShape<N, RED>::EPB>& x, const TckParams& p) {
  if constexpr (J <= N && M >= 2) {  // at M = 1 the derivative of a constant vanishes: so does every later term
    const Real cj = (Real)p.coef[J];
    if constexpr (RED > 0 && J % RED == 0) {
      if constexpr (M - RED >= 1) {  // else projected to a negative degree: T_J = 0, stop
        tcki_derivative_project<N, Real, RED, M, M - RED>(c, x);
        tcki_accumulate<N, Real, RED, J / RED, M - RED, true>(c, acc, x, cj);
        tcki_steps<N, Real, RED, J + 1, M - RED>(c, acc, x, p);
      }
    } else {
      tcki_derivative<N, Real, RED, M>(c, x);
      constexpr int L = RED > 0 ? (N - M) / RED : 0;
      tcki_accumulate<N, Real, RED, L, M, false>(c, acc, x, cj);
      tcki_steps<N, Real, RED, J + 1, M>(c, acc, x, p);
    }
  }
}

// acc(level L - 1) += I(M -> M + RED) acc(level L): x, y through shared
// memory, z in the registers of the (M + RED)-point column owners.
template <int N, typename Real, int RED, int L>
__device__ __forceinline__ void tcki_fold(Real (&acc)[4][N], const TckiCtx<Real, TckiShape<N, RED>::EPB>& x) {
  using SH = TckiShape<N, RED>;
  constexpr int M = N - RED * L, B = M + RED;
  constexpr int M2 = M * M, M3 = M2 * M;
  constexpr int PB = tcki_P(B), QB = tcki_Q(B), FT = SH::FT;
  constexpr int OFF = OFF_IR(B, RED);  // B x M
  constexpr int SRC = SH::acc_off(L), S1 = 0, S2 = 4 * FT;
  if (x.act && x.t < M2) {  // x-lines (y, z) of the compact M^3 sums
    const int y = x.t % M, z = x.t / M;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      Real in[M], o[B];
#pragma unroll
      for (int s = 0; s < M; ++s) in[s] = x.at(SRC + f * M3 + s + M * y + M2 * z);
      mv<Real, OFF, B, M>(in, o);
#pragma unroll
      for (int s = 0; s < B; ++s) x.at(S1 + f * FT + s + PB * y + QB * z) = o[s];
    }
  }
  __syncthreads();
  if (x.act && x.t < B * M) {  // y-lines (x, z), x < B, z < M
    const int xx = x.t % B, z = x.t / B;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      Real in[M], o[B];
#pragma unroll
      for (int s = 0; s < M; ++s) in[s] = x.at(S1 + f * FT + xx + PB * s + QB * z);
      mv<Real, OFF, B, M>(in, o);
#pragma unroll
      for (int s = 0; s < B; ++s) x.at(S2 + f * FT + xx + PB * s + QB * z) = o[s];
    }
  }
  __syncthreads();
  if (x.act && x.t < B * B) {  // z, by the B-point column owners
    const int cb = x.t % B + PB * (x.t / B);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      Real in[M], o[B];
#pragma unroll
      for (int s = 0; s < M; ++s) in[s] = x.at(S2 + f * FT + cb + QB * s);
      mv<Real, OFF, B, M>(in, o);
      if constexpr (L == 1) {
#pragma unroll
        for (int z = 0; z < B; ++z) acc[f][z] += o[z];
      } else {
        constexpr int DST = SH::acc_off(L - 1);
#pragma unroll
        for (int z = 0; z < B; ++z) x.at(DST + f * B * B * B + x.t + B * B * z) += o[z];
      }
    }
  }
  __syncthreads();
  if constexpr (L > 1) tcki_fold<N, Real, RED, L - 1>(acc, x);
}

// The predictor for elements e0 .. e0+ne-1 (ne <= EPB).
template <int N, typename Real, int RED>
__device__ __forceinline__ void tcki_block(const TckParams& p, const int e0, const int ne, Real* sm) {
  using SH = TckiShape<N, RED>;
  constexpr int EPB = SH::EPB, N2 = N * N, N3 = N2 * N, SL = SH::SL;
  constexpr uint32_t EB = 4 * N3 * sizeof(Real);  // bytes of one element's state
  __shared__ __align__(8) uint64_t bar;
  TckiCtx<Real, EPB> x;
  x.sm = sm;
  x.le = threadIdx.x % EPB;
  x.t = threadIdx.x / EPB;
  x.act = x.le < ne;
  const Real* __restrict__ U = static_cast<const Real*>(p.U) + (size_t)e0 * 4 * N3;
  Real* __restrict__ Ubar = static_cast<Real*>(p.Ubar) + (size_t)e0 * 4 * N3;
  // the block's states, one bulk copy per element into the staging slots
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, ne * EB);
    for (int l = 0; l < ne; ++l) bulk_copy_g2s(sm + l * SL, U + (size_t)l * 4 * N3, EB, &bar);
  }
  if (x.act) {
    const Real* gk = static_cast<const Real*>(p.geoKT) + (size_t)(e0 + x.le) * DG_AFF_TCK;
#pragma unroll
    for (int i = 0; i < 11; ++i) x.gk[i] = __ldg(gk + i);
  }
  // every thread takes the same branch below (it holds barriers)
  const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, 0, p.err) ? 1 : 0) != 0;
  Real c[4][N], acc[4][N];
  const Real c0 = (Real)p.coef[0];
  if (x.act && x.t < N2) {
    const Real* st = sm + x.le * SL;
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int z = 0; z < N; ++z) {
        c[f][z] = st[f * N3 + x.t + N2 * z];
        acc[f][z] = c0 * c[f][z];
      }
  }
  __syncthreads();  // the staging area is reused by the work buffers
  if (ok) {
    tcki_steps<N, Real, RED, 1, N>(c, acc, x, p);
    if constexpr (SH::NL > 1) {
      __syncthreads();
      tcki_fold<N, Real, RED, SH::NL - 1>(acc, x);
    }
  }
  __syncthreads();
  if (ok && x.act && x.t < N2) {
    Real* st = sm + x.le * SL;
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int z = 0; z < N; ++z) st[f * N3 + x.t + N2 * z] = acc[f][z];
    fence_proxy_async_shared();  // the bulk stores read what these stores wrote
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (ok) {
      for (int l = 0; l < ne; ++l) bulk_copy_s2g(Ubar + (size_t)l * 4 * N3, sm + l * SL, EB);
      bulk_commit_group();
      bulk_wait_read_all();  // the shared memory stays valid until the copies have read it
    }
    mbar_inval(&bar);
  }
}

// Blocks per SM the register budget is sized for (occupancy is what hides the
// phases' barriers: at a reduced Gauss set most of a block's warps wait).
// (chosen where the bound costs no spills)
__host__ __device__ constexpr int tcki_min_blocks(int n, int red) {
  return n <= 4 ? 6 : (n == 5 ? (red == 2 ? 4 : 3) : 2);
}

template <int N, typename Real, int RED>
__global__ void __launch_bounds__(tcki_epb(N) * N * N, tcki_min_blocks(N, RED)) tcki_kernel(const TckParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int EPB = TckiShape<N, RED>::EPB;
  const int e0 = blockIdx.x * EPB;
  tcki_block<N, Real, RED>(p, e0, min(EPB, p.E - e0), reinterpret_cast<Real*>(smem_raw));
}

template <int N, typename Real, int RED>
cudaError_t launch_tcki_red(const TckParams& p, cudaStream_t st) {
  constexpr int EPB = TckiShape<N, RED>::EPB;
  const int blocks = (p.E + EPB - 1) / EPB;
  const size_t smem = (size_t)TckiShape<N, RED>::WORDS * sizeof(Real);
  tcki_kernel<N, Real, RED><<<blocks, EPB * N * N, smem, st>>>(p);
  return cudaGetLastError();
}

// Reduction every 0 or 2 derivatives; affine Gauss-point states only.
template <int N, typename Real>
cudaError_t launch_tcki(const TckParams& p, int red, int epb, cudaStream_t st) {
  (void)epb;  // fixed by the layout: tcki_epb(N)
  if (!p.gmode || !p.aff || p.W) return cudaErrorInvalidValue;
  if (red == 2) return launch_tcki_red<N, Real, 2>(p, st);
  if (red == 0) return launch_tcki_red<N, Real, 0>(p, st);
  return cudaErrorInvalidValue;
}

template <int N, typename Real>
cudaError_t tcki_allow_smem() {
  cudaError_t e;
  if ((e = allow_smem(tcki_kernel<N, Real, 0>)) != cudaSuccess) return e;
  return allow_smem(tcki_kernel<N, Real, 2>);
}

template <int N, typename Real>
void register_tcki_one(KernelTable* t) {
  const int pi = sizeof(Real) == 8 ? 0 : 1;
  t->tcki[pi][N] = &launch_tcki<N, Real>;
}

}  // namespace dg
