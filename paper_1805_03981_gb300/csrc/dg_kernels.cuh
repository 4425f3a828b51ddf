// Device kernels of the matrix-free DG acoustic solver (sm_103a).
//
// Work decomposition: a thread block owns EPB consecutive elements and gives
// each element (k+1)^2 threads.  Sum-factorised 1D contractions (Sec. 3,
// "tensor product kernel") are done by letting every thread own one line of
// the element tile along the contraction direction: it loads the line from
// shared memory into registers, multiplies by the 1D matrix whose entries
// sit in constant memory (uniform across the warp), and writes the line back.
// Line ownership rotates between directions through shared memory.
//
// Tile index convention: node (x, y, z) of an n^3 tile is x + n y + n^2 z.
// A thread with in-element index t = a + n b owns
//   direction 0 (x): the line (y, z) = (a, b)
//   direction 1 (y): the line (x, z) = (a, b)
//   direction 2 (z): the line (x, y) = (a, b)
// and in each case (a, b) are also the face-point indices (i, j) of the two
// faces normal to that direction.  Per-point geometry used in a direction-d
// phase is stored "line-major": point (line t, position s) at t + n^2 s, so
// that a warp's loads are contiguous.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "tables.h"

// Each translation unit has its own copy of the constant tables (no
// relocatable device code); the upload_* function of each kernel
// instantiation unit fills it.
static __constant__ double c_tab_d[DG_TAB_LEN];
static __constant__ float c_tab_f[DG_TAB_LEN];


namespace dg {

// Operator epilogues.  EPI_LSRK: a stage of the 2N-storage scheme (register
// dU).  EPI_LSRK2R: a stage of a two-register scheme (Sec. 2.2, LSRK4(5) and
// LSRK5(9)): with S the running sum (read from Uadd, written to dU) the
// stage writes the next stage input S + cA R (out; skipped in the last
// stage) and S + cB R, with cA = dt A_i and cB = dt B_i.
enum { EPI_WRITE = 0, EPI_LSRK = 1, EPI_ADD = 2, EPI_LSRK2R = 3 };

template <typename Real>
__device__ __forceinline__ Real tab(int i);
template <>
__device__ __forceinline__ double tab<double>(int i) { return c_tab_d[i]; }
template <>
__device__ __forceinline__ float tab<float>(int i) { return c_tab_f[i]; }

// ---- bulk asynchronous copies global -> shared, completed on an mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// size and both addresses must be multiples of 16 bytes
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of the barrier, giving up after a bounded number of
// polls: then the error flag is set, a second bounded wait lets the block's
// own copies land, and false is returned.  The second limit is the same 2^22
// polls, far longer than the largest copy a block issues (a few tens of KB).
// expire_first (a test setting, OpParams::expire_wait) makes the first wait
// give up at once, so that the give-up path runs without a real hang; the
// second wait still drains the copies before the block returns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err,
                                                  bool expire_first = false) {
  const int first_limit = expire_first ? 0 : (1 << 22);
  for (int i = 0; i < first_limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  if (err) atomicExch(err, 2);
  for (int i = 0; i < (1 << 22); ++i)
    if (mbar_try_wait(bar, parity)) break;
  return false;
}

// out = M in for a centrosymmetric (SKEW = false) or skew-centrosymmetric
// (SKEW = true) N x N matrix M, in the even-odd form stored at EO (tables.h):
// e_j = in_j + in_{N-1-j}, o_j = in_j - in_{N-1-j} (j < N/2), p = A e (+ C in_mid),
// q = B o, out_i = p_i + q_i, out_{N-1-i} = p_i - q_i (skew: q_i - p_i).
// About N^2/2 + 2N operations instead of N^2 (the C_tensorial count of
// Sec. 4.1).
template <typename Real, int EO, int N, bool SKEW>
__device__ __forceinline__ void mv_eo(const Real* in, Real* out) {
  constexpr int H = N / 2;
  constexpr bool ODD = (N & 1) != 0;
  constexpr int A = EO, B = EO + (H + 1) * H, C = EO + 2 * (H + 1) * H;
  Real e[H], o[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = in[j] + in[N - 1 - j];
    o[j] = in[j] - in[N - 1 - j];
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    Real p = tab<Real>(A + i * H) * e[0];
#pragma unroll
    for (int j = 1; j < H; ++j) p = fma(tab<Real>(A + i * H + j), e[j], p);
    if constexpr (ODD) p = fma(tab<Real>(C + i), in[H], p);
    Real q = tab<Real>(B + i * H) * o[0];
#pragma unroll
    for (int j = 1; j < H; ++j) q = fma(tab<Real>(B + i * H + j), o[j], q);
    out[i] = p + q;
    out[N - 1 - i] = SKEW ? q - p : p - q;
  }
  if constexpr (ODD) {
    if constexpr (SKEW) {  // the middle row of a skew matrix is odd: only o contributes
      Real q = tab<Real>(B + H * H) * o[0];
#pragma unroll
      for (int j = 1; j < H; ++j) q = fma(tab<Real>(B + H * H + j), o[j], q);
      out[H] = q;
    } else {  // the middle row of a centrosymmetric matrix is even
      Real p = tab<Real>(A + H * H) * e[0];
#pragma unroll
      for (int j = 1; j < H; ++j) p = fma(tab<Real>(A + H * H + j), e[j], p);
      out[H] = fma(tab<Real>(C + H), in[H], p);
    }
  }
}

// out[i] = sum_j M[i][j] in[j];  M is RO x RI at table offset OFF.  The
// square basis changes V, VI and the collocation derivative D of n >= 5
// points take the even-odd form (fewer operations); every kernel applies
// them through this one routine, so all paths round alike.
template <typename Real, int OFF, int RO, int RI>
__device__ __forceinline__ void mv(const Real* in, Real* out) {
  if constexpr (RO == RI && RI >= 5 && OFF == OFF_V(RI)) {
    mv_eo<Real, OFF_EO(RI, 0), RI, false>(in, out);
  } else if constexpr (RO == RI && RI >= 5 && OFF == OFF_VI(RI)) {
    mv_eo<Real, OFF_EO(RI, 1), RI, false>(in, out);
  } else if constexpr (RO == RI && RI >= 5 && OFF == OFF_D(RI)) {
    mv_eo<Real, OFF_EO(RI, 2), RI, true>(in, out);
  } else {
#pragma unroll
    for (int i = 0; i < RO; ++i) {
      Real acc = tab<Real>(OFF + i * RI) * in[0];
#pragma unroll
      for (int j = 1; j < RI; ++j) acc = fma(tab<Real>(OFF + i * RI + j), in[j], acc);
      out[i] = acc;
    }
  }
}

// out[j] = sum_i M[i][j] in[i];  M is RI x RO at table offset OFF (transpose).
template <typename Real, int OFF, int RI, int RO>
__device__ __forceinline__ void mtv(const Real* in, Real* out) {
#pragma unroll
  for (int j = 0; j < RO; ++j) {
    Real acc = tab<Real>(OFF + j) * in[0];
#pragma unroll
    for (int i = 1; i < RI; ++i) acc = fma(tab<Real>(OFF + i * RO + j), in[i], acc);
    out[j] = acc;
  }
}

// out[j] += sum_i M[i][j] in[i]  (accumulating transpose: an FMA chain that
// starts from the running sum)
template <typename Real, int OFF, int RI, int RO>
__device__ __forceinline__ void mtv_acc(const Real* in, Real* out) {
#pragma unroll
  for (int j = 0; j < RO; ++j) {
    Real acc = out[j];
#pragma unroll
    for (int i = 0; i < RI; ++i) acc = fma(tab<Real>(OFF + i * RO + j), in[i], acc);
    out[j] = acc;
  }
}

// Base index and stride of the line (a, b) along DIR in an X x Y x Z tile.
template <int DIR, int X, int Y>
__device__ __forceinline__ int line_base(int a, int b) {
  return DIR == 0 ? X * a + X * Y * b : (DIR == 1 ? a + X * Y * b : a + X * b);
}
template <int DIR, int X, int Y>
__host__ __device__ constexpr int line_stride() {
  return DIR == 0 ? 1 : (DIR == 1 ? X : X * Y);
}

// Contract an X x Y x Z tile (4 fields, field stride FS_IN) along DIR with
// the RO x RI matrix at OFF (RI = extent along DIR), writing the result tile
// (extent RO along DIR, field stride FS_OUT) to dst.  contract_line does one
// line l of the tile.  dst may equal src only if RO == RI.
template <typename Real, int DIR, int X, int Y, int Z, int RO, int OFF, int FS_IN, int FS_OUT,
          bool ADD = false>
__device__ __forceinline__ void contract_line(const Real* src, Real* dst, int l, Real scale = Real(1)) {
  constexpr int RI = DIR == 0 ? X : (DIR == 1 ? Y : Z);
  constexpr int A = DIR == 0 ? Y : X;  // extent of the first line coordinate
  constexpr int OX = DIR == 0 ? RO : X, OY = DIR == 1 ? RO : Y;
  const int a = l % A, b = l / A;
  const int bi = line_base<DIR, X, Y>(a, b);
  const int bo = line_base<DIR, OX, OY>(a, b);
  constexpr int si = line_stride<DIR, X, Y>();
  constexpr int so = line_stride<DIR, OX, OY>();
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    Real in[RI], out[RO];
#pragma unroll
    for (int s = 0; s < RI; ++s) in[s] = src[f * FS_IN + bi + si * s];
    mv<Real, OFF, RO, RI>(in, out);
#pragma unroll
    for (int s = 0; s < RO; ++s) {
      if (ADD)
        dst[f * FS_OUT + bo + so * s] += scale * out[s];
      else
        dst[f * FS_OUT + bo + so * s] = out[s];
    }
  }
}

// The whole tile of one element: threads 0..nthr-1 of the element share the lines.
template <typename Real, int DIR, int X, int Y, int Z, int RO, int OFF, int FS_IN, int FS_OUT,
          bool ADD = false>
__device__ __forceinline__ void contract_tile(const Real* src, Real* dst, int t, int nthr,
                                              Real scale = Real(1)) {
  constexpr int A = DIR == 0 ? Y : X;
  constexpr int B = DIR == 2 ? Y : Z;  // extent of the second line coordinate
  for (int l = t; l < A * B; l += nthr)
    contract_line<Real, DIR, X, Y, Z, RO, OFF, FS_IN, FS_OUT, ADD>(src, dst, l, scale);
}

// The tiles of ne elements (element stride es in src and dst): the lines of
// all of them are spread over threads T = 0..nthr-1 of the block, so that a
// small tile keeps whole warps busy instead of a few lanes of every warp.
template <typename Real, int DIR, int X, int Y, int Z, int RO, int OFF, int FS_IN, int FS_OUT,
          bool ADD = false>
__device__ __forceinline__ void contract_tile_b(const Real* src0, Real* dst0, int es, int ne, int T,
                                                int nthr) {
  constexpr int A = DIR == 0 ? Y : X;
  constexpr int B = DIR == 2 ? Y : Z;
  for (int L = T; L < ne * A * B; L += nthr) {
    const int le = L / (A * B);
    contract_line<Real, DIR, X, Y, Z, RO, OFF, FS_IN, FS_OUT, ADD>(src0 + le * es, dst0 + le * es,
                                                                    L - le * (A * B));
  }
}

// ---------------------------------------------------------------------------
// Operator R = -M^-1 K U (Sec. 2.1, Eq. (3)) with fused epilogues.
// ---------------------------------------------------------------------------
struct OpParams {
  const void* U;      // input state, GL basis [E][4][n^3]
  void* out;          // WRITE: R; ADD / LSRK: updated state
  const void* Uadd;   // ADD / LSRK: state the update is added to
  void* dU;           // LSRK register
  double cA, cB, dt;  // LSRK: dU = cA dU + dt R (cA ignored if first), out = Uadd + cB dU
                      // LSRK2R: out = Uadd + cA R, dU = Uadd + cB R
  int first;          // LSRK: first stage (dU not read); LSRK2R: Uadd is the input U itself
  int last;           // LSRK2R: last stage (out not written)
  const int32_t* nbr;
  const int8_t* nbr_face;
  const int8_t* orient;
  const void* geoA;  // [E][3 d][3 i][n^3] line-major per d: w adj(J)_{d i}   (stride geo_stride_A)
  const void* geoM;  // [E][2][n^3]: rho c^2 / (w detJ), 1 / (rho w detJ)    (stride geo_stride_M)
  const void* geoF;  // [E][6 f][6][n^2]: nw_x, nw_y, nw_z, Z-/(Z-+Z+), b, c (stride geo_stride_F)
  const void* geoK;  // [E][DG_AFF_OP] compact data of affine elements (affine kernels only)
  int* err;          // set (non-zero) if a bounded wait gave up
  int E;
  int expire_wait;   // testing only: the first bounded wait gives up at once
};

template <int N>
__host__ __device__ constexpr int op_smem_per_elem() {
  return 8 * N * N * N + 24 * N * N;
}

// Cell and face contributions of the direction-DIR phase along the thread's
// line: cell test-gradient integration (the collocation derivative
// transposed applied to the contravariant fluxes) and the lifting of the
// two faces normal to DIR.  u: Gauss-point values of (p, v) on the line;
// r: contributions to the Gauss-basis residual along the line.
template <typename Real, bool SMEM>
__device__ __forceinline__ Real geo_ld(const Real* p) {
  if constexpr (SMEM)
    return *p;
  else
    return __ldg(p);
}

template <int N, typename Real, int DIR, bool ACC = false, bool SMEM = false>
__device__ __forceinline__ void cell_face_dir(const Real (&u)[4][N], Real (&r)[4][N],
                                              const Real* __restrict__ gA,
                                              const Real* __restrict__ gF, const Real* snb,
                                              int t, int fmask) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const Real* A0 = gA + (DIR * 3 + 0) * N3 + t;
  const Real* A1 = gA + (DIR * 3 + 1) * N3 + t;
  const Real* A2 = gA + (DIR * 3 + 2) * N3 + t;
  Real F[N];
  // pressure test: flux sum_i A_{DIR i} v_i
#pragma unroll
  for (int s = 0; s < N; ++s)
    F[s] = fma(geo_ld<Real, SMEM>(A0 + N2 * s), u[1][s],
               fma(geo_ld<Real, SMEM>(A1 + N2 * s), u[2][s], geo_ld<Real, SMEM>(A2 + N2 * s) * u[3][s]));
  if (ACC)
    mtv_acc<Real, OFF_D(N), N, N>(F, r[0]);
  else
    mtv<Real, OFF_D(N), N, N>(F, r[0]);
  // velocity tests: flux A_{DIR i} p
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const Real* Ai = i == 0 ? A0 : (i == 1 ? A1 : A2);
#pragma unroll
    for (int s = 0; s < N; ++s) F[s] = geo_ld<Real, SMEM>(Ai + N2 * s) * u[0][s];
    if (ACC)
      mtv_acc<Real, OFF_D(N), N, N>(F, r[1 + i]);
    else
      mtv<Real, OFF_D(N), N, N>(F, r[1 + i]);
  }
  // faces 2 DIR (xi_DIR = -1) and 2 DIR + 1 (xi_DIR = +1)
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const int f = 2 * DIR + sd;
    constexpr int LF = OFF_LF(N);
    Real um[4];
#pragma unroll
    for (int fl = 0; fl < 4; ++fl) {
      Real acc = tab<Real>(LF + sd * N) * u[fl][0];
#pragma unroll
      for (int s = 1; s < N; ++s) acc = fma(tab<Real>(LF + sd * N + s), u[fl][s], acc);
      um[fl] = acc;
    }
    const Real* fc = gF + f * 6 * N2 + t;
    const Real nw0 = geo_ld<Real, SMEM>(fc), nw1 = geo_ld<Real, SMEM>(fc + N2), nw2 = geo_ld<Real, SMEM>(fc + 2 * N2);
    const Real a2 = geo_ld<Real, SMEM>(fc + 3 * N2), bb = geo_ld<Real, SMEM>(fc + 4 * N2), cc = geo_ld<Real, SMEM>(fc + 5 * N2);
    const Real vnm = fma(nw0, um[1], fma(nw1, um[2], nw2 * um[3]));
    Real pp, vnp;
    if ((fmask >> f) & 1) {
      const Real* nb = snb + f * 4 * N2 + t;
      pp = nb[0];
      vnp = fma(nw0, nb[N2], fma(nw1, nb[2 * N2], nw2 * nb[3 * N2]));
    } else {  // reflecting wall: mirror state
      pp = um[0];
      vnp = -vnm;
    }
    const Real dp = um[0] - pp, dvn = vnm - vnp;
    const Real pstar = fma(-a2, dp, fma(bb, dvn, um[0]));  // p*
    const Real flp = fma(a2, dvn, fma(cc, dp, vnp));        // |J_f| w (v.n)*
    const Real g0 = nw0 * pstar, g1 = nw1 * pstar, g2 = nw2 * pstar;
#pragma unroll
    for (int s = 0; s < N; ++s) {
      const Real l = tab<Real>(LF + sd * N + s);
      r[0][s] = fma(-l, flp, r[0][s]);
      r[1][s] = fma(-l, g0, r[1][s]);
      r[2][s] = fma(-l, g1, r[2][s]);
      r[3][s] = fma(-l, g2, r[3][s]);
    }
  }
}

// One block's share of the operator: elements e0 .. e0+ne-1, (k+1)^2
// threads each (threads beyond ne (k+1)^2 only help with the flat copies).
// Every element's arithmetic is independent of e0, ne and the block shape.
template <int N, typename Real, int EPI>
__device__ __forceinline__ void op_block(const OpParams& p, const int e0, const int ne, Real* sm) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int SE = op_smem_per_elem<N>();
  const int le = threadIdx.x / N2, t = threadIdx.x - le * N2;
  const int a = t % N, b = t / N;
  const int e = e0 + le;
  const bool act = le < ne;
  Real* su = sm + le * SE;
  Real* sr = su + 4 * N3;
  Real* snb = sr + 4 * N3;
  const Real* __restrict__ U = static_cast<const Real*>(p.U);

  // 1. element tiles, contiguous in memory: flat coalesced copy
  for (int i = threadIdx.x; i < ne * 4 * N3; i += blockDim.x) {
    const int l = i / (4 * N3);
    sm[l * SE + (i - l * 4 * N3)] = U[(size_t)e0 * 4 * N3 + i];
  }
  // neighbours' GL face nodes, gathered into this element's face coordinates
  int fmask = 0;
  if (act) {
#pragma unroll 1
    for (int f = 0; f < 6; ++f) {
      const int en = p.nbr[e * 6 + f];
      if (en < 0) continue;
      fmask |= 1 << f;
      const int fn = p.nbr_face[e * 6 + f], o = p.orient[e * 6 + f];
      const int uu = (o & 1) ? b : a, vv = (o & 1) ? a : b;
      const int ip = (o & 2) ? N - 1 - uu : uu, jp = (o & 4) ? N - 1 - vv : vv;
      const int dn = fn >> 1;
      int crd[3];
      crd[dn] = (fn & 1) ? N - 1 : 0;
      crd[dn == 0 ? 1 : 0] = ip;
      crd[dn == 2 ? 1 : 2] = jp;
      const Real* src = U + (size_t)en * 4 * N3 + crd[0] + N * crd[1] + N2 * crd[2];
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) snb[(f * 4 + fl) * N2 + t] = src[fl * N3];
    }
  }
  __syncthreads();

  // 2. GL -> G (Sec. 3.1) along z of the tile and along the first tangential
  //    axis of the neighbour face data
  if (act) {
    contract_tile<Real, 2, N, N, N, N, OFF_V(N), N3, N3>(su, su, t, N2);
    for (int it = t; it < 6 * N; it += N2) {
      const int f = it / N, j = it - f * N;
      if (!((fmask >> f) & 1)) continue;
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        Real in[N], out[N];
        Real* q = snb + (f * 4 + fl) * N2 + N * j;
#pragma unroll
        for (int s = 0; s < N; ++s) in[s] = q[s];
        mv<Real, OFF_V(N), N, N>(in, out);
#pragma unroll
        for (int s = 0; s < N; ++s) q[s] = out[s];
      }
    }
  }
  __syncthreads();
  if (act) {
    contract_tile<Real, 0, N, N, N, N, OFF_V(N), N3, N3>(su, su, t, N2);
    for (int it = t; it < 6 * N; it += N2) {
      const int f = it / N, i = it - f * N;
      if (!((fmask >> f) & 1)) continue;
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        Real in[N], out[N];
        Real* q = snb + (f * 4 + fl) * N2 + i;
#pragma unroll
        for (int s = 0; s < N; ++s) in[s] = q[N * s];
        mv<Real, OFF_V(N), N, N>(in, out);
#pragma unroll
        for (int s = 0; s < N; ++s) q[N * s] = out[s];
      }
    }
  }
  __syncthreads();

  const Real* gA = static_cast<const Real*>(p.geoA) + (size_t)e * geo_stride_A(N);
  const Real* gF = static_cast<const Real*>(p.geoF) + (size_t)e * geo_stride_F(N);
  const Real* gM = static_cast<const Real*>(p.geoM) + (size_t)e * geo_stride_M(N);

  // 3. y: finish GL -> G along y in registers, then the y cell/face terms
  if (act) {
    Real u[4][N], r[4][N];
    const int base = line_base<1, N, N>(a, b);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl) {
      Real in[N];
#pragma unroll
      for (int s = 0; s < N; ++s) in[s] = su[fl * N3 + base + N * s];
      mv<Real, OFF_V(N), N, N>(in, u[fl]);
#pragma unroll
      for (int s = 0; s < N; ++s) su[fl * N3 + base + N * s] = u[fl][s];
    }
    cell_face_dir<N, Real, 1>(u, r, gA, gF, snb, t, fmask);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) sr[fl * N3 + base + N * s] = r[fl][s];
  }
  __syncthreads();
  // 4. x
  if (act) {
    Real u[4][N], r[4][N];
    const int base = line_base<0, N, N>(a, b);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) {
        u[fl][s] = su[fl * N3 + base + s];
        r[fl][s] = sr[fl * N3 + base + s];
      }
    cell_face_dir<N, Real, 0, true>(u, r, gA, gF, snb, t, fmask);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) sr[fl * N3 + base + s] = r[fl][s];
  }
  __syncthreads();
  // 5. z, then inverse mass (diagonal in G, Sec. 3.1) and G -> GL along z
  if (act) {
    Real u[4][N], r[4][N];
    const int base = line_base<2, N, N>(a, b);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) {
        u[fl][s] = su[fl * N3 + base + N2 * s];
        r[fl][s] = sr[fl * N3 + base + N2 * s];
      }
    cell_face_dir<N, Real, 2, true>(u, r, gA, gF, snb, t, fmask);
#pragma unroll
    for (int s = 0; s < N; ++s) {
      const Real mp = __ldg(gM + base + N2 * s), mvv = __ldg(gM + N3 + base + N2 * s);
      r[0][s] *= mp;
#pragma unroll
      for (int fl = 1; fl < 4; ++fl) r[fl][s] *= mvv;
    }
#pragma unroll
    for (int fl = 0; fl < 4; ++fl) {
      Real out[N];
      mv<Real, OFF_VI(N), N, N>(r[fl], out);
#pragma unroll
      for (int s = 0; s < N; ++s) sr[fl * N3 + base + N2 * s] = out[s];
    }
  }
  __syncthreads();
  if (act) contract_tile<Real, 0, N, N, N, N, OFF_VI(N), N3, N3>(sr, sr, t, N2);
  __syncthreads();
  if (act) contract_tile<Real, 1, N, N, N, N, OFF_VI(N), N3, N3>(sr, sr, t, N2);
  __syncthreads();

  // 6. epilogue, flat and coalesced over the block's elements
  Real* __restrict__ out = static_cast<Real*>(p.out);
  const Real* __restrict__ Uadd = static_cast<const Real*>(p.Uadd);
  Real* __restrict__ dU = static_cast<Real*>(p.dU);
  const Real cA = (Real)p.cA, cB = (Real)p.cB, dt = (Real)p.dt;
  for (int i = threadIdx.x; i < ne * 4 * N3; i += blockDim.x) {
    const int l = i / (4 * N3);
    const Real R = sm[l * SE + 4 * N3 + (i - l * 4 * N3)];
    const size_t g = (size_t)e0 * 4 * N3 + i;
    if (EPI == EPI_WRITE) {
      out[g] = R;
    } else if (EPI == EPI_ADD) {
      out[g] = Uadd[g] + R;
    } else if (EPI == EPI_LSRK2R) {
      const Real S = Uadd[g];
      if (!p.last) out[g] = fma(cA, R, S);
      dU[g] = fma(cB, R, S);
    } else {
      const Real d = p.first ? dt * R : fma(cA, dU[g], dt * R);
      dU[g] = d;
      out[g] = fma(cB, d, Uadd[g]);
    }
  }
}

template <int N, typename Real, int EPI>
__global__ void op_kernel(const OpParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int epb = blockDim.x / (N * N);
  const int e0 = blockIdx.x * epb;
  op_block<N, Real, EPI>(p, e0, min(epb, p.E - e0), reinterpret_cast<Real*>(smem_raw));
}

// ---------------------------------------------------------------------------
// The operator on states kept in the Gauss basis G (values at the (k+1)^3
// Gauss points): no basis change of the own tile, M^-1 is the diagonal alone,
// and a neighbour's trace at a face Gauss point is the l(+-1) contraction of
// the neighbour's line through that point.  Same discrete operator as
// op_block, other representation of the state (Sec. 3.1 weighs exactly this
// choice of basis against the face data it needs).
// ---------------------------------------------------------------------------
template <int N, typename Real, int EPI>
__device__ __forceinline__ void opg_block(const OpParams& p, const int e0, const int ne, Real* sm) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int SE = op_smem_per_elem<N>();
  const int le = threadIdx.x / N2, t = threadIdx.x - le * N2;
  const int a = t % N, b = t / N;
  const int e = e0 + le;
  const bool act = le < ne;
  Real* su = sm + le * SE;
  Real* sr = su + 4 * N3;
  Real* snb = sr + 4 * N3;
  const Real* __restrict__ U = static_cast<const Real*>(p.U);

  for (int i = threadIdx.x; i < ne * 4 * N3; i += blockDim.x) {
    const int l = i / (4 * N3);
    sm[l * SE + (i - l * 4 * N3)] = U[(size_t)e0 * 4 * N3 + i];
  }
  // neighbours' traces at this element's face Gauss points
  int fmask = 0;
  if (act) {
#pragma unroll 1
    for (int f = 0; f < 6; ++f) {
      const int en = p.nbr[e * 6 + f];
      if (en < 0) continue;
      fmask |= 1 << f;
      const int fn = p.nbr_face[e * 6 + f], o = p.orient[e * 6 + f];
      const int uu = (o & 1) ? b : a, vv = (o & 1) ? a : b;
      const int ip = (o & 2) ? N - 1 - uu : uu, jp = (o & 4) ? N - 1 - vv : vv;
      const int dn = fn >> 1, sd = fn & 1;
      const int t0 = dn == 0 ? 1 : 0, t1 = dn == 2 ? 1 : 2;
      const int stride[3] = {1, N, N2};
      const Real* src = U + (size_t)en * 4 * N3 + ip * stride[t0] + jp * stride[t1];
      const int st = stride[dn];
      constexpr int LF = OFF_LF(N);
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        Real acc = tab<Real>(LF + sd * N) * src[fl * N3];
#pragma unroll
        for (int s = 1; s < N; ++s) acc = fma(tab<Real>(LF + sd * N + s), src[fl * N3 + s * st], acc);
        snb[(f * 4 + fl) * N2 + t] = acc;
      }
    }
  }
  __syncthreads();
  const Real* gA = static_cast<const Real*>(p.geoA) + (size_t)e * geo_stride_A(N);
  const Real* gF = static_cast<const Real*>(p.geoF) + (size_t)e * geo_stride_F(N);
  const Real* gM = static_cast<const Real*>(p.geoM) + (size_t)e * geo_stride_M(N);
  if (act) {  // y
    Real u[4][N], r[4][N];
    const int base = line_base<1, N, N>(a, b);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) u[fl][s] = su[fl * N3 + base + N * s];
    cell_face_dir<N, Real, 1>(u, r, gA, gF, snb, t, fmask);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) sr[fl * N3 + base + N * s] = r[fl][s];
  }
  __syncthreads();
  if (act) {  // x
    Real u[4][N], r[4][N];
    const int base = line_base<0, N, N>(a, b);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) {
        u[fl][s] = su[fl * N3 + base + s];
        r[fl][s] = sr[fl * N3 + base + s];
      }
    cell_face_dir<N, Real, 0, true>(u, r, gA, gF, snb, t, fmask);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) sr[fl * N3 + base + s] = r[fl][s];
  }
  __syncthreads();
  if (act) {  // z, then the diagonal inverse mass
    Real u[4][N], r[4][N];
    const int base = line_base<2, N, N>(a, b);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) {
        u[fl][s] = su[fl * N3 + base + N2 * s];
        r[fl][s] = sr[fl * N3 + base + N2 * s];
      }
    cell_face_dir<N, Real, 2, true>(u, r, gA, gF, snb, t, fmask);
    // the residual of this z-line is final: the epilogue runs here, on the
    // line's points (contiguous across the warp), with no shared-memory pass
    Real* __restrict__ out = static_cast<Real*>(p.out);
    const Real* __restrict__ Uadd = static_cast<const Real*>(p.Uadd);
    Real* __restrict__ dU = static_cast<Real*>(p.dU);
    const Real cA = (Real)p.cA, cB = (Real)p.cB, dt = (Real)p.dt;
    const size_t g0 = (size_t)e * 4 * N3 + base;
#pragma unroll
    for (int s = 0; s < N; ++s) {
      const Real mp = __ldg(gM + base + N2 * s), mvv = __ldg(gM + N3 + base + N2 * s);
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        const Real R = r[fl][s] * (fl == 0 ? mp : mvv);
        const size_t g = g0 + fl * N3 + N2 * s;
        if (EPI == EPI_WRITE) {
          out[g] = R;
        } else if (EPI == EPI_ADD) {
          out[g] = Uadd[g] + R;
        } else if (EPI == EPI_LSRK2R) {
          const Real S = Uadd[g];
          if (!p.last) out[g] = fma(cA, R, S);
          dU[g] = fma(cB, R, S);
        } else {
          const Real d = p.first ? dt * R : fma(cA, dU[g], dt * R);
          dU[g] = d;
          out[g] = fma(cB, d, Uadd[g]);
        }
      }
    }
  }
}

// Shared-memory layout of the staged Gauss-basis operator, per block of epb
// elements: [U][R][neighbour traces][geoA][geoM][geoF][X], X = the LSRK
// register (or the state the ADER update adds to); every region 16-byte
// aligned.
template <int N>
__host__ __device__ constexpr int opgs_smem_per_elem() {
  return 4 * N * N * N * 3 + 24 * N * N + geo_stride_A(N) + geo_stride_M(N) + geo_stride_F(N);
}

// The Gauss-basis operator with its inputs staged: one thread issues bulk
// asynchronous copies of the block's elements (state, LSRK register or added
// state, cell metric, mass diagonal, face data; each a contiguous run in
// global memory) into shared memory, so the block's whole input is in flight
// at once; the phases then read shared memory.  Neighbour lines are still
// read from global memory (mostly L2 hits).
template <int N, typename Real, int EPI>
__device__ __forceinline__ void opgs_block(const OpParams& p, const int e0, const int ne, const int epb,
                                           Real* sm) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int GA = geo_stride_A(N), GM = geo_stride_M(N), GF = geo_stride_F(N);
  __shared__ __align__(8) uint64_t bar;
  const int le = threadIdx.x / N2, t = threadIdx.x - le * N2;
  const int a = t % N, b = t / N;
  const int e = e0 + le;
  const bool act = le < ne;
  Real* suA = sm;
  Real* srA = suA + epb * 4 * N3;
  Real* snA = srA + epb * 4 * N3;
  Real* gAA = snA + epb * 24 * N2;
  Real* gMA = gAA + epb * GA;
  Real* gFA = gMA + epb * GM;
  Real* sxA = gFA + epb * GF;
  const bool need_x = ((EPI == EPI_LSRK || EPI == EPI_LSRK2R) && !p.first) || EPI == EPI_ADD;
  const Real* __restrict__ U = static_cast<const Real*>(p.U);
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t sb = ne * 4 * N3 * sizeof(Real);
    const uint32_t tot = sb * (need_x ? 2 : 1) + ne * (GA + GM + GF) * sizeof(Real);
    mbar_expect_tx(&bar, tot);
    bulk_copy_g2s(suA, U + (size_t)e0 * 4 * N3, sb, &bar);
    bulk_copy_g2s(gAA, static_cast<const Real*>(p.geoA) + (size_t)e0 * GA, ne * GA * sizeof(Real), &bar);
    bulk_copy_g2s(gMA, static_cast<const Real*>(p.geoM) + (size_t)e0 * GM, ne * GM * sizeof(Real), &bar);
    bulk_copy_g2s(gFA, static_cast<const Real*>(p.geoF) + (size_t)e0 * GF, ne * GF * sizeof(Real), &bar);
    if (need_x) {
      const Real* X = EPI == EPI_LSRK ? static_cast<const Real*>(p.dU) : static_cast<const Real*>(p.Uadd);
      bulk_copy_g2s(sxA, X + (size_t)e0 * 4 * N3, sb, &bar);
    }
  }
  Real* su = suA + le * 4 * N3;
  Real* sr = srA + le * 4 * N3;
  Real* snb = snA + le * 24 * N2;
  // neighbours' traces from global memory while the copies are in flight
  int fmask = 0;
  if (act) {
    int en[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) en[f] = p.nbr[e * 6 + f];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      if (en[f] < 0) continue;
      fmask |= 1 << f;
      const int fn = p.nbr_face[e * 6 + f], o = p.orient[e * 6 + f];
      const int uu = (o & 1) ? b : a, vv = (o & 1) ? a : b;
      const int ip = (o & 2) ? N - 1 - uu : uu, jp = (o & 4) ? N - 1 - vv : vv;
      const int dn = fn >> 1, sd = fn & 1;
      const int t0 = dn == 0 ? 1 : 0, t1 = dn == 2 ? 1 : 2;
      const int st = dn == 0 ? 1 : (dn == 1 ? N : N2);
      const int s0 = t0 == 0 ? 1 : (t0 == 1 ? N : N2), s1 = t1 == 1 ? N : N2;
      const Real* src = U + (size_t)en[f] * 4 * N3 + ip * s0 + jp * s1;
      constexpr int LF = OFF_LF(N);
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        Real acc = tab<Real>(LF + sd * N) * __ldg(src + fl * N3);
#pragma unroll
        for (int s = 1; s < N; ++s) acc = fma(tab<Real>(LF + sd * N + s), __ldg(src + fl * N3 + s * st), acc);
        snb[(f * 4 + fl) * N2 + t] = acc;
      }
    }
  }
  const bool ok = mbar_wait_bounded(&bar, 0, p.err, p.expire_wait != 0);
  __syncthreads();
  const Real* gA = gAA + le * GA;
  const Real* gF = gFA + le * GF;
  const Real* gM = gMA + le * GM;
  if (act && ok) {  // y
    Real u[4][N], r[4][N];
    const int base = line_base<1, N, N>(a, b);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) u[fl][s] = su[fl * N3 + base + N * s];
    cell_face_dir<N, Real, 1, false, true>(u, r, gA, gF, snb, t, fmask);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) sr[fl * N3 + base + N * s] = r[fl][s];
  }
  __syncthreads();
  if (act && ok) {  // x
    Real u[4][N], r[4][N];
    const int base = line_base<0, N, N>(a, b);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) {
        u[fl][s] = su[fl * N3 + base + s];
        r[fl][s] = sr[fl * N3 + base + s];
      }
    cell_face_dir<N, Real, 0, true, true>(u, r, gA, gF, snb, t, fmask);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) sr[fl * N3 + base + s] = r[fl][s];
  }
  __syncthreads();
  if (act && ok) {  // z, then the diagonal inverse mass
    Real u[4][N], r[4][N];
    const int base = line_base<2, N, N>(a, b);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) {
        u[fl][s] = su[fl * N3 + base + N2 * s];
        r[fl][s] = sr[fl * N3 + base + N2 * s];
      }
    cell_face_dir<N, Real, 2, true, true>(u, r, gA, gF, snb, t, fmask);
    // the residual of this z-line is final: the epilogue runs here, on the
    // line's points (contiguous across the warp), with no shared-memory pass
    Real* __restrict__ out = static_cast<Real*>(p.out);
    Real* __restrict__ dU = static_cast<Real*>(p.dU);
    const Real cA = (Real)p.cA, cB = (Real)p.cB, dt = (Real)p.dt;
    const Real* sx = sxA + le * 4 * N3;
    const size_t g0 = (size_t)e * 4 * N3 + base;
#pragma unroll
    for (int s = 0; s < N; ++s) {
      const Real mp = gM[base + N2 * s], mvv = gM[N3 + base + N2 * s];
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        const Real R = r[fl][s] * (fl == 0 ? mp : mvv);
        const int i = fl * N3 + base + N2 * s;
        const size_t g = g0 + fl * N3 + N2 * s;
        if (EPI == EPI_WRITE) {
          out[g] = R;
        } else if (EPI == EPI_ADD) {
          out[g] = sx[i] + R;
        } else if (EPI == EPI_LSRK2R) {  // first stage: the running sum is the input itself
          const Real S = p.first ? su[i] : sx[i];
          if (!p.last) out[g] = fma(cA, R, S);
          dU[g] = fma(cB, R, S);
        } else {  // LSRK: the stage input is the staged state
          const Real d = p.first ? dt * R : fma(cA, sx[i], dt * R);
          dU[g] = d;
          out[g] = fma(cB, d, su[i]);
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_inval(&bar);
}

template <int N, typename Real, int EPI>
__global__ void opg_kernel(const OpParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int epb = blockDim.x / (N * N);
  const int e0 = blockIdx.x * epb;
  if constexpr (sizeof(Real) == 4)
    opgs_block<N, Real, EPI>(p, e0, min(epb, p.E - e0), epb, reinterpret_cast<Real*>(smem_raw));
  else
    opg_block<N, Real, EPI>(p, e0, min(epb, p.E - e0), reinterpret_cast<Real*>(smem_raw));
}


// ---------------------------------------------------------------------------
// Affine elements with element-wise constant coefficients: the metric, the
// mass diagonal and the face data are per-element constants times Gauss
// weights (w at a cell point, w_f = w_i w_j at a face point), read from the
// compact block of DG_AFF_OP values (see setup.cu).  With a constant metric
// the velocity tests need one contraction of w p per direction,
// distributed with adj(J)_{d i}.
// ---------------------------------------------------------------------------
template <int N, typename Real, int DIR, bool ACC, bool SMEM>
__device__ __forceinline__ void cell_face_dir_aff(const Real (&u)[4][N], Real (&r)[4][N],
                                                  const Real* __restrict__ g, const Real wab,
                                                  const Real iwab, const Real* snb, int t, int fmask) {
  constexpr int N2 = N * N;
  constexpr int W = OFF_W(N);
  const Real a0 = geo_ld<Real, SMEM>(g + DIR * 3), a1 = geo_ld<Real, SMEM>(g + DIR * 3 + 1),
             a2 = geo_ld<Real, SMEM>(g + DIR * 3 + 2);
  Real F[N], DG[N];
#pragma unroll
  for (int s = 0; s < N; ++s)
    F[s] = (wab * tab<Real>(W + s)) * fma(a0, u[1][s], fma(a1, u[2][s], a2 * u[3][s]));
  if (ACC)
    mtv_acc<Real, OFF_D(N), N, N>(F, r[0]);
  else
    mtv<Real, OFF_D(N), N, N>(F, r[0]);
#pragma unroll
  for (int s = 0; s < N; ++s) F[s] = (wab * tab<Real>(W + s)) * u[0][s];
  mtv<Real, OFF_D(N), N, N>(F, DG);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (ACC) {
      r[1][j] = fma(a0, DG[j], r[1][j]);
      r[2][j] = fma(a1, DG[j], r[2][j]);
      r[3][j] = fma(a2, DG[j], r[3][j]);
    } else {
      r[1][j] = a0 * DG[j];
      r[2][j] = a1 * DG[j];
      r[3][j] = a2 * DG[j];
    }
  }
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const int f = 2 * DIR + sd;
    constexpr int LF = OFF_LF(N);
    Real um[4];
#pragma unroll
    for (int fl = 0; fl < 4; ++fl) {
      Real acc = tab<Real>(LF + sd * N) * u[fl][0];
#pragma unroll
      for (int s = 1; s < N; ++s) acc = fma(tab<Real>(LF + sd * N + s), u[fl][s], acc);
      um[fl] = acc;
    }
    const Real* fc = g + 11 + f * 6;
    const Real nw0 = wab * geo_ld<Real, SMEM>(fc), nw1 = wab * geo_ld<Real, SMEM>(fc + 1),
               nw2 = wab * geo_ld<Real, SMEM>(fc + 2);
    const Real ca2 = geo_ld<Real, SMEM>(fc + 3), bb = iwab * geo_ld<Real, SMEM>(fc + 4),
               cc = wab * geo_ld<Real, SMEM>(fc + 5);
    const Real vnm = fma(nw0, um[1], fma(nw1, um[2], nw2 * um[3]));
    Real pp, vnp;
    if ((fmask >> f) & 1) {
      const Real* nb = snb + f * 4 * N2 + t;
      pp = nb[0];
      vnp = fma(nw0, nb[N2], fma(nw1, nb[2 * N2], nw2 * nb[3 * N2]));
    } else {
      pp = um[0];
      vnp = -vnm;
    }
    const Real dp = um[0] - pp, dvn = vnm - vnp;
    const Real pstar = fma(-ca2, dp, fma(bb, dvn, um[0]));
    const Real flp = fma(ca2, dvn, fma(cc, dp, vnp));
    const Real g0 = nw0 * pstar, g1 = nw1 * pstar, g2 = nw2 * pstar;
#pragma unroll
    for (int s = 0; s < N; ++s) {
      const Real l = tab<Real>(LF + sd * N + s);
      r[0][s] = fma(-l, flp, r[0][s]);
      r[1][s] = fma(-l, g0, r[1][s]);
      r[2][s] = fma(-l, g1, r[2][s]);
      r[3][s] = fma(-l, g2, r[3][s]);
    }
  }
}

template <int N>
__host__ __device__ constexpr int opga_smem_per_elem(bool stage) {
  return 4 * N * N * N * (stage ? 3 : 2) + 24 * N * N + (stage ? DG_AFF_OP : 0);
}

// Gauss-basis operator on affine elements.  STAGE: the block's state, LSRK
// register (or added state) and compact geometry come in by bulk
// asynchronous copies on an mbarrier (as opgs_block); otherwise the state is
// copied flat and the compact data read through the read-only path.
template <int N, typename Real, int EPI, bool STAGE>
__device__ __forceinline__ void opga_block(const OpParams& p, const int e0, const int ne, const int epb,
                                           Real* sm) {
  constexpr int N2 = N * N, N3 = N2 * N;
  __shared__ __align__(8) uint64_t bar;
  const int le = threadIdx.x / N2, t = threadIdx.x - le * N2;
  const int a = t % N, b = t / N;
  const int e = e0 + le;
  const bool act = le < ne;
  Real* suA = sm;
  Real* srA = suA + epb * 4 * N3;
  Real* snA = srA + epb * 4 * N3;
  Real* gKA = snA + epb * 24 * N2;  // STAGE only
  Real* sxA = gKA + epb * DG_AFF_OP;  // STAGE only
  const bool need_x = ((EPI == EPI_LSRK || EPI == EPI_LSRK2R) && !p.first) || EPI == EPI_ADD;
  const Real* __restrict__ U = static_cast<const Real*>(p.U);
  if constexpr (STAGE) {
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t sb = ne * 4 * N3 * sizeof(Real);
      const uint32_t gb = ne * DG_AFF_OP * sizeof(Real);
      mbar_expect_tx(&bar, sb * (need_x ? 2 : 1) + gb);
      bulk_copy_g2s(suA, U + (size_t)e0 * 4 * N3, sb, &bar);
      bulk_copy_g2s(gKA, static_cast<const Real*>(p.geoK) + (size_t)e0 * DG_AFF_OP, gb, &bar);
      if (need_x) {
        const Real* X = EPI == EPI_LSRK ? static_cast<const Real*>(p.dU) : static_cast<const Real*>(p.Uadd);
        bulk_copy_g2s(sxA, X + (size_t)e0 * 4 * N3, sb, &bar);
      }
    }
  } else {
    for (int i = threadIdx.x; i < ne * 4 * N3; i += blockDim.x) suA[i] = U[(size_t)e0 * 4 * N3 + i];
  }
  Real* su = suA + le * 4 * N3;
  Real* sr = srA + le * 4 * N3;
  Real* snb = snA + le * 24 * N2;
  // weights of this thread's line: the two fixed coordinates are (a, b)
  const Real wab = tab<Real>(OFF_W(N) + a) * tab<Real>(OFF_W(N) + b);
  const Real iwab = tab<Real>(OFF_IW(N) + a) * tab<Real>(OFF_IW(N) + b);
  int fmask = 0;
  if (act) {
    int en[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) en[f] = p.nbr[e * 6 + f];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      if (en[f] < 0) continue;
      fmask |= 1 << f;
      const int fn = p.nbr_face[e * 6 + f], o = p.orient[e * 6 + f];
      const int uu = (o & 1) ? b : a, vv = (o & 1) ? a : b;
      const int ip = (o & 2) ? N - 1 - uu : uu, jp = (o & 4) ? N - 1 - vv : vv;
      const int dn = fn >> 1, sd = fn & 1;
      const int t0 = dn == 0 ? 1 : 0, t1 = dn == 2 ? 1 : 2;
      const int st = dn == 0 ? 1 : (dn == 1 ? N : N2);
      const int s0 = t0 == 0 ? 1 : (t0 == 1 ? N : N2), s1 = t1 == 1 ? N : N2;
      const Real* src = U + (size_t)en[f] * 4 * N3 + ip * s0 + jp * s1;
      constexpr int LF = OFF_LF(N);
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        Real acc = tab<Real>(LF + sd * N) * __ldg(src + fl * N3);
#pragma unroll
        for (int s = 1; s < N; ++s) acc = fma(tab<Real>(LF + sd * N + s), __ldg(src + fl * N3 + s * st), acc);
        snb[(f * 4 + fl) * N2 + t] = acc;
      }
    }
  }
  bool ok = true;
  if constexpr (STAGE) ok = mbar_wait_bounded(&bar, 0, p.err, p.expire_wait != 0);
  __syncthreads();
  const Real* gK = STAGE ? gKA + le * DG_AFF_OP : static_cast<const Real*>(p.geoK) + (size_t)(act ? e : 0) * DG_AFF_OP;
  if (act && ok) {  // y
    Real u[4][N], r[4][N];
    const int base = line_base<1, N, N>(a, b);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) u[fl][s] = su[fl * N3 + base + N * s];
    cell_face_dir_aff<N, Real, 1, false, STAGE>(u, r, gK, wab, iwab, snb, t, fmask);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) sr[fl * N3 + base + N * s] = r[fl][s];
  }
  __syncthreads();
  if (act && ok) {  // x
    Real u[4][N], r[4][N];
    const int base = line_base<0, N, N>(a, b);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) {
        u[fl][s] = su[fl * N3 + base + s];
        r[fl][s] = sr[fl * N3 + base + s];
      }
    cell_face_dir_aff<N, Real, 0, true, STAGE>(u, r, gK, wab, iwab, snb, t, fmask);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) sr[fl * N3 + base + s] = r[fl][s];
  }
  __syncthreads();
  if (act && ok) {  // z, then the diagonal inverse mass m / w
    Real u[4][N], r[4][N];
    const int base = line_base<2, N, N>(a, b);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl)
#pragma unroll
      for (int s = 0; s < N; ++s) {
        u[fl][s] = su[fl * N3 + base + N2 * s];
        r[fl][s] = sr[fl * N3 + base + N2 * s];
      }
    cell_face_dir_aff<N, Real, 2, true, STAGE>(u, r, gK, wab, iwab, snb, t, fmask);
    const Real mpab = geo_ld<Real, STAGE>(gK + 9) * iwab, mvab = geo_ld<Real, STAGE>(gK + 10) * iwab;
    // the residual of this z-line is final: the epilogue runs here, on the
    // line's points (across the warp the lines' points are contiguous in
    // memory), without a round trip through shared memory
    Real* __restrict__ out = static_cast<Real*>(p.out);
    Real* __restrict__ dU = static_cast<Real*>(p.dU);
    const Real* __restrict__ Uadd = static_cast<const Real*>(p.Uadd);
    const Real cA = (Real)p.cA, cB = (Real)p.cB, dt = (Real)p.dt;
    const Real* sx = sxA + le * 4 * N3;
    const size_t g0 = (size_t)e * 4 * N3 + base;
#pragma unroll
    for (int s = 0; s < N; ++s) {
      const Real iw = tab<Real>(OFF_IW(N) + s);
      const Real mp = mpab * iw, mvv = mvab * iw;
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        const Real R = r[fl][s] * (fl == 0 ? mp : mvv);
        const int i = fl * N3 + base + N2 * s;
        const size_t g = g0 + fl * N3 + N2 * s;
        if (EPI == EPI_WRITE) {
          out[g] = R;
        } else if (EPI == EPI_ADD) {
          out[g] = (STAGE ? sx[i] : Uadd[g]) + R;
        } else if (EPI == EPI_LSRK2R) {
          const Real S = STAGE ? (p.first ? su[i] : sx[i]) : Uadd[g];
          if (!p.last) out[g] = fma(cA, R, S);
          dU[g] = fma(cB, R, S);
        } else {
          const Real d = p.first ? dt * R : fma(cA, STAGE ? sx[i] : dU[g], dt * R);
          dU[g] = d;
          out[g] = fma(cB, d, su[i]);
        }
      }
    }
  }
  if constexpr (STAGE) {
    __syncthreads();
    if (threadIdx.x == 0) mbar_inval(&bar);
  }
}

template <int N, typename Real, int EPI>
__global__ void opga_kernel(const OpParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int epb = blockDim.x / (N * N);
  const int e0 = blockIdx.x * epb;
  opga_block<N, Real, EPI, sizeof(Real) == 4>(p, e0, min(epb, p.E - e0), epb, reinterpret_cast<Real*>(smem_raw));
}

// Change of basis of whole states, GL -> G (to_g) or G -> GL, from src to
// dst (the same array for an in-place change).  src or dst may be pinned
// host memory mapped into the device's address space: the element blocks
// are contiguous, so both copies are 16-byte vector accesses, coalesced
// across the block, and a host-to-device transfer fused with the change of
// basis costs one pass.
template <int N, typename Real>
__global__ void basis_kernel(const void* src, void* dst, int E, int to_g) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int VW = 16 / sizeof(Real);  // Reals per 16-byte vector
  typedef typename std::conditional<sizeof(Real) == 8, double2, float4>::type Vec;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int epb = blockDim.x / N2;
  const int le = threadIdx.x / N2, t = threadIdx.x - le * N2;
  const int e0 = blockIdx.x * epb;
  const int ne = min(epb, E - e0);
  Real* su = sm + le * 4 * N3;
  // 4 N^3 Reals per element is a multiple of VW, and states are 16-byte aligned
  const Vec* in = reinterpret_cast<const Vec*>(static_cast<const Real*>(src) + (size_t)e0 * 4 * N3);
  Vec* smv = reinterpret_cast<Vec*>(sm);
  {  // four loads in flight per thread: a host source answers with a long latency
    const int nv = ne * 4 * N3 / VW, bd = blockDim.x;
    int i = threadIdx.x;
    for (; i + 3 * bd < nv; i += 4 * bd) {
      const Vec v0 = in[i], v1 = in[i + bd], v2 = in[i + 2 * bd], v3 = in[i + 3 * bd];
      smv[i] = v0;
      smv[i + bd] = v1;
      smv[i + 2 * bd] = v2;
      smv[i + 3 * bd] = v3;
    }
    for (; i < nv; i += bd) smv[i] = in[i];
  }
  __syncthreads();
  const bool act = le < ne;
  if (to_g) {
    if (act) contract_tile<Real, 2, N, N, N, N, OFF_V(N), N3, N3>(su, su, t, N2);
    __syncthreads();
    if (act) contract_tile<Real, 0, N, N, N, N, OFF_V(N), N3, N3>(su, su, t, N2);
    __syncthreads();
    if (act) contract_tile<Real, 1, N, N, N, N, OFF_V(N), N3, N3>(su, su, t, N2);
  } else {
    if (act) contract_tile<Real, 2, N, N, N, N, OFF_VI(N), N3, N3>(su, su, t, N2);
    __syncthreads();
    if (act) contract_tile<Real, 0, N, N, N, N, OFF_VI(N), N3, N3>(su, su, t, N2);
    __syncthreads();
    if (act) contract_tile<Real, 1, N, N, N, N, OFF_VI(N), N3, N3>(su, su, t, N2);
  }
  __syncthreads();
  Vec* out = reinterpret_cast<Vec*>(static_cast<Real*>(dst) + (size_t)e0 * 4 * N3);
  for (int i = threadIdx.x; i < ne * 4 * N3 / VW; i += blockDim.x) out[i] = smv[i];
}

// ---------------------------------------------------------------------------
// Taylor-Cauchy-Kowalevski predictor (Sec. 2.3 Eq. (6), Sec. 3.2 Alg. 2,
// Sec. 3.3 Alg. 3).
// ---------------------------------------------------------------------------
struct TckParams {
  const void* U;   // state (GL, or G if gmode)
  void* Ubar;      // predictor output (same basis as U)
  const void* geoT;
  long long geoT_stride;  // Reals per element
  double coef[DG_NMAX + 2];  // dt^{j+1} / (j+1)!
  int E;
  int gmode;  // 1: U and Ubar hold Gauss-point values (no basis change)
  int aff;    // 1: affine elements with constant coefficients (geoKT)
  int geo_step;  // geoT holds the Gauss sets m = n, n - geo_step, ... >= 2 (1 or 2)
  const void* geoKT;  // [E][DG_AFF_TCK]: J^-1 (9), -rho c^2, -1/rho
  const void* W;      // HDG-ADER: T_1 = W (the DG derivative, same basis as U) instead of -S U; else null
  int* err;           // set (non-zero) if a bounded wait gave up (staged kernels only)
};

// m-point levels visited with reduction every RED-th derivative (RED = 0:
// none): N, N-RED, ... >= 1
template <int N, int RED>
__host__ __device__ constexpr int tck_level_count() {
  return RED == 0 ? 1 : (N - 1) / RED + 1;
}
template <int N, int RED>
__host__ __device__ constexpr int tck_level_m(int l) {
  return RED == 0 ? N : N - RED * l;
}
// accumulator offset of level l (Reals, 4 fields each)
template <int N, int RED>
__host__ __device__ constexpr int tck_acc_off(int l) {
  return l == 0 ? 0 : tck_acc_off<N, RED>(l - 1) + 4 * tck_level_m<N, RED>(l - 1) *
                                                        tck_level_m<N, RED>(l - 1) *
                                                        tck_level_m<N, RED>(l - 1);
}
template <int N, int RED>
__host__ __device__ constexpr int tck_smem_per_elem() {
  return 8 * N * N * N + tck_acc_off<N, RED>(tck_level_count<N, RED>());
}
// per-element geometry of the predictor: Gauss sets m = n, n-s, n-2s, ... >= 2
// (s = 2 serves reduction every 0 or 2 derivatives, s = 1 every 1, 2 or 3),
// each [3 d][3 i][m^3] line-major J^-1_{d i}, then [2][m^3] (-rho c^2, -1/rho)
__host__ __device__ constexpr int tck_geo_stride(int n, int s) {
  return n < 2 ? 0 : 11 * n * n * n + tck_geo_stride(n - s, s);
}

// One derivative T_j = -S T_{j-1} at an M^3 Gauss set (Alg. 2 "evaluate the
// gradient, set values") for the ne elements of a block: src0 holds element
// 0's T_{j-1} (4 x M^3, field stride FS), dst0 receives T_j, es is the
// element stride in shared memory; g0 points at element 0's geometry of this
// set, gs is the per-element geometry stride.  The ne M^2 lines of a
// direction are spread over all threads of the block.
template <int M, typename Real, int FS>
__device__ __forceinline__ void tck_derivative(const Real* src0, Real* dst0, int es,
                                               const Real* __restrict__ g0, long long gs, int ne, int T,
                                               int nthr) {
  constexpr int M2 = M * M, M3 = M2 * M;
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    for (int L = T; L < ne * M2; L += nthr) {
      const int le = L / M2, l = L - le * M2;
      const Real* src = src0 + le * es;
      Real* dst = dst0 + le * es;
      const Real* g = g0 + le * gs;
      const int a = l % M, b = l / M;
      const int base = dir == 0 ? M * a + M2 * b : (dir == 1 ? a + M2 * b : a + M * b);
      const int st = dir == 0 ? 1 : (dir == 1 ? M : M2);
      Real q[4][M], d[4][M];
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
#pragma unroll
        for (int s = 0; s < M; ++s) q[fl][s] = src[fl * FS + base + st * s];
        mv<Real, OFF_D(M), M, M>(q[fl], d[fl]);
      }
      const Real* J0 = g + (dir * 3 + 0) * M3 + l;
      const Real* J1 = g + (dir * 3 + 1) * M3 + l;
      const Real* J2 = g + (dir * 3 + 2) * M3 + l;
#pragma unroll
      for (int s = 0; s < M; ++s) {
        const Real j0 = __ldg(J0 + M2 * s), j1 = __ldg(J1 + M2 * s), j2 = __ldg(J2 + M2 * s);
        const int idx = base + st * s;
        Real tp, tv0, tv1, tv2;
        if (dir > 0) {  // continue the sums of the previous directions
          tp = fma(j0, d[1][s], fma(j1, d[2][s], fma(j2, d[3][s], dst[idx])));
          tv0 = fma(j0, d[0][s], dst[FS + idx]);
          tv1 = fma(j1, d[0][s], dst[2 * FS + idx]);
          tv2 = fma(j2, d[0][s], dst[3 * FS + idx]);
        } else {
          tp = fma(j0, d[1][s], fma(j1, d[2][s], j2 * d[3][s]));
          tv0 = j0 * d[0][s];
          tv1 = j1 * d[0][s];
          tv2 = j2 * d[0][s];
        }
        if (dir == 2) {  // coefficients: -rho c^2 (p), -1/rho (v)
          const Real cp = __ldg(g + 9 * M3 + idx), cv = __ldg(g + 10 * M3 + idx);
          tp *= cp;
          tv0 *= cv;
          tv1 *= cv;
          tv2 *= cv;
        }
        dst[idx] = tp;
        dst[FS + idx] = tv0;
        dst[2 * FS + idx] = tv1;
        dst[3 * FS + idx] = tv2;
      }
    }
    __syncthreads();
  }
}

// The derivative step on an affine element with constant coefficients:
// J^-1 is constant, so the pressure equation differentiates the combination
// sum_i (J^-1)_{d i} v_i once per direction, and the velocity equations share
// one derivative of p per direction (two contractions per direction instead
// of four).  g: the element's DG_AFF_TCK values.
template <int M, typename Real, int FS>
__device__ __forceinline__ void tck_derivative_aff(const Real* src0, Real* dst0, int es,
                                                   const Real* __restrict__ g0, int ne, int T, int nthr) {
  constexpr int M2 = M * M;
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    for (int L = T; L < ne * M2; L += nthr) {
      const int le = L / M2, l = L - le * M2;
      const Real* src = src0 + le * es;
      Real* dst = dst0 + le * es;
      const Real* g = g0 + le * DG_AFF_TCK;
      const Real cp = __ldg(g + 9), cv = __ldg(g + 10);
      const Real j0 = __ldg(g + dir * 3), j1 = __ldg(g + dir * 3 + 1), j2 = __ldg(g + dir * 3 + 2);
      const int a = l % M, b = l / M;
      const int base = dir == 0 ? M * a + M2 * b : (dir == 1 ? a + M2 * b : a + M * b);
      const int st = dir == 0 ? 1 : (dir == 1 ? M : M2);
      Real q0[M], w[M], dp[M], dw[M];
#pragma unroll
      for (int s = 0; s < M; ++s) {
        q0[s] = src[base + st * s];
        w[s] = fma(j0, src[FS + base + st * s], fma(j1, src[2 * FS + base + st * s], j2 * src[3 * FS + base + st * s]));
      }
      mv<Real, OFF_D(M), M, M>(q0, dp);
      mv<Real, OFF_D(M), M, M>(w, dw);
#pragma unroll
      for (int s = 0; s < M; ++s) {
        const int idx = base + st * s;
        Real tp, tv0, tv1, tv2;
        if (dir > 0) {
          tp = dw[s] + dst[idx];
          tv0 = fma(j0, dp[s], dst[FS + idx]);
          tv1 = fma(j1, dp[s], dst[2 * FS + idx]);
          tv2 = fma(j2, dp[s], dst[3 * FS + idx]);
        } else {
          tp = dw[s];
          tv0 = j0 * dp[s];
          tv1 = j1 * dp[s];
          tv2 = j2 * dp[s];
        }
        if (dir == 2) {
          tp *= cp;
          tv0 *= cv;
          tv1 *= cv;
          tv2 *= cv;
        }
        dst[idx] = tp;
        dst[FS + idx] = tv0;
        dst[2 * FS + idx] = tv1;
        dst[3 * FS + idx] = tv2;
      }
    }
    __syncthreads();
  }
}

// Reference L2 projection M^3 -> (M-RR)^3 (Sec. 3.3, Alg. 3 for RR = 2):
// three contractions, src (M^3, field stride FS) -> tmp -> src; the result
// is left in tmp.
template <int M, int RR, typename Real, int FS>
__device__ __forceinline__ void tck_project(Real* src0, Real* tmp0, int es, int ne, int T, int nthr) {
  constexpr int R = M - RR;
  contract_tile_b<Real, 0, M, M, M, R, OFF_PR(M, RR), FS, FS>(src0, tmp0, es, ne, T, nthr);
  __syncthreads();
  contract_tile_b<Real, 1, R, M, M, R, OFF_PR(M, RR), FS, FS>(tmp0, src0, es, ne, T, nthr);
  __syncthreads();
  contract_tile_b<Real, 2, R, R, M, R, OFF_PR(M, RR), FS, FS>(src0, tmp0, es, ne, T, nthr);
  __syncthreads();
}

// acc_big += I(M+RR <- M) applied to acc_small in all three directions
template <int M, int RR, typename Real, int FS>
__device__ __forceinline__ void tck_fold(const Real* small0, Real* big0, Real* t10, Real* t20, int es,
                                         int ne, int T, int nthr) {
  constexpr int B = M + RR;
  contract_tile_b<Real, 0, M, M, M, B, OFF_IR(B, RR), M * M * M, FS>(small0, t10, es, ne, T, nthr);
  __syncthreads();
  contract_tile_b<Real, 1, B, M, M, B, OFF_IR(B, RR), FS, FS>(t10, t20, es, ne, T, nthr);
  __syncthreads();
  contract_tile_b<Real, 2, B, B, M, B, OFF_IR(B, RR), FS, B * B * B, true>(t20, big0, es, ne, T, nthr);
  __syncthreads();
}

// acc += c T over the ne elements of a block (element stride es; T has
// field stride fs, acc field stride m3), spread over the block's threads.
template <typename Real>
__device__ __forceinline__ void tck_accumulate(Real* acc0, const Real* T0, int es, int m3, Real c,
                                               int fs, int ne, int tid, int nthr) {
  const int per = 4 * m3;
  for (int i = tid; i < ne * per; i += nthr) {
    const int le = i / per, r = i - le * per;
    const int fl = r / m3, q = r - fl * m3;
    Real* acc = acc0 + le * es;
    acc[r] = fma(c, T0[le * es + fl * fs + q], acc[r]);
  }
}

// One block's share of the predictor: elements e0 .. e0+ne-1 of a block
// laid out for epb elements.  The basis changes at the full point set give
// each element's N^2 threads one line each; threads of element slots >= epb
// (a block sized for another degree) take none of those lines.  From the
// first derivative on, the lines, points and accumulator entries of all ne
// elements are spread over every thread of the block, so that the reduced
// sets (m^2 < N^2 lines per element) still fill whole warps.
template <int N, typename Real, int RED>
__device__ __forceinline__ void tck_block(const TckParams& p, const int e0, const int ne, const int epb,
                                          Real* sm) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int SE = tck_smem_per_elem<N, RED>();
  constexpr int NL = tck_level_count<N, RED>();
  constexpr int ACC = 8 * N3;  // accumulators after the two T buffers
  const int T = threadIdx.x, NT = blockDim.x;
  const int le0 = T / N2;
  const bool own = le0 < epb;
  const int le = own ? le0 : 0;
  const int t = own ? T - le0 * N2 : (1 << 28);  // no line for non-owners
  Real* s0 = sm + le * SE;  // T buffers (field stride N3)
  const Real* __restrict__ U = static_cast<const Real*>(p.U);
  const Real* geo0 = static_cast<const Real*>(p.geoT) + (size_t)e0 * p.geoT_stride;
  const Real* geoK0 = p.aff ? static_cast<const Real*>(p.geoKT) + (size_t)e0 * DG_AFF_TCK : nullptr;

  for (int i = T; i < ne * 4 * N3; i += NT) {
    const int l = i / (4 * N3);
    sm[l * SE + (i - l * 4 * N3)] = U[(size_t)e0 * 4 * N3 + i];
  }
  constexpr int NACC = tck_acc_off<N, RED>(NL);
  for (int i = T; i < ne * NACC; i += NT) {
    const int l = i / NACC;
    sm[l * SE + ACC + (i - l * NACC)] = Real(0);
  }
  __syncthreads();
  // GL -> G (Sec. 3.2: the basis change is done per element on the fly)
  if (!p.gmode) {
    contract_tile<Real, 2, N, N, N, N, OFF_V(N), N3, N3>(s0, s0, t, N2);
    __syncthreads();
    contract_tile<Real, 0, N, N, N, N, OFF_V(N), N3, N3>(s0, s0, t, N2);
    __syncthreads();
    contract_tile<Real, 1, N, N, N, N, OFF_V(N), N3, N3>(s0, s0, t, N2);
    __syncthreads();
  }
  tck_accumulate<Real>(sm + ACC, sm, SE, N3, (Real)p.coef[0], N3, ne, T, NT);

  // Taylor terms j = 1 .. k+1 (k + 1 = N); cur / nxt: element 0's buffers
  Real* cur = sm;
  Real* nxt = sm + 4 * N3;
  int m = N, goff = 0, aoff = 0;  // goff: this set's geometry; aoff: its accumulator
#pragma unroll 1
  for (int j = 1; j <= N; ++j) {
    if (j == 1 && p.W) {  // HDG-ADER (Eq. hdg-ader): the DG derivative in place of -S U
      const Real* __restrict__ Wg = static_cast<const Real*>(p.W);
      for (int i = T; i < ne * 4 * N3; i += NT) {
        const int l = i / (4 * N3);
        nxt[l * SE + (i - l * 4 * N3)] = Wg[(size_t)e0 * 4 * N3 + i];
      }
      __syncthreads();
      if (!p.gmode) {
        Real* w = nxt + le * SE;
        contract_tile<Real, 2, N, N, N, N, OFF_V(N), N3, N3>(w, w, t, N2);
        __syncthreads();
        contract_tile<Real, 0, N, N, N, N, OFF_V(N), N3, N3>(w, w, t, N2);
        __syncthreads();
        contract_tile<Real, 1, N, N, N, N, OFF_V(N), N3, N3>(w, w, t, N2);
        __syncthreads();
      }
    } else {
    // derivative at the current m (T_{j-1} in cur, field stride N3)
    switch (m) {
#define DG_TCK_DERIV(MM)                                                                  \
  case MM:                                                                                \
    if constexpr (MM <= N) {                                                              \
      if (p.aff)                                                                          \
        tck_derivative_aff<MM, Real, N3>(cur, nxt, SE, geoK0, ne, T, NT);                 \
      else                                                                                \
        tck_derivative<MM, Real, N3>(cur, nxt, SE, geo0 + goff, p.geoT_stride, ne, T, NT); \
    }                                                                                     \
    break;
      DG_TCK_DERIV(2) DG_TCK_DERIV(3) DG_TCK_DERIV(4) DG_TCK_DERIV(5) DG_TCK_DERIV(6)
      DG_TCK_DERIV(7) DG_TCK_DERIV(8)
#undef DG_TCK_DERIV
      default:  // m == 1: the derivative of a constant vanishes
        for (int i = T; i < ne * 4 * N3; i += NT) {
          const int l = i / (4 * N3);
          nxt[l * SE + (i - l * 4 * N3)] = Real(0);
        }
        __syncthreads();
        break;
    }
    }
    if (RED > 0 && (j % RED) == 0) {
      if (m - RED < 1) break;  // projected to degree < 0: T_j = 0, stop
      switch (m) {
#define DG_TCK_PROJ(MM)                                                                              \
  case MM:                                                                                           \
    if constexpr (RED > 0 && MM <= N && MM - RED >= 1) tck_project<MM, RED, Real, N3>(nxt, cur, SE, ne, T, NT); \
    break;
        DG_TCK_PROJ(2) DG_TCK_PROJ(3) DG_TCK_PROJ(4) DG_TCK_PROJ(5) DG_TCK_PROJ(6)
        DG_TCK_PROJ(7) DG_TCK_PROJ(8)
#undef DG_TCK_PROJ
        default:
          break;
      }
      // the projection leaves its result in cur
      Real* tmp = cur;
      cur = nxt;
      nxt = tmp;
      // the stored Gauss sets between m and m - RED (step geo_step) precede the next one
      const int gs = p.geo_step > 1 ? 2 : 1;
      for (int mm = m; mm > m - RED; mm -= gs) goff += 11 * mm * mm * mm;
      aoff += 4 * m * m * m;
      m -= RED;
    }
    // T_j is in nxt at m points
    tck_accumulate<Real>(sm + ACC + aoff, nxt, SE, m * m * m, (Real)p.coef[j], N3, ne, T, NT);
    __syncthreads();
    Real* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  // fold the levels from the smallest up: acc(m+RED) += I(m -> m+RED) acc(m)
  if (RED > 0) {
#pragma unroll
    for (int l = NL - 1; l >= 1; --l) {
      const int ms = tck_level_m<N, RED>(l);
      Real* small = sm + ACC + tck_acc_off<N, RED>(l);
      Real* big = sm + ACC + tck_acc_off<N, RED>(l - 1);
      switch (ms) {
#define DG_TCK_FOLD(MM)                                                                                   \
  case MM:                                                                                                \
    if constexpr (RED > 0 && MM + RED <= N) tck_fold<MM, RED, Real, N3>(small, big, sm, sm + 4 * N3, SE, ne, T, NT); \
    break;
        DG_TCK_FOLD(1) DG_TCK_FOLD(2) DG_TCK_FOLD(3) DG_TCK_FOLD(4) DG_TCK_FOLD(5)
        DG_TCK_FOLD(6) DG_TCK_FOLD(7)
#undef DG_TCK_FOLD
        default:
          break;
      }
    }
  }
  // G -> GL and store
  Real* __restrict__ out = static_cast<Real*>(p.Ubar);
  if (p.gmode) {
    __syncthreads();
    for (int i = T; i < ne * 4 * N3; i += NT) {
      const int l = i / (4 * N3);
      out[(size_t)e0 * 4 * N3 + i] = sm[l * SE + ACC + (i - l * 4 * N3)];  // level-n accumulator
    }
    return;
  }
  Real* acc = s0 + ACC;
  Real* s1 = s0 + 4 * N3;
  contract_tile<Real, 2, N, N, N, N, OFF_VI(N), N3, N3>(acc, s0, t, N2);
  __syncthreads();
  contract_tile<Real, 0, N, N, N, N, OFF_VI(N), N3, N3>(s0, s1, t, N2);
  __syncthreads();
  contract_tile<Real, 1, N, N, N, N, OFF_VI(N), N3, N3>(s1, s0, t, N2);
  __syncthreads();
  for (int i = T; i < ne * 4 * N3; i += NT) {
    const int l = i / (4 * N3);
    out[(size_t)e0 * 4 * N3 + i] = sm[l * SE + (i - l * 4 * N3)];
  }
}

template <int N, typename Real, int RED>
__global__ void tck_kernel(const TckParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int epb = blockDim.x / (N * N);
  const int e0 = blockIdx.x * epb;
  tck_block<N, Real, RED>(p, e0, min(epb, p.E - e0), epb, reinterpret_cast<Real*>(smem_raw));
}

// ---------------------------------------------------------------------------
// Energy 1/2 U^T M U (Gauss rule, diagonal mass in G) and sums of squares.
// Each block writes one partial; a second pass sums the partials in order.
// ---------------------------------------------------------------------------
struct EnergyParams {
  const void* U;
  const void* geoM;
  double* partial;
  int E;
};

template <int N, typename Real>
__global__ void energy_kernel(const EnergyParams p) {
  constexpr int N2 = N * N, N3 = N2 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int epb = blockDim.x / N2;
  const int le = threadIdx.x / N2, t = threadIdx.x - le * N2;
  const int e0 = blockIdx.x * epb;
  const int ne = min(epb, p.E - e0);
  const int e = e0 + le;
  const bool act = le < ne;
  Real* su = sm + le * 4 * N3;
  const Real* U = static_cast<const Real*>(p.U);
  for (int i = threadIdx.x; i < ne * 4 * N3; i += blockDim.x)
    sm[i] = U[(size_t)e0 * 4 * N3 + i];
  __syncthreads();
  if (act) contract_tile<Real, 2, N, N, N, N, OFF_V(N), N3, N3>(su, su, t, N2);
  __syncthreads();
  if (act) contract_tile<Real, 0, N, N, N, N, OFF_V(N), N3, N3>(su, su, t, N2);
  __syncthreads();
  if (act) contract_tile<Real, 1, N, N, N, N, OFF_V(N), N3, N3>(su, su, t, N2);
  __syncthreads();
  double s = 0.0;
  if (act) {
    const Real* gM = static_cast<const Real*>(p.geoM) + (size_t)e * geo_stride_M(N);
    for (int q = t; q < N3; q += N2) {
      const double pp = su[q], vx = su[N3 + q], vy = su[2 * N3 + q], vz = su[3 * N3 + q];
      s += pp * pp / (double)gM[q] + (vx * vx + vy * vy + vz * vz) / (double)gM[N3 + q];
    }
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

// ---------------------------------------------------------------------------
// Batched form: many independent solves (different meshes, degrees, time
// steps) advanced by persistent launches.  A work item is a run of
// consecutive elements of one instance, processed one block's worth (epb
// elements) at a time; blocks take items from a counter (dynamic
// scheduling, no waiting) and run the same per-element code as the
// single-solve kernels, so each instance's result does not depend on what
// else is in the batch.
// ---------------------------------------------------------------------------
struct BatchItem {
  int inst, e0, ne, n, epb;
};
// per instance: operator parameters of the five LSRK stages and of the ADER
// update, and the predictor parameters
struct BatchInst {
  OpParams op[6];
  TckParams tck;
};

// One launch per degree present in the batch: every item has n == N, so the
// block shape and register use are those of that degree alone; launches of
// different degrees run concurrently (they belong to different solves).
// MODE: 0 GL states (op_block), 1 Gauss-basis states (opgs/opg_block),
// 2 Gauss-basis states on affine elements (opga_block).
template <int N, typename Real, int EPI, int MODE>
__global__ void batch_op_kernel(const BatchItem* __restrict__ items, int nitems,
                                const BatchInst* __restrict__ inst, int phase, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    const BatchItem w = items[it];
    const OpParams& p = inst[w.inst].op[phase];
    // the item's elements in slices of epb (one block's worth)
    for (int e0 = w.e0; e0 < w.e0 + w.ne; e0 += w.epb) {
      const int ne = min(w.epb, w.e0 + w.ne - e0);
      if constexpr (MODE == 0)
        op_block<N, Real, EPI>(p, e0, ne, sm);
      else if constexpr (MODE == 2)
        opga_block<N, Real, EPI, sizeof(Real) == 4>(p, e0, ne, w.epb, sm);
      else if constexpr (sizeof(Real) == 4)
        opgs_block<N, Real, EPI>(p, e0, ne, w.epb, sm);
      else
        opg_block<N, Real, EPI>(p, e0, ne, sm);
      __syncthreads();  // shared memory is reused by the next slice
    }
  }
}

// In-place change of basis of the states of a batch's solves of degree N
// (GL -> G if to_g, else G -> GL), over the same work items.
template <int N, typename Real>
__global__ void batch_basis_kernel(const BatchItem* __restrict__ items, int nitems,
                                   const BatchInst* __restrict__ inst, int to_g, int* counter) {
  constexpr int N2 = N * N, N3 = N2 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    const BatchItem w = items[it];
    Real* U = static_cast<Real*>(const_cast<void*>(inst[w.inst].tck.U));
    for (int e0 = w.e0; e0 < w.e0 + w.ne; e0 += w.epb) {
      const int ne = min(w.epb, w.e0 + w.ne - e0);
      const int le = threadIdx.x / N2, t = threadIdx.x - le * N2;
      const bool act = le < ne;
      Real* su = sm + le * 4 * N3;
      for (int i = threadIdx.x; i < ne * 4 * N3; i += blockDim.x) sm[i] = U[(size_t)e0 * 4 * N3 + i];
      __syncthreads();
      if (to_g) {
        if (act) contract_tile<Real, 2, N, N, N, N, OFF_V(N), N3, N3>(su, su, t, N2);
        __syncthreads();
        if (act) contract_tile<Real, 0, N, N, N, N, OFF_V(N), N3, N3>(su, su, t, N2);
        __syncthreads();
        if (act) contract_tile<Real, 1, N, N, N, N, OFF_V(N), N3, N3>(su, su, t, N2);
      } else {
        if (act) contract_tile<Real, 2, N, N, N, N, OFF_VI(N), N3, N3>(su, su, t, N2);
        __syncthreads();
        if (act) contract_tile<Real, 0, N, N, N, N, OFF_VI(N), N3, N3>(su, su, t, N2);
        __syncthreads();
        if (act) contract_tile<Real, 1, N, N, N, N, OFF_VI(N), N3, N3>(su, su, t, N2);
      }
      __syncthreads();
      for (int i = threadIdx.x; i < ne * 4 * N3; i += blockDim.x) U[(size_t)e0 * 4 * N3 + i] = sm[i];
      __syncthreads();
    }
  }
}

template <int N, typename Real, int RED>
__global__ void batch_tck_kernel(const BatchItem* __restrict__ items, int nitems,
                                 const BatchInst* __restrict__ inst, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    const BatchItem w = items[it];
    for (int e0 = w.e0; e0 < w.e0 + w.ne; e0 += w.epb) {
      tck_block<N, Real, RED>(inst[w.inst].tck, e0, min(w.epb, w.e0 + w.ne - e0), w.epb, sm);
      __syncthreads();
    }
  }
}

}  // namespace dg
