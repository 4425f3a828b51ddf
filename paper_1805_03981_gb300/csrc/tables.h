// 1D tables of the tensor-product DG discretisation (host side, FP64).
//
// A "count" c is a number of points per direction; c = k+1 for the element
// and c = k+1, k-1, ... for the reduced point sets of the Taylor-Cauchy-
// Kowalevski predictor (Sec. 3.3).  For every c in [1, DG_NMAX] the flat
// table holds, row-major:
//   V  [c][c]      GL(c) -> G(c): V[q][a] = l^GL_a(x^G_q)       (Sec. 3.1)
//   VI [c][c]      G(c) -> GL(c): VI[a][q] = l^G_q(x^GL_a)      (exact inverse)
//   D  [c][c]      collocation derivative on the Gauss points:
//                  D[q][a] = (l^G_a)'(x^G_q)                    (Sec. 3.2, Alg. 2)
//   LF [2][c]      l^G_a(-1), l^G_a(+1): Gauss-basis face traces
//   for each reduction r = 1, 2, 3 with c > r:
//     P_r [c-r][c] reference-element L2 projection Gauss(c) -> Gauss(c-r):
//                  P_r[a][b] = w^c_b l^{c-r}_a(x^c_b) / w^{c-r}_a  (Sec. 3.3)
//     I_r [c][c-r] prolongation Gauss(c-r) -> Gauss(c):
//                  I_r[q][b] = l^{c-r}_b(x^c_q)
//   W  [c]         Gauss weights; IW [c] their inverses
//   PD2 [c-2][c]   P_2 D (c > 2), the derivative projected by two points
//   EO [3][...]    even-odd forms of V, VI (centrosymmetric, M[c-1-i][c-1-j]
//                  = M[i][j], the point sets being symmetric) and D (skew:
//                  = -M[i][j]); with h = c / 2, for rows i and columns j < h:
//                  A[i][j] = (M[i][j] + M[i][c-1-j]) / 2,
//                  B[i][j] = (M[i][j] - M[i][c-1-j]) / 2, C[i] = M[i][h]
//                  (odd c): out = M in is then, with e_j = in_j + in_{c-1-j}
//                  and o_j = in_j - in_{c-1-j}, p_i = A e + C_i in_h,
//                  q_i = B o, out_i = p_i + q_i, out_{c-1-i} = +-(p_i - q_i)
// The projection by r is exact because the c-point rule integrates the
// product of degrees c-1 and c-r-1.
#pragma once

#define DG_NMAX 8

#ifdef __CUDACC__
#define DG_HD __host__ __device__
#else
#define DG_HD
#endif

DG_HD constexpr int dg_red_len(int c, int r) { return c > r ? 2 * c * (c - r) : 0; }
// even-odd form of one centrosymmetric or skew-centrosymmetric c x c matrix
// (h = c / 2): A [h+1][h], B [h+1][h], C [h+1]
DG_HD constexpr int dg_eo_len(int c) { return 2 * (c / 2 + 1) * (c / 2) + (c / 2 + 1); }
// the projected derivative P_2 D (count c -> c - 2), when c > 2
DG_HD constexpr int dg_pd_len(int c) { return c > 2 ? (c - 2) * c : 0; }
DG_HD constexpr int dg_tab_block(int c) {
  return 3 * c * c + 2 * c + dg_red_len(c, 1) + dg_red_len(c, 2) + dg_red_len(c, 3) + 2 * c + 3 * dg_eo_len(c) +
         dg_pd_len(c);
}
DG_HD constexpr int dg_tab_base(int c) {
  return c <= 1 ? 0 : dg_tab_base(c - 1) + dg_tab_block(c - 1);
}
DG_HD constexpr int OFF_V(int c) { return dg_tab_base(c); }
DG_HD constexpr int OFF_VI(int c) { return dg_tab_base(c) + c * c; }
DG_HD constexpr int OFF_D(int c) { return dg_tab_base(c) + 2 * c * c; }
DG_HD constexpr int OFF_LF(int c) { return dg_tab_base(c) + 3 * c * c; }
// projection by r points (r = 1, 2, 3) from count c, and the prolongation
// from count c - r back to count c
DG_HD constexpr int OFF_PR(int c, int r) {
  return dg_tab_base(c) + 3 * c * c + 2 * c + (r > 1 ? dg_red_len(c, 1) : 0) +
         (r > 2 ? dg_red_len(c, 2) : 0);
}
DG_HD constexpr int OFF_IR(int c, int r) { return OFF_PR(c, r) + (c > r ? c * (c - r) : 0); }
DG_HD constexpr int OFF_W(int c) {
  return dg_tab_base(c) + 3 * c * c + 2 * c + dg_red_len(c, 1) + dg_red_len(c, 2) + dg_red_len(c, 3);
}
DG_HD constexpr int OFF_IW(int c) { return OFF_W(c) + c; }
// even-odd forms of V (which 0), VI (1) and D (2) of count c
DG_HD constexpr int OFF_EO(int c, int which) { return OFF_IW(c) + c + which * dg_eo_len(c); }
// PD2 [c-2][c] = P_2 D: the collocation derivative followed by the reference
// L2 projection onto c - 2 points (the two steps of a reduced Taylor term,
// Sec. 3.3, in one matrix)
DG_HD constexpr int OFF_PD2(int c) { return OFF_EO(c, 3); }

// Compact per-element data of affine elements with element-wise constant
// coefficients (see setup.cu): operator block and predictor block sizes.
constexpr int DG_AFF_OP = 48;
constexpr int DG_AFF_TCK = 16;
constexpr int DG_TAB_LEN = dg_tab_base(DG_NMAX + 1);

// Raw points for the geometry set-up: for each count c in [1, DG_NMAX],
// Gauss points, Gauss weights and (c >= 2) Gauss-Lobatto points at offset
// dg_pts_off(c) = c (c - 1) / 2 within each of three arrays.
DG_HD constexpr int dg_pts_off(int c) { return c * (c - 1) / 2; }
constexpr int DG_PTS_LEN = dg_pts_off(DG_NMAX + 2);

// Per-element strides (in values) of the operator's geometry arrays, padded
// to multiples of 8 values so that every element's block starts on a 32-byte
// boundary (bulk asynchronous copies need 16-byte alignment).
DG_HD constexpr int dg_pad8(int x) { return (x + 7) / 8 * 8; }
DG_HD constexpr int geo_stride_A(int n) { return dg_pad8(9 * n * n * n); }
DG_HD constexpr int geo_stride_M(int n) { return dg_pad8(2 * n * n * n); }
DG_HD constexpr int geo_stride_F(int n) { return dg_pad8(36 * n * n); }

namespace dg {

struct HostTables {
  double tab[DG_TAB_LEN];
  double xg[DG_PTS_LEN], wg[DG_PTS_LEN], xgl[DG_PTS_LEN];
};

// Fill all tables (idempotent). Returns 0 on success.
int build_tables(HostTables* t);

// Gauss-Lobatto points of count c (c >= 2), ascending, into x[c].
void gauss_lobatto(int c, double* x);

}  // namespace dg
