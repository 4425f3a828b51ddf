// 1D point sets and Lagrange matrices in FP64 (see tables.h).
// Gauss points: Newton's method on the Legendre polynomial P_c with
// Chebyshev-type initial guesses; weights 2 / ((1 - x^2) P_c'(x)^2).
// Gauss-Lobatto points: end points plus the roots of P'_{c-1}, Newton's
// method with P'' from Legendre's equation.  Lagrange values by the product
// formula, collocation derivatives by barycentric weights.
#include "tables.h"

#include <cmath>
#include <vector>

namespace dg {
namespace {

// P_n(x) and P_n'(x) by the three-term recurrence.
void legendre(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int j = 2; j <= n; ++j) {
    double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

void gauss(int c, double* x, double* w) {
  for (int i = 0; i < c; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (c + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(c, z, &p, &dp);
      double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p, dp;
    legendre(c, z, &p, &dp);
    x[c - 1 - i] = z;  // ascending
    w[c - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  for (int i = 0; i < c / 2; ++i) {  // enforce exact symmetry
    double a = 0.5 * (x[c - 1 - i] - x[i]);
    x[i] = -a;
    x[c - 1 - i] = a;
    double ww = 0.5 * (w[i] + w[c - 1 - i]);
    w[i] = w[c - 1 - i] = ww;
  }
  if (c % 2) x[c / 2] = 0.0;
}

double lagrange(const double* nodes, int c, int a, double x) {
  double v = 1.0;
  for (int b = 0; b < c; ++b)
    if (b != a) v *= (x - nodes[b]) / (nodes[a] - nodes[b]);
  return v;
}

}  // namespace

void gauss_lobatto(int c, double* x) {
  const int N = c - 1;  // polynomial degree
  x[0] = -1.0;
  x[c - 1] = 1.0;
  for (int i = 1; i < c - 1; ++i) {
    double z = -std::cos(M_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(N, z, &p, &dp);
      double d2p = (2.0 * z * dp - N * (N + 1.0) * p) / (1.0 - z * z);
      double dz = dp / d2p;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  for (int i = 0; i < c / 2; ++i) {
    double a = 0.5 * (x[c - 1 - i] - x[i]);
    x[i] = -a;
    x[c - 1 - i] = a;
  }
  if (c % 2) x[c / 2] = 0.0;
}

int build_tables(HostTables* t) {
  for (int i = 0; i < DG_TAB_LEN; ++i) t->tab[i] = 0.0;
  for (int i = 0; i < DG_PTS_LEN; ++i) t->xg[i] = t->wg[i] = t->xgl[i] = 0.0;
  std::vector<double> xg(DG_NMAX + 1), wg(DG_NMAX + 1), xgl(DG_NMAX + 1), xr(DG_NMAX + 1),
      wr(DG_NMAX + 1);
  for (int c = 1; c <= DG_NMAX; ++c) {
    gauss(c, xg.data(), wg.data());
    for (int i = 0; i < c; ++i) {
      t->xg[dg_pts_off(c) + i] = xg[i];
      t->wg[dg_pts_off(c) + i] = wg[i];
    }
    double* V = t->tab + OFF_V(c);
    double* VI = t->tab + OFF_VI(c);
    double* D = t->tab + OFF_D(c);
    double* LF = t->tab + OFF_LF(c);
    if (c >= 2) {
      gauss_lobatto(c, xgl.data());
      for (int i = 0; i < c; ++i) t->xgl[dg_pts_off(c) + i] = xgl[i];
      for (int q = 0; q < c; ++q)
        for (int a = 0; a < c; ++a) {
          V[q * c + a] = lagrange(xgl.data(), c, a, xg[q]);
          VI[q * c + a] = lagrange(xg.data(), c, a, xgl[q]);  // VI[a'=q][q'=a]
        }
    } else {
      V[0] = VI[0] = 1.0;
    }
    // barycentric weights of the Gauss nodes
    std::vector<double> lam(c);
    for (int a = 0; a < c; ++a) {
      double p = 1.0;
      for (int b = 0; b < c; ++b)
        if (b != a) p *= (xg[a] - xg[b]);
      lam[a] = 1.0 / p;
    }
    for (int q = 0; q < c; ++q) {
      double diag = 0.0;
      for (int a = 0; a < c; ++a) {
        if (a == q) continue;
        D[q * c + a] = (lam[a] / lam[q]) / (xg[q] - xg[a]);
        diag += 1.0 / (xg[q] - xg[a]);
      }
      D[q * c + q] = diag;
    }
    for (int a = 0; a < c; ++a) {
      LF[a] = lagrange(xg.data(), c, a, -1.0);
      LF[c + a] = lagrange(xg.data(), c, a, 1.0);
      t->tab[OFF_W(c) + a] = wg[a];
      t->tab[OFF_IW(c) + a] = 1.0 / wg[a];
    }
    // even-odd forms of V, VI and D (see tables.h)
    {
      const int h = c / 2;
      const double* mats[3] = {V, VI, D};
      for (int w = 0; w < 3; ++w) {
        const double* M = mats[w];
        double* E = t->tab + OFF_EO(c, w);
        for (int i = 0; i < dg_eo_len(c); ++i) E[i] = 0.0;
        double* EA = E;
        double* EB = E + (h + 1) * h;
        double* EC = E + 2 * (h + 1) * h;
        for (int i = 0; i <= h && i < c; ++i) {
          for (int j = 0; j < h; ++j) {
            EA[i * h + j] = 0.5 * (M[i * c + j] + M[i * c + (c - 1 - j)]);
            EB[i * h + j] = 0.5 * (M[i * c + j] - M[i * c + (c - 1 - j)]);
          }
          if (c % 2 == 1) EC[i] = M[i * c + h];
        }
      }
    }
    // P_2 D: the projected derivative, summed in FP64
    if (c > 2) {
      const int r = c - 2;
      gauss(r, xr.data(), wr.data());
      double* PD = t->tab + OFF_PD2(c);
      for (int a = 0; a < r; ++a)
        for (int b = 0; b < c; ++b) {
          double sum = 0.0;
          for (int q = 0; q < c; ++q)
            sum += wg[q] * lagrange(xr.data(), r, a, xg[q]) / wr[a] * D[q * c + b];
          PD[a * c + b] = sum;
        }
    }
    for (int red = 1; red <= 3; ++red) {
      if (c <= red) continue;
      const int r = c - red;
      gauss(r, xr.data(), wr.data());
      double* P = t->tab + OFF_PR(c, red);
      double* IU = t->tab + OFF_IR(c, red);
      for (int a = 0; a < r; ++a)
        for (int b = 0; b < c; ++b)
          P[a * c + b] = wg[b] * lagrange(xr.data(), r, a, xg[b]) / wr[a];
      for (int q = 0; q < c; ++q)
        for (int b = 0; b < r; ++b) IU[q * r + b] = lagrange(xr.data(), r, b, xg[q]);
    }
  }
  return 0;
}

}  // namespace dg
