"""1D point sets and Lagrange polynomials (oracle; test infrastructure only).

Sec. 3 of the paper integrates with Gauss quadrature on k+1 points per
direction; Sec. 3.1-3.2 use Lagrange bases with nodes either in those Gauss
points (basis "G") or in the k+1 Gauss-Lobatto points (basis "GL").

Pinned by tests/test_oracle_tables.py: closed-form points and weights for
n = 2, 3, polynomial exactness up to degree 2n-1 and failure at 2n,
interpolation and differentiation of polynomials.
"""
import numpy as np


def gauss_1d(n):
    """n-point Gauss-Legendre points (ascending) and weights on [-1, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return np.asarray(x, float), np.asarray(w, float)


def gauss_lobatto_1d(n):
    """n-point Gauss-Lobatto points (ascending) on [-1, 1]: the end points and
    the roots of P'_{n-1}, each root refined by Newton's method."""
    if n == 2:
        return np.array([-1.0, 1.0])
    P = np.polynomial.legendre.Legendre.basis(n - 1)
    dP, d2P = P.deriv(), P.deriv(2)
    r = np.sort(np.real(dP.roots()))
    for _ in range(4):
        r = r - dP(r) / d2P(r)
    return np.concatenate(([-1.0], r, [1.0]))


def lagrange_1d(nodes, x):
    """L[i, a] = l_a(x_i), the Lagrange polynomials on ``nodes`` at points x,
    by the product formula prod_{b != a} (x - x_b) / (x_a - x_b)."""
    nodes = np.asarray(nodes, float)
    x = np.atleast_1d(np.asarray(x, float))
    m = len(nodes)
    L = np.ones((len(x), m))
    for a in range(m):
        for b in range(m):
            if b != a:
                L[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
    return L


def lagrange_deriv_1d(nodes, x):
    """dL[i, a] = l_a'(x_i) by the product rule:
    l_a' = sum_{c != a} 1/(x_a - x_c) prod_{b != a, c} (x - x_b)/(x_a - x_b)."""
    nodes = np.asarray(nodes, float)
    x = np.atleast_1d(np.asarray(x, float))
    m = len(nodes)
    dL = np.zeros((len(x), m))
    for a in range(m):
        for c in range(m):
            if c == a:
                continue
            term = np.full(len(x), 1.0 / (nodes[a] - nodes[c]))
            for b in range(m):
                if b != a and b != c:
                    term *= (x - nodes[b]) / (nodes[a] - nodes[b])
            dL[:, a] += term
    return dL


def tensor_points(x1d):
    """[m^3, 3] tensor-product points, first coordinate fastest."""
    m = len(x1d)
    i = np.arange(m ** 3)
    return np.stack([x1d[i % m], x1d[(i // m) % m], x1d[i // (m * m)]], axis=1)


def tensor_weights(w1d):
    m = len(w1d)
    i = np.arange(m ** 3)
    return w1d[i % m] * w1d[(i // m) % m] * w1d[i // (m * m)]


def basis_3d(nodes1d, pts):
    """phi[q, a] = 3D tensor Lagrange basis on ``nodes1d`` (a = a0 + n a1 +
    n^2 a2) evaluated at reference points pts [Q, 3]."""
    n = len(nodes1d)
    L = [lagrange_1d(nodes1d, pts[:, d]) for d in range(3)]
    a = np.arange(n ** 3)
    return L[0][:, a % n] * L[1][:, (a // n) % n] * L[2][:, a // (n * n)]


def basis_grad_3d(nodes1d, pts):
    """dphi[d, q, a] = d/dxi_d of the 3D tensor Lagrange basis at pts."""
    n = len(nodes1d)
    L = [lagrange_1d(nodes1d, pts[:, d]) for d in range(3)]
    D = [lagrange_deriv_1d(nodes1d, pts[:, d]) for d in range(3)]
    a = np.arange(n ** 3)
    i0, i1, i2 = a % n, (a // n) % n, a // (n * n)
    return np.stack([D[0][:, i0] * L[1][:, i1] * L[2][:, i2],
                     L[0][:, i0] * D[1][:, i1] * L[2][:, i2],
                     L[0][:, i0] * L[1][:, i1] * D[2][:, i2]])
