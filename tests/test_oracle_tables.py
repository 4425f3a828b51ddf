"""Pins of the oracle's 1D point sets and Lagrange polynomials (Sec. 3)."""
import math

import numpy as np
import pytest

from oracle import gauss_1d, gauss_lobatto_1d, lagrange_1d, lagrange_deriv_1d


def test_gauss_closed_forms():
    x, w = gauss_1d(2)
    assert np.allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [1, 1], atol=1e-15)
    x, w = gauss_1d(3)
    assert np.allclose(x, [-math.sqrt(0.6), 0, math.sqrt(0.6)], atol=1e-15)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


def test_gauss_lobatto_closed_forms():
    assert np.allclose(gauss_lobatto_1d(2), [-1, 1])
    assert np.allclose(gauss_lobatto_1d(3), [-1, 0, 1], atol=1e-15)
    # n = 4: roots of P_3' = (15 x^2 - 3)/2 -> +-1/sqrt(5)
    assert np.allclose(gauss_lobatto_1d(4), [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], atol=1e-15)
    # n = 5: roots of P_4' -> 0, +-sqrt(3/7)
    assert np.allclose(gauss_lobatto_1d(5), [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], atol=1e-15)


@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_exactness_degree(n):
    x, w = gauss_1d(n)
    assert abs(w.sum() - 2.0) < 1e-14
    for p in range(0, 2 * n):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.sum(w * x ** p) - exact) < 1e-13, (n, p)
    # degree 2n is no longer integrated exactly
    p = 2 * n
    assert abs(np.sum(w * x ** p) - 2.0 / (p + 1)) > 1e-6


@pytest.mark.parametrize("n", range(2, 10))
def test_lagrange_interpolates_and_differentiates(n):
    rng = np.random.default_rng(n)
    for nodes in (gauss_1d(n)[0], gauss_lobatto_1d(n)):
        c = rng.normal(size=n)                  # random degree n-1 polynomial
        poly = np.polynomial.Polynomial(c)
        xs = np.linspace(-1, 1, 17)
        L = lagrange_1d(nodes, xs)
        assert np.allclose(L @ poly(nodes), poly(xs), atol=1e-12)
        dL = lagrange_deriv_1d(nodes, xs)
        assert np.allclose(dL @ poly(nodes), poly.deriv()(xs), atol=1e-10)
        # Kronecker property at the nodes
        assert np.allclose(lagrange_1d(nodes, nodes), np.eye(n), atol=1e-13)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_gl_projection_of_gauss_values_is_their_interpolant(n):
    """The reading behind the predictor without the basis change (Sec. 3.2,
    Alg. 1): with the mass matrix defined by the same n-point Gauss rule and
    any positive point weights (w det J varies from point to point), the L2
    projection onto the GL basis of values f known at the Gauss points,
    M^-1 V^T W f with M = V^T W V, equals their interpolant V^-1 f.  V[q, a]
    is GL function a at Gauss point q.  Checked in 1D and as a 3D tensor
    product with a non-separable weight."""
    rng = np.random.default_rng(n)
    x, w = gauss_1d(n)
    g = gauss_lobatto_1d(n)
    V = np.asarray(lagrange_1d(g, x))               # V[q, a] = l_a(x_q)
    assert np.allclose(V.sum(axis=1), 1.0)           # partition of unity at every point
    f = rng.standard_normal(n)
    W = np.diag(w * rng.uniform(0.5, 2.0, n))
    proj = np.linalg.solve(V.T @ W @ V, V.T @ W @ f)
    assert np.allclose(proj, np.linalg.solve(V, f), rtol=0, atol=1e-12 * np.abs(f).max())
    V3 = np.kron(np.kron(V, V), V)
    f3 = rng.standard_normal(n ** 3)
    W3 = np.diag(np.kron(np.kron(w, w), w) * rng.uniform(0.5, 2.0, n ** 3))
    proj3 = np.linalg.solve(V3.T @ W3 @ V3, V3.T @ W3 @ f3)
    assert np.allclose(proj3, np.linalg.solve(V3, f3), rtol=0, atol=1e-10 * np.abs(f3).max())
    # a genuinely smaller quadrature (n-1 points) would not reproduce the
    # interpolant: the identity rests on the square, invertible V
    if n > 2:
        xs, ws = gauss_1d(n - 1)
        Vs = np.asarray(lagrange_1d(g, xs))           # (n-1) x n
        Ms = Vs.T @ np.diag(ws) @ Vs
        assert np.linalg.matrix_rank(Ms) < n
