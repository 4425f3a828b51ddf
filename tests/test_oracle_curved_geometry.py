"""Exact pins of the oracle's curved geometry (Sec. 3: curved elements,
inverse Jacobians at the quadrature points, Nanson's formula on the faces).

* Free-stream preservation.  A constant state (p0, v0) has no jumps, so
  R(U) = 0 exactly iff the discrete cell integrals of w detJ J^-T grad(phi)
  equal the face integrals of w n|J_f| phi, i.e. iff the quadrature
  integrates both exactly (the divergence theorem holds for the exact
  integrals of a polynomial map, whose cofactor matrix is divergence free).
  For a map of degree q, detJ J^-T has degree <= 2q per direction, a basis
  derivative degree k - 1 in its own direction and k in the others, so the
  cell integrands have degree <= 2q + k - 1 per direction; the Nanson
  normal on a face has degree <= 2q - 1 there, times phi of degree k.  The
  (k+1)-point Gauss rule is exact up to degree 2k + 1, so both are exact
  when 2q + k - 1 <= 2k + 1, i.e. q <= (k + 2) / 2.  Then R = 0 to rounding
  on a curved periodic mesh with any coefficients and either flux; for
  larger q the quadrature error of the curved metric shows (the variational
  crime Sec. 3 accepts), which makes the pin sharp.
* An affine map described by geometry nodes of degree q > 1 gives the same
  operator as its degree-1 description.
* In 2D the cofactor entries are single derivatives of the map (degree q
  along one direction, q - 1 along the other), so the cell integrands have
  degree <= q + k - 1 and the face terms <= q - 1 + k: exact, and a
  constant state steady, for q <= k + 2, and not beyond.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import mesh2d
from oracle_helpers import SHEAR, generic_curving, generic_curving_2d, linear_map


def constant_state(E, n3, p0=0.7, v0=(0.3, -0.5, 0.2)):
    U = np.empty((E, 4, n3))
    U[:, 0] = p0
    U[:, 1:] = np.asarray(v0)[:, None]
    return U


def free_stream_residual(k, q, N, alpha, seed=3, oracle_cls=oracle.Oracle, mutate=None):
    """max |R(constant state)| on a generically curved periodic mesh with
    random element-wise polynomial coefficients."""
    mesh = synth.cube_mesh(N, q=q, periodic=True, deform=generic_curving(0.04))
    n3 = (k + 1) ** 3
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.6, 1.8, (N ** 3, n3))
    c = rng.uniform(0.6, 1.8, (N ** 3, n3))
    o = oracle_cls(mesh, k, rho, c, alpha)
    if mutate:
        mutate(o)
    return np.abs(o.apply(constant_state(N ** 3, n3))).max()


@pytest.mark.parametrize("k,q,N", [(1, 1, 3), (2, 1, 3), (2, 2, 3), (3, 2, 3), (4, 3, 2)])
@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_constant_state_is_steady_when_the_quadrature_is_exact(k, q, N, alpha):
    assert 2 * q + k - 1 <= 2 * k + 1
    assert free_stream_residual(k, q, N, alpha) < 5e-11


@pytest.mark.parametrize("k,q,N", [(2, 3, 3), (3, 3, 3), (4, 4, 2)])
def test_constant_state_drifts_when_the_metric_is_under_integrated(k, q, N):
    assert 2 * q + k - 1 > 2 * k + 1
    assert free_stream_residual(k, q, N, 1.0) > 1e-3


@pytest.mark.parametrize("k", [2, 3])
def test_high_degree_description_of_an_affine_map(k):
    N = 3
    rng = np.random.default_rng(21)
    n3 = (k + 1) ** 3
    rho = rng.uniform(0.6, 1.8, (N ** 3, n3))
    c = rng.uniform(0.6, 1.8, (N ** 3, n3))
    U = rng.standard_normal((N ** 3, 4, n3))
    R = []
    for q in (1, k, k + 2):
        mesh = synth.cube_mesh(N, q=q, periodic=True, deform=linear_map(SHEAR))
        R.append(oracle.Oracle(mesh, k, rho, c, 1.0).apply(U))
    scale = np.abs(R[0]).max()
    assert np.abs(R[1] - R[0]).max() < 1e-12 * scale
    assert np.abs(R[2] - R[0]).max() < 1e-12 * scale


def free_stream_residual_2d(k, q, N=4, alpha=1.0, seed=3):
    mesh = mesh2d.square_mesh(N, q=q, periodic=True, deform=generic_curving_2d(0.04))
    n2 = (k + 1) ** 2
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.6, 1.8, (N * N, n2))
    c = rng.uniform(0.6, 1.8, (N * N, n2))
    o = oracle.Oracle2D(mesh, k, rho, c, alpha)
    U = np.empty((N * N, 3, n2))
    U[:, 0] = 0.7
    U[:, 1] = 0.3
    U[:, 2] = -0.5
    return np.abs(o.apply(U)).max()


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_2d_constant_state_steady_up_to_q_k_plus_2(k):
    for q in range(1, k + 3):
        assert free_stream_residual_2d(k, q) < 5e-11, q
    assert free_stream_residual_2d(k, k + 3) > 1e-4
