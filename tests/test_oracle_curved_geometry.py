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


def linear_fields(x, rng):
    """p = a.x + b and v = B x + v0 at the points x [E, P, 3], packed as a
    state [E, 4, P], with the exact T_1 = -S u for constant rho, c:
    (-rho c^2 tr B, -a / rho), and T_j = 0 beyond (T_1 is constant)."""
    a, b = rng.standard_normal(3), rng.standard_normal()
    B, v0 = rng.standard_normal((3, 3)), rng.standard_normal(3)
    U = np.empty((x.shape[0], 4, x.shape[1]))
    U[:, 0] = x @ a + b
    U[:, 1:] = np.transpose(x @ B.T + v0, (0, 2, 1))
    return U, a, np.trace(B)


def curved_linear_case(k, seed=31):
    """A generically curved periodic mesh with geometry degree q = k, whose
    geometry nodes are the solution nodes, so a linear function of the
    discrete map is exactly a degree-k field; constant rho and c."""
    mesh = synth.cube_mesh(3, q=k, periodic=True, deform=generic_curving(0.04))
    n3 = (k + 1) ** 3
    rho0, c0 = 1.3, 0.8
    U, a, trB = linear_fields(np.asarray(mesh["nodes"]), np.random.default_rng(seed))
    T1 = np.empty_like(U)
    T1[:, 0] = -rho0 * c0 ** 2 * trB
    T1[:, 1:] = (-a / rho0)[None, :, None]
    return mesh, np.full((27, n3), rho0), np.full((27, n3), c0), U, T1


@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("red", [0, 2])
def test_tck_of_linear_fields_on_a_curved_mesh(k, red):
    """On a curved mesh the collocated gradient and divergence of a linear
    field of the discrete map are exact (grad_ref p = J^T a), so the first
    Taylor term is the constant -S u and the predictor is dt u + dt^2/2 T_1."""
    mesh, rho, c, U, T1 = curved_linear_case(k)
    o = oracle.Oracle(mesh, k, rho, c, 1.0)
    dt = 0.01
    Ubar, terms = o.tck(U, dt, red, return_terms=True)
    ref = dt * U + 0.5 * dt ** 2 * T1
    assert np.abs(Ubar - ref).max() < 1e-13 * np.abs(ref).max()
    m1, t1 = terms[1]
    assert m1 == k + 1 and np.abs(t1 - T1[:, :, :1]).max() < 1e-11 * np.abs(T1).max()
    m2, t2 = terms[2]  # the derivative of a constant: rounding only (later terms differentiate that again)
    assert t2 is None or np.abs(t2).max() < 1e-9 * np.abs(T1).max()
