"""The GPU's curved geometry against exact properties and the oracle.

* Free-stream preservation: for a map of degree q <= (k + 2) / 2 the
  (k+1)-point Gauss rule integrates the metric terms exactly, so a constant
  state has R = 0 to rounding and stays constant under LSRK and ADER steps
  (the oracle pin in test_oracle_curved_geometry.py).  This checks the GPU's
  own geometry set-up (Jacobians, inverse-mass diagonals, Nanson normals,
  orientation of the face data) without reference to the oracle, in both
  storage bases and both precisions.
* A generic curving (different displacement per coordinate) at q = k:
  operator and one step of each method at oracle parity.
* The 2D path: a constant state is steady for q <= k + 2.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1805_03981_gb300 as dgw
from synth import mesh2d
from gpu_helpers import rel_l2
from oracle_helpers import generic_curving, generic_curving_2d

pytestmark = pytest.mark.gpu


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _problem(k, q, N, seed=3):
    mesh = synth.cube_mesh(N, q=q, periodic=True, deform=generic_curving(0.04))
    n3 = (k + 1) ** 3
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.6, 1.8, (N ** 3, n3))
    c = rng.uniform(0.6, 1.8, (N ** 3, n3))
    return mesh, rho, c


@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
@pytest.mark.parametrize("basis", [dgw.BASIS_GL, dgw.BASIS_G])
@pytest.mark.parametrize("k,q,N", [(2, 2, 3), (3, 2, 3), (4, 3, 2), (5, 3, 2)])
def test_constant_state_is_steady(k, q, N, basis, prec):
    torch = _cuda()
    assert 2 * q + k - 1 <= 2 * k + 1
    mesh, rho, c = _problem(k, q, N)
    s = dgw.Solver(mesh, k, prec, 1.0, rho, c)
    s.set_basis(basis)
    n3 = (k + 1) ** 3
    U0 = np.empty((N ** 3, 4, n3))
    U0[:, 0] = 0.7
    U0[:, 1:] = np.array([0.3, -0.5, 0.2])[:, None]
    tol = 5e-11 if prec == dgw.DG_FP64 else 2e-4   # |R| of a random state is O(10^2)
    R = s.apply(s.to_device(U0))
    torch.cuda.synchronize()
    assert R.abs().max().item() < tol
    dt = 0.2 / (N * k ** 1.5) / 1.8
    step_tol = 1e-13 if prec == dgw.DG_FP64 else 2e-6
    for method in ("lsrk", "ader"):
        U = s.to_device(U0)
        if method == "lsrk":
            s.step_lsrk(U, dt, 3)
        else:
            s.step_ader(U, dt, 3, 2)
        torch.cuda.synchronize()
        assert np.abs(U.double().cpu().numpy() - U0).max() < step_tol, method
    s.close()


@pytest.mark.parametrize("basis", [dgw.BASIS_GL, dgw.BASIS_G])
def test_generic_curving_at_oracle_parity(basis):
    torch = _cuda()
    k, q, N = 3, 3, 3
    mesh, rho, c = _problem(k, q, N, seed=8)
    o = oracle.Oracle(mesh, k, rho, c, 1.0)
    s = dgw.Solver(mesh, k, dgw.DG_FP64, 1.0, rho, c)
    s.set_basis(basis)
    U0 = np.random.default_rng(4).standard_normal((N ** 3, 4, (k + 1) ** 3))
    R = s.apply(s.to_device(U0))
    torch.cuda.synchronize()
    assert rel_l2(R.cpu().numpy(), o.apply(U0)) < 1e-12
    dt = 0.1 / (N * k ** 1.5) / 1.8
    U = s.to_device(U0)
    s.step_lsrk(U, dt, 2)
    torch.cuda.synchronize()
    assert rel_l2(U.cpu().numpy(), o.lsrk(U0, dt, 2)) < 1e-12
    U = s.to_device(U0)
    s.step_ader(U, dt, 2, 2)
    torch.cuda.synchronize()
    assert rel_l2(U.cpu().numpy(), o.ader(U0, dt, 2, 2)) < 1e-12
    s.close()


@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
@pytest.mark.parametrize("k,q", [(1, 3), (3, 5), (5, 7)])
def test_2d_constant_state_is_steady(k, q, prec):
    torch = _cuda()
    N = 4
    mesh = mesh2d.square_mesh(N, q=q, periodic=True, deform=generic_curving_2d(0.04))
    n2 = (k + 1) ** 2
    rng = np.random.default_rng(5)
    rho = rng.uniform(0.6, 1.8, (N * N, n2))
    c = rng.uniform(0.6, 1.8, (N * N, n2))
    s = dgw.Solver2D(mesh, k, prec, 1.0, rho, c)
    U0 = np.empty((N * N, 3, n2))
    U0[:, 0] = 0.7
    U0[:, 1] = 0.3
    U0[:, 2] = -0.5
    R = s.apply(s.to_device(U0))
    torch.cuda.synchronize()
    assert R.abs().max().item() < (5e-11 if prec == dgw.DG_FP64 else 2e-4)
    dt = 0.2 / (N * k ** 1.5) / 1.8
    for method in ("lsrk", "ader"):
        U = s.to_device(U0)
        if method == "lsrk":
            s.step_lsrk(U, dt, 3)
        else:
            s.step_ader(U, dt, 3, 2)
        torch.cuda.synchronize()
        assert np.abs(U.double().cpu().numpy() - U0).max() < (1e-13 if prec == dgw.DG_FP64 else 2e-6), method
    s.close()


@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
@pytest.mark.parametrize("k", [2, 3, 5])
@pytest.mark.parametrize("red", [0, 2])
def test_tck_of_linear_fields_closed_form(k, red, prec):
    """The predictor of a linear field of the discrete map on a curved mesh
    (geometry degree k, constant coefficients) is dt u + dt^2/2 T_1 with the
    constant T_1 = (-rho c^2 tr B, -a / rho) (the oracle pin in
    test_oracle_curved_geometry.py): dg_tck (GL states) directly, and the
    Gauss-point predictors in both forms through one ADER step, whose
    increment must then be R(dt u + dt^2/2 T_1)."""
    torch = _cuda()
    from test_oracle_curved_geometry import curved_linear_case
    mesh, rho, c, U, T1 = curved_linear_case(k)
    s = dgw.Solver(mesh, k, prec, 1.0, rho, c)
    dt = 0.01
    ref = dt * U + 0.5 * dt ** 2 * T1
    tol = 1e-13 if prec == dgw.DG_FP64 else 2e-6
    Ub = s.tck(s.to_device(U), dt, red)
    torch.cuda.synchronize()
    assert np.abs(Ub.double().cpu().numpy() - ref).max() < tol * np.abs(ref).max()
    incr = s.apply(s.to_device(ref)).double().cpu().numpy()
    s.set_basis(dgw.BASIS_G)
    for pred in (dgw.PRED_LINES, dgw.PRED_COLUMNS):
        s.set_predictor_kernel(pred)
        V = s.to_device(U)
        s.step_ader(V, dt, 1, red)
        torch.cuda.synchronize()
        got = V.double().cpu().numpy() - U
        assert np.abs(got - incr).max() < (1e-11 if prec == dgw.DG_FP64 else 2e-4) * np.abs(incr).max(), pred
    s.close()
