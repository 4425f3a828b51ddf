"""Pins of the oracle's diagnostics (Sec. 4.7): the discrete energy
E = 1/2 U^T M U and the relative L2 errors of pressure and velocity.

* The energy equals 1/2 U^T M U with the dense mass matrices, whose entries
  are pinned against exact integrals elsewhere, on curved meshes with
  variable coefficients and rotated element frames (3D and 2D).
* Closed forms: on a graded affine mesh of the unit cube (boxes of unequal
  size, so a dropped det J or a wrong volume weight shows), polynomial
  coefficient and state fields make every integrand a low-degree
  polynomial, and the energy is 27/16 exactly.
* A plane wave with rho = 2, c = 3 carries the energy 1/(2 rho c^2) = 1/36
  per unit volume; the discrete energy approaches it under refinement.
* l2_error: a constant pressure 1/2 against the exact field x has relative
  error 1/2; the velocity (x, 0, 0) against (x, y, 0) has sqrt(1/2); both on
  the graded mesh.  A polynomial of degree <= k stored by its nodal values
  has zero error on affine meshes.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import Oracle2D
from oracle.basis import gauss_lobatto_1d
from synth import mesh2d


def _graded(x):
    """Monotone map of [0, 1] onto itself: applied to the corner nodes of a
    cube mesh it gives axis-aligned boxes of unequal size."""
    return 0.5 * (x + x * x)


def _box_nodes(mesh, k, dim):
    """GL solution-node positions [E, n^dim, dim] of axis-aligned box
    elements, from the corner nodes (reference axis d along global axis d)."""
    xgl = gauss_lobatto_1d(k + 1)
    n = k + 1
    idx = np.arange(n ** dim)
    ref = np.stack([xgl[(idx // n ** d) % n] for d in range(dim)], axis=1)   # first axis fastest
    lo = mesh["nodes"].min(axis=1)
    hi = mesh["nodes"].max(axis=1)
    return lo[:, None, :] + 0.5 * (ref[None] + 1.0) * (hi - lo)[:, None, :]


def _graded_mesh(dim, N):
    if dim == 3:
        return synth.cube_mesh(N, q=1, periodic=False, deform=_graded)
    return mesh2d.square_mesh(N, q=1, periodic=False, deform=_graded)


def _make(dim, mesh, k, rho, c):
    cls = oracle.Oracle if dim == 3 else Oracle2D
    return cls(mesh, k, rho, c, 1.0)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [3, 2])
def test_energy_is_half_mass_inner_product(dim):
    k, N = 3, 3 if dim == 3 else 4
    rng = np.random.default_rng(21)
    if dim == 3:
        frames = synth.mesh.random_frames(N ** 3, rng)
        mesh = synth.cube_mesh(N, q=k, periodic=False, deform=synth.mesh.curving(0.05), frames=frames)
        E, npts, nf = N ** 3, (k + 1) ** 3, 4
    else:
        frames = mesh2d.random_frames_2d(N * N, rng)
        mesh = mesh2d.square_mesh(N, q=k, periodic=False, deform=mesh2d.curving_2d(0.05), frames=frames)
        E, npts, nf = N * N, (k + 1) ** 2, 3
    rho = rng.uniform(0.5, 2.0, size=(E, npts))
    c = rng.uniform(0.5, 2.0, size=(E, npts))
    o = _make(dim, mesh, k, rho, c)
    U = rng.uniform(-1, 1, size=(E, nf, npts))
    e = o.energy(U)
    assert e > 0
    assert abs(e - 0.5 * o.mass_inner(U, U)) <= 1e-13 * e


@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("k", [1, 3])
def test_energy_closed_form_on_graded_mesh(dim, k):
    """rho = 1 + x, c = 2, p = 1 + x, v = (1, 1, 0): the density
    rho |v|^2 + p^2/(rho c^2) = (2 + 1/4)(1 + x), so E = 1/2 * 9/4 * 3/2 = 27/16
    over the unit cube (or square)."""
    N = 3
    mesh = _graded_mesh(dim, N)
    x = _box_nodes(mesh, k, dim)
    E, npts = x.shape[0], x.shape[1]
    rho = 1.0 + x[..., 0]
    c = np.full((E, npts), 2.0)
    U = np.zeros((E, dim + 1, npts))
    U[:, 0] = 1.0 + x[..., 0]
    U[:, 1] = 1.0
    U[:, 2] = 1.0
    o = _make(dim, mesh, k, rho, c)
    assert abs(o.energy(U) - 27.0 / 16.0) < 1e-13


@pytest.mark.parametrize("dim", [3, 2])
def test_energy_of_plane_wave_converges_to_closed_form(dim):
    """p = cos(kv.x), v = p/(rho c) kv/|kv| with rho = 2, c = 3: the energy
    density is p^2/(rho c^2), whose mean over the periodic unit cell is
    1/(2 rho c^2) = 1/36."""
    rho0, c0, k = 2.0, 3.0, 2
    kv = np.full(dim, 2 * np.pi)
    errs = []
    for N in (2, 4, 8):
        if dim == 3:
            mesh = synth.cube_mesh(N, q=1, periodic=True)
            x = synth.solution_node_positions(mesh, k)
        else:
            mesh = mesh2d.square_mesh(N, q=1, periodic=True)
            x = mesh2d.solution_node_positions_2d(mesh, k)
        E, npts = x.shape[0], x.shape[1]
        p = np.cos(x @ kv)
        U = np.zeros((E, dim + 1, npts))
        U[:, 0] = p
        for d in range(dim):
            U[:, 1 + d] = p / (rho0 * c0) * kv[d] / np.linalg.norm(kv)
        o = _make(dim, mesh, k, np.full((E, npts), rho0), np.full((E, npts), c0))
        errs.append(abs(o.energy(U) - 1.0 / 36.0) * 36.0)
    assert errs[-1] < 5e-3, errs
    assert errs[1] < errs[0] / 4 and errs[2] < errs[1] / 4, errs


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [3, 2])
def test_l2_error_closed_form_on_graded_mesh(dim):
    """p_h = 1/2 against p = x: int (1/2 - x)^2 / int x^2 = (1/12)/(1/3), so the
    relative error is 1/2; v_h = (x, 0, ..) against v = (x, y, ..):
    int y^2 / int (x^2 + y^2) = 1/2, error sqrt(1/2)."""
    k, N = 2, 3
    mesh = _graded_mesh(dim, N)
    x = _box_nodes(mesh, k, dim)
    E, npts = x.shape[0], x.shape[1]
    ones = np.ones((E, npts))
    o = _make(dim, mesh, k, ones, ones)
    U = np.zeros((E, dim + 1, npts))
    U[:, 0] = 0.5
    U[:, 1] = x[..., 0]

    def exact(xx, t):
        out = np.zeros(xx.shape[:-1] + (dim + 1,))
        out[..., 0] = xx[..., 0]
        out[..., 1] = xx[..., 0]
        out[..., 2] = xx[..., 1]
        return out
    ep, ev = o.l2_error(U, exact, 0.0)
    assert abs(ep - 0.5) < 1e-13, ep
    assert abs(ev - np.sqrt(0.5)) < 1e-13, ev


@pytest.mark.parametrize("dim", [3, 2])
def test_l2_error_vanishes_for_stored_polynomial(dim):
    """A field of degree <= k in x stored by its GL nodal values is the
    interpolant exactly on affine elements: zero error."""
    k, N = 3, 2
    rng = np.random.default_rng(5)
    if dim == 3:
        A = np.array([[1.0, 0.2, 0.1], [0.05, 0.9, 0.15], [-0.1, 0.07, 1.1]])
        mesh = synth.cube_mesh(N, q=1, periodic=False, deform=lambda y: y @ A.T)
        x = synth.solution_node_positions(mesh, k)
    else:
        A = np.array([[1.0, 0.3], [-0.2, 0.9]])
        mesh = mesh2d.square_mesh(N, q=1, periodic=False, deform=lambda y: y @ A.T)
        x = mesh2d.solution_node_positions_2d(mesh, k)
    coef = rng.uniform(-1, 1, size=(dim + 1, dim, k + 1))

    def exact(xx, t):
        out = np.zeros(xx.shape[:-1] + (dim + 1,))
        for f in range(dim + 1):
            for d in range(dim):
                out[..., f] += np.polynomial.polynomial.polyval(xx[..., d], coef[f, d])
        return out
    E, npts = x.shape[0], x.shape[1]
    ones = np.ones((E, npts))
    o = _make(dim, mesh, k, ones, ones)
    U = np.transpose(exact(x, 0.0), (0, 2, 1)).copy()
    ep, ev = o.l2_error(U, exact, 0.0)
    assert ep < 1e-13 and ev < 1e-13, (ep, ev)
