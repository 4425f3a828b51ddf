"""Pins of the oracle's operator R(U) = -M^-1 K U (Sec. 2.1, Eqs. (2)-(3)).

* Polynomial consistency: for a global polynomial field of degree <= k, in
  elements whose neighbours all see the same polynomial (away from the
  periodic seam), R equals -S u of Eq. (1) exactly, for any flux parameter.
* Energy identity: on affine meshes with arbitrary (even discontinuous)
  coefficients, U^T M R(U) = 0 for the central flux and < 0 for upwind,
  with walls included.
* Invariance under relabelled element axes (orientation codes).
"""
import numpy as np
import pytest

import synth
import oracle
from oracle.dg import face_points, orient_perm
from oracle_helpers import SHEAR, linear_map


def _poly_fields(x, rng, k):
    """Random total-degree <= k polynomials (p, vx, vy, vz) with gradients
    (total degree is what an affine map keeps inside the element space)."""
    coefs = rng.normal(size=(4, k + 1, k + 1, k + 1))
    a, b, c = np.meshgrid(np.arange(k + 1), np.arange(k + 1), np.arange(k + 1), indexing="ij")
    coefs[:, (a + b + c) > k] = 0.0
    out = np.zeros(x.shape[:-1] + (4,))
    grad = np.zeros(x.shape[:-1] + (4, 3))
    pw = np.arange(k + 1)
    P = [x[..., d, None] ** pw for d in range(3)]                       # x_d^a
    dP = [pw * x[..., d, None] ** np.maximum(pw - 1, 0) for d in range(3)]
    # P[d][..., a] = x_d^a
    for f in range(4):
        C = coefs[f]
        out[..., f] = np.einsum("...a,...b,...c,abc->...", P[0], P[1], P[2], C)
        grad[..., f, 0] = np.einsum("...a,...b,...c,abc->...", dP[0], P[1], P[2], C)
        grad[..., f, 1] = np.einsum("...a,...b,...c,abc->...", P[0], dP[1], P[2], C)
        grad[..., f, 2] = np.einsum("...a,...b,...c,abc->...", P[0], P[1], dP[2], C)
    return out, grad


@pytest.mark.parametrize("k,alpha", [(1, 1.0), (2, 0.0), (3, 1.0), (4, 0.5)])
def test_polynomial_consistency_interior(k, alpha):
    rng = np.random.default_rng(10 + k)
    N = 4
    mesh = synth.cube_mesh(N, q=1, periodic=True, deform=linear_map(SHEAR))
    x = synth.solution_node_positions(mesh, k)
    rho0, c0 = 1.3, 0.7
    n3 = (k + 1) ** 3
    o = oracle.Oracle(mesh, k, np.full((N ** 3, n3), rho0), np.full((N ** 3, n3), c0), alpha)
    u, g = _poly_fields(x, rng, k)
    U = np.transpose(u, (0, 2, 1)).copy()
    R = o.apply(U)
    # -S u: R_v = -(1/rho) grad p, R_p = -rho c^2 div v
    Rex = np.zeros_like(U)
    Rex[:, 1:] = -np.transpose(g[:, :, 0, :], (0, 2, 1)) / rho0
    Rex[:, 0] = -rho0 * c0 ** 2 * (g[:, :, 1, 0] + g[:, :, 2, 1] + g[:, :, 3, 2])
    interior = [e for e in range(N ** 3)
                if all(1 <= v <= N - 2 for v in (e % N, (e // N) % N, e // (N * N)))]
    scale = np.abs(Rex[interior]).max()
    err = np.abs(R[interior] - Rex[interior]).max() / scale
    assert err < 1e-11, err
    # the seam elements do see the jump: not a trivially local operator
    assert np.abs(R - Rex).max() / scale > 1e-3


@pytest.mark.parametrize("alpha", [0.0, 1.0])
@pytest.mark.parametrize("periodic", [True, (True, False, False), False])
def test_energy_identity_affine(alpha, periodic):
    k, N = 3, 3
    n3 = (k + 1) ** 3
    rng = np.random.default_rng(7)
    mesh = synth.cube_mesh(N, q=1, periodic=periodic, deform=linear_map(SHEAR))
    rho = rng.uniform(0.5, 2.0, size=(N ** 3, n3))     # discontinuous between elements
    c = rng.uniform(0.5, 2.0, size=(N ** 3, n3))
    o = oracle.Oracle(mesh, k, rho, c, alpha)
    U = rng.uniform(-1, 1, size=(N ** 3, 4, n3))
    R = o.apply(U)
    dEdt = o.mass_inner(U, R)
    scale = np.sqrt(o.mass_inner(U, U) * o.mass_inner(R, R))
    if alpha == 0.0:
        assert abs(dEdt) / scale < 1e-13, dEdt / scale
    else:
        assert dEdt / scale < -1e-3


def test_orientation_codes_match_physical_points():
    """Every interior face point of an element and its image on the
    neighbour (through nbr_face and orient) are the same physical point, up
    to the periodic shift."""
    k = 3
    mesh = synth.cube_mesh(3, q=2, periodic=True, deform=synth.mesh.curving(0.04),
                           frames=synth.mesh.random_frames(27, np.random.default_rng(3)))
    n3 = (k + 1) ** 3
    o = oracle.Oracle(mesh, k, np.ones((27, n3)), np.ones((27, n3)))
    xg = o.xg
    nontrivial = 0
    for e in range(27):
        for f in range(6):
            en, fn, code = mesh["nbr"][e, f], mesh["nbr_face"][e, f], mesh["orient"][e, f]
            nontrivial += code != 0
            xo = o.positions(face_points(f, xg))[e]
            xn = o.positions(face_points(fn, xg)[orient_perm(code, k + 1)])[en]
            dx = xo - xn
            dx -= np.round(dx)          # periodic shift by whole periods
            assert np.abs(dx).max() < 1e-12
    assert nontrivial > 20


@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_relabelled_axes_invariance(alpha):
    """Relabelling the reference axes of every element (non-trivial orient
    codes, permuted face numbering) changes nothing physical."""
    k, N = 3, 3
    n3 = (k + 1) ** 3
    rng = np.random.default_rng(5)
    frames = synth.mesh.random_frames(N ** 3, rng)
    deform = synth.mesh.curving(0.04)
    fields_fn = lambda x: np.stack([np.sin(2 * np.pi * x[..., 0] + 1) * np.cos(2 * np.pi * x[..., 2]),
                                    np.cos(2 * np.pi * x[..., 1]), np.sin(2 * np.pi * (x[..., 0] + x[..., 2])),
                                    np.cos(2 * np.pi * x[..., 1] + 0.3)], -1)
    coef = lambda x: 1.0 + 0.3 * np.sin(2 * np.pi * x[..., 0]) * np.cos(2 * np.pi * x[..., 1])
    out = []
    for fr in (None, frames):
        mesh = synth.cube_mesh(N, q=k, periodic=True, deform=deform, frames=fr)
        x = synth.solution_node_positions(mesh, k)
        o = oracle.Oracle(mesh, k, coef(x), 1.0 / coef(x), alpha)
        U = np.transpose(fields_fn(x), (0, 2, 1)).copy()
        R = o.apply(U)
        # sort nodes of each element by physical position for comparison
        key = np.round(x, 9)
        order = np.lexsort((key[..., 0], key[..., 1], key[..., 2]), axis=-1)
        out.append(np.take_along_axis(R, order[:, None, :], axis=2))
    scale = np.abs(out[0]).max()
    assert np.abs(out[0] - out[1]).max() / scale < 1e-11


@pytest.mark.parametrize("k", [1, 3])
def test_upwind_flux_is_riemann_solution(k):
    """For piecewise-constant states, the oracle's face flux (read back from
    R through the test function (1 + xi_x)/2, which is 1 on the +x face and
    0 on the -x face) equals the exact Riemann solution of the acoustic
    system: p* + Z_L v* = p_L + Z_L v_L and p* - Z_R v* = p_R - Z_R v_R
    (outgoing / incoming characteristics, Sec. 2.4 upwind flux)."""
    N, n = 2, k + 1
    n3 = n ** 3
    mesh = synth.cube_mesh(N, q=1, periodic=True)
    ex = np.arange(N ** 3) % N
    rho = np.where(ex == 0, 1.0, 2.0)[:, None] * np.ones((1, n3))
    c = np.where(ex == 0, 1.0, 1.5)[:, None] * np.ones((1, n3))
    ZL, ZR = 1.0, 3.0
    o = oracle.Oracle(mesh, k, rho, c, alpha=1.0)
    sL = np.array([0.7, 0.4, -0.2, 0.1])
    sR = np.array([-0.3, -0.5, 0.6, 0.2])
    U = np.where((ex == 0)[:, None, None], sL[None, :, None], sR[None, :, None]) * np.ones((1, 1, n3))
    R = o.apply(U)
    e = 0                                           # left element, +x face is an L|R face
    xgl = oracle.gauss_lobatto_1d(n)
    phi = (1 + xgl[np.arange(n3) % n]) / 2
    area = (1.0 / N) ** 2
    mom = phi @ (o.Mv[e] @ R[e, 1])                 # = -area (p* - p_L)
    mas = phi @ (o.Mp[e] @ R[e, 0])                 # = -area ((v.n)* - v_L.n)
    pstar = sL[0] - mom / area
    vstar = sL[1] - mas / area
    assert abs(pstar + ZL * vstar - (sL[0] + ZL * sL[1])) < 1e-12
    assert abs(pstar - ZR * vstar - (sR[0] - ZR * sR[1])) < 1e-12
