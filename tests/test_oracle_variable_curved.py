"""Pins of the oracle on variable coefficients and curved geometry.

* Variable coefficients (Sec. 2 Eq. (1) with rho(x)): for rho = 1 + 0.3 x
  (linear, so exactly a degree-k nodal field), c = 1, a pressure p(x) with
  dp/dx = rho g(x) for a polynomial g, and a polynomial velocity, the exact
  right-hand side R_v = -rho^-1 grad p = -g e_x and R_p = -rho c^2 div v are
  polynomials of degree <= k, and the scheme must return them exactly in
  elements away from the periodic seam.  This fixes the rho and 1/(rho c^2)
  weights of the mass matrices, which the energy identity cannot see.
* Curved geometry (Sec. 3, curved elements): a plane wave on a periodic,
  curved mesh (geometry degree q = k) converges at rate >= k, and at rate
  about k+1 on the same mesh without curving.  The quadrature with k+1 points
  per direction does not integrate the curved metric terms exactly (the
  variational crime Sec. 3 accepts); that costs up to one order (k = 3: 3.8
  from 2^3 to 4^3 elements, 3.1 from 4^3 to 8^3), independent of the time
  step and of raising the geometry degree.
"""
import numpy as np
import pytest

import synth
import oracle
from oracle_helpers import SHEAR, linear_map


@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_variable_coefficient_consistency(alpha):
    k, N = 3, 4
    mesh = synth.cube_mesh(N, q=1, periodic=True, deform=linear_map(SHEAR))
    x = synth.solution_node_positions(mesh, k)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    rho = 1.0 + 0.3 * X
    c = np.ones_like(rho)
    o = oracle.Oracle(mesh, k, rho, c, alpha)
    # dp/dx = rho g, g = 1 + x:  p = x + 0.65 x^2 + 0.1 x^3
    p = X + 0.65 * X ** 2 + 0.1 * X ** 3
    v = np.stack([X ** 2 - Y, Y * Z + X, Z ** 2], axis=1)          # total degree 2
    U = np.concatenate([p[:, None], v], axis=1)
    R = o.apply(U)
    g = 1.0 + X
    div_v = 2 * X + Z + 2 * Z
    Rex = np.zeros_like(U)
    Rex[:, 1] = -g
    Rex[:, 0] = -rho * div_v
    interior = [e for e in range(N ** 3)
                if all(1 <= w <= N - 2 for w in (e % N, (e // N) % N, e // (N * N)))]
    err = np.abs(R[interior] - Rex[interior]).max() / np.abs(Rex[interior]).max()
    assert err < 1e-11, err
    # a swapped weighting (rho on the pressure mass) is visibly wrong
    o_bad = oracle.Oracle(mesh, k, 1.0 / rho, c * rho, alpha)
    R_bad = o_bad.apply(U)
    assert np.abs(R_bad[interior] - Rex[interior]).max() / np.abs(Rex[interior]).max() > 1e-2


def _plane_curved_error(N, k, t_end=0.05, a=0.05):
    mesh = synth.cube_mesh(N, q=k, periodic=True, deform=synth.mesh.curving(a) if a else None)
    x = synth.solution_node_positions(mesh, k)
    kv = (2 * np.pi, 0.0, 0.0)
    exact = lambda xx, t: synth.fields.plane_wave(xx, t, kvec=kv)
    U0 = np.transpose(exact(x, 0.0), (0, 2, 1)).copy()
    ones = np.ones(x.shape[:2])
    o = oracle.Oracle(mesh, k, ones, ones, 1.0)
    dt = 0.05 * (1.0 / N) / k ** 1.5
    n = int(np.ceil(t_end / dt))
    U = o.lsrk(U0, t_end / n, n)
    return o.l2_error(U, exact, t_end)[0]


@pytest.mark.parametrize("k", [2, 3])
def test_curved_mesh_plane_wave_convergence(k):
    e = [_plane_curved_error(N, k) for N in (2, 4, 8)]
    rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert rates.min() > k - 0.2, (e, rates)
    flat = [_plane_curved_error(N, k, a=0.0) for N in (4, 8)]
    assert np.log2(flat[0] / flat[1]) > k + 1 - 0.3, flat
