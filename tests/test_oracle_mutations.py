"""The pins constrain the oracle: each test plants one plausible mistake in
an oracle instance (a sign, a dropped term, a transposed operand, a wrong
table, a coefficient typo, a wrong orientation map), on the CPU, re-runs the
measurement of the pin that should catch it, and checks that the pin's own
criterion holds for the oracle as written and fails for the mutant.
"""
import math

import numpy as np
import pytest
import sympy as sp

import oracle
import oracle.dg as odg
import synth
from oracle import LSRK54_A, LSRK54_B
from oracle.basis import gauss_1d, gauss_lobatto_1d, tensor_points
from oracle_helpers import SHEAR, linear_map, single_element_mesh
from test_oracle_operator import _poly_fields
from test_oracle_timestep import _sym_minus_S, stability_poly


# --- operator: polynomial consistency (interior elements reproduce -S u) ---
def _consistency(mutate=None):
    k, N, alpha = 3, 4, 1.0
    rng = np.random.default_rng(13)
    mesh = synth.cube_mesh(N, q=1, periodic=True, deform=linear_map(SHEAR))
    x = synth.solution_node_positions(mesh, k)
    rho0, c0 = 1.3, 0.7
    n3 = (k + 1) ** 3
    o = oracle.Oracle(mesh, k, np.full((N ** 3, n3), rho0), np.full((N ** 3, n3), c0), alpha)
    if mutate:
        mutate(o)
    u, g = _poly_fields(x, rng, k)
    U = np.transpose(u, (0, 2, 1)).copy()
    R = o.apply(U)
    Rex = np.zeros_like(U)
    Rex[:, 1:] = -np.transpose(g[:, :, 0, :], (0, 2, 1)) / rho0
    Rex[:, 0] = -rho0 * c0 ** 2 * (g[:, :, 1, 0] + g[:, :, 2, 1] + g[:, :, 3, 2])
    interior = [e for e in range(N ** 3) if all(1 <= v <= N - 2 for v in (e % N, (e // N) % N, e // (N * N)))]
    return np.abs(R[interior] - Rex[interior]).max() / np.abs(Rex[interior]).max()


def _drop_face(o):
    o.s[:, 3] = 0.0                          # the +eta face integral forgotten


def _transpose_cell(o):
    o.B = np.ascontiguousarray(np.swapaxes(o.B, 2, 3))   # test and trial functions swapped


def _mass_typo(o):
    o.Minv_p = o.Minv_p * 1.001              # a slightly wrong pressure mass


def _normal_sign(o):
    o.nrm[:, 4] = -o.nrm[:, 4]               # an inward normal on one face


@pytest.mark.parametrize("mutant", [_drop_face, _transpose_cell, _mass_typo, _normal_sign])
def test_consistency_pin_catches(mutant):
    assert _consistency() < 1e-11
    assert _consistency(mutant) > 1e-4, mutant.__name__


# --- operator: energy identity (central conserves, upwind dissipates) ------
def _energy_rate(alpha, mutate=None):
    k, N = 3, 3
    n3 = (k + 1) ** 3
    rng = np.random.default_rng(7)
    mesh = synth.cube_mesh(N, q=1, periodic=True, deform=linear_map(SHEAR))
    rho = rng.uniform(0.5, 2.0, size=(N ** 3, n3))
    c = rng.uniform(0.5, 2.0, size=(N ** 3, n3))
    o = oracle.Oracle(mesh, k, rho, c, alpha)
    if mutate:
        mutate(o)
    U = rng.uniform(-1, 1, size=(N ** 3, 4, n3))
    R = o.apply(U)
    return o.mass_inner(U, R) / np.sqrt(o.mass_inner(U, U) * o.mass_inner(R, R))


def test_energy_pin_catches_antidissipative_flux():
    assert _energy_rate(1.0) < -1e-3

    def flip(o):
        o.alpha = -1.0                       # the upwind penalty with the wrong sign
    assert _energy_rate(1.0, flip) > 1e-3


def test_energy_pin_catches_unbalanced_central_flux():
    assert abs(_energy_rate(0.0)) < 1e-13

    def lopsided(o):
        o.Zp = 2.0 * o.Zp                    # weights of p* and (v.n)* no longer sum to one
    assert abs(_energy_rate(0.0, lopsided)) > 1e-4


# --- flux: the upwind flux is the exact Riemann solution -------------------
def _riemann_residual(mutate=None, k=1):
    N, n = 2, k + 1
    n3 = n ** 3
    mesh = synth.cube_mesh(N, q=1, periodic=True)
    ex = np.arange(N ** 3) % N
    rho = np.where(ex == 0, 1.0, 2.0)[:, None] * np.ones((1, n3))
    c = np.where(ex == 0, 1.0, 1.5)[:, None] * np.ones((1, n3))
    ZL, ZR = 1.0, 3.0
    o = oracle.Oracle(mesh, k, rho, c, alpha=1.0)
    if mutate:
        mutate(o)
    sL = np.array([0.7, 0.4, -0.2, 0.1])
    sR = np.array([-0.3, -0.5, 0.6, 0.2])
    U = np.where((ex == 0)[:, None, None], sL[None, :, None], sR[None, :, None]) * np.ones((1, 1, n3))
    R = o.apply(U)
    xgl = gauss_lobatto_1d(n)
    phi = (1 + xgl[np.arange(n3) % n]) / 2
    area = (1.0 / N) ** 2
    pstar = sL[0] - (phi @ (o.Mv[0] @ R[0, 1])) / area
    vstar = sL[1] - (phi @ (o.Mp[0] @ R[0, 0])) / area
    return max(abs(pstar + ZL * vstar - (sL[0] + ZL * sL[1])), abs(pstar - ZR * vstar - (sR[0] - ZR * sR[1])))


def test_riemann_pin_catches_swapped_impedances():
    assert _riemann_residual() < 1e-12

    def swap(o):
        o.Zm, o.Zp = o.Zp.copy(), o.Zm.copy()   # each side weighted by its own impedance
    assert _riemann_residual(swap) > 1e-3


# --- orientation: relabelled element axes change nothing physical ----------
def _relabel_difference():
    k, N = 3, 3
    rng = np.random.default_rng(5)
    frames = synth.mesh.random_frames(N ** 3, rng)
    deform = synth.mesh.curving(0.04)
    fields_fn = lambda x: np.stack([np.sin(2 * np.pi * x[..., 0] + 1) * np.cos(2 * np.pi * x[..., 2]),
                                    np.cos(2 * np.pi * x[..., 1]), np.sin(2 * np.pi * (x[..., 0] + x[..., 2])),
                                    np.cos(2 * np.pi * x[..., 1] + 0.3)], -1)
    out = []
    for fr in (None, frames):
        mesh = synth.cube_mesh(N, q=k, periodic=True, deform=deform, frames=fr)
        x = synth.solution_node_positions(mesh, k)
        o = oracle.Oracle(mesh, k, np.ones(x.shape[:2]), np.ones(x.shape[:2]), 1.0)
        R = o.apply(np.transpose(fields_fn(x), (0, 2, 1)).copy())
        key = np.round(x, 9)
        order = np.lexsort((key[..., 0], key[..., 1], key[..., 2]), axis=-1)
        out.append(np.take_along_axis(R, order[:, None, :], axis=2))
    return np.abs(out[0] - out[1]).max() / np.abs(out[0]).max()


def test_relabelling_pin_catches_wrong_orientation_map(monkeypatch):
    assert _relabel_difference() < 1e-11
    right = odg.orient_perm

    def no_swap(o, m):
        return right(o & ~1, m)              # the axis-swap bit of the code ignored
    monkeypatch.setattr(odg, "orient_perm", no_swap)
    assert _relabel_difference() > 1e-3


# --- LSRK: the stage loop realises the fourth-order stability polynomial ---
def test_lsrk_pins_catch_a_coefficient_typo():
    A = list(LSRK54_A)
    A[2] = A[2] * (1 + 1e-6)                 # one digit wrong in one coefficient
    g = stability_poly(A, LSRK54_B)
    assert max(abs(g[j] - 1.0 / math.factorial(j)) for j in range(5)) > 1e-9
    cfg = synth.configs.standing_wave(N=2, k=2)
    o = oracle.Oracle(cfg["mesh"], 2, cfg["rho"], cfg["c"], 1.0)
    U0 = synth.configs.random_state(8, 2, 3)
    dt = 0.01
    g0 = stability_poly(LSRK54_A, LSRK54_B)
    acc, term = g0[0] * U0, U0
    for j in range(1, 6):
        term = dt * o.apply(term)
        acc = acc + g0[j] * term
    assert np.abs(o.lsrk(U0, dt, 1) - acc).max() / np.abs(U0).max() < 1e-14
    assert np.abs(o.lsrk(U0, dt, 1, A=A) - acc).max() / np.abs(U0).max() > 1e-12


# --- TCK: Taylor terms equal (-S)^j u computed symbolically ----------------
def _tck_symbolic_error(mutate=None):
    k = 3
    n, n3 = k + 1, (k + 1) ** 3
    A = np.array([[0.31, 0.05, -0.02], [0.03, 0.27, 0.04], [0.06, -0.01, 0.22]])
    Ainv = np.linalg.inv(A)
    rho, c = 1.4, 0.8
    o = oracle.Oracle(single_element_mesh(A), k, np.full((1, n3), rho), np.full((1, n3), c))
    if mutate:
        mutate(o)
    rng = np.random.default_rng(30)
    xi = sp.symbols("x0 x1 x2")
    flds = []
    for _ in range(4):
        expr = 0
        for a in range(n):
            for b in range(n):
                for cc in range(n):
                    expr += float(rng.normal()) * xi[0] ** a * xi[1] ** b * xi[2] ** cc
        flds.append(expr)
    pts = tensor_points(gauss_lobatto_1d(n))
    ev = lambda f, P: np.array(sp.lambdify(xi, f, "numpy")(P[:, 0], P[:, 1], P[:, 2]) + 0 * P[:, 0])
    U = np.stack([ev(f, pts) for f in flds])[None]
    _, terms = o.tck(U, 0.03, 0, return_terms=True)
    cur, err, scale = flds, 0.0, np.abs(U).max()
    for j, (m, T) in enumerate(terms[1:], start=1):
        cur = _sym_minus_S(cur, Ainv, rho, c, xi)
        ex = np.stack([ev(f, tensor_points(gauss_1d(m)[0])) for f in cur])
        scale = max(np.abs(ex).max(), scale)
        err = max(err, np.abs(T[0] - ex).max() / scale)
    return err


def test_tck_pin_catches_wrong_derivative_table():
    assert _tck_symbolic_error() < 1e-11

    def scaled_derivative(o):
        t = o._tck_level(o.n)
        t["D"] = t["D"] * (1 + 1e-6)         # a derivative table off in the sixth digit
    assert _tck_symbolic_error(scaled_derivative) > 1e-8

    def wrong_metric(o):
        t = o._tck_level(o.n)
        t["Jinv"] = np.ascontiguousarray(np.swapaxes(t["Jinv"], 2, 3))   # J^-1 transposed
    assert _tck_symbolic_error(wrong_metric) > 1e-3


# --- quadrature: n Gauss points integrate degree 2n-1 exactly -------------
def test_exactness_pin_catches_perturbed_weights():
    n = 4
    x, w = gauss_1d(n)
    exact = 2.0 / (2 * n - 1)                # integral of x^(2n-2) over [-1, 1]
    assert abs(np.sum(w * x ** (2 * n - 2)) - exact) < 1e-14
    w_bad = w * (1 + 1e-7 * np.arange(n))
    assert abs(np.sum(w_bad * x ** (2 * n - 2)) - exact) > 1e-9


# --- degree reduction: the projection is Legendre truncation --------------
def _projection_error(m, r, mutate=None):
    from numpy.polynomial import legendre as leg
    k = m - 1
    o = oracle.Oracle(single_element_mesh(np.diag([0.5, 0.5, 0.5])), k,
                      np.ones((1, (k + 1) ** 3)), np.ones((1, (k + 1) ** 3)))
    if mutate:
        mutate(o, m)
    rng = np.random.default_rng(100 * m + r)
    C = rng.normal(size=(4, m, m, m))

    def values(C, npts):
        V = leg.legvander(gauss_1d(npts)[0], C.shape[1] - 1)
        return np.einsum("fijl,ai,bj,cl->fcba", C, V, V, V).reshape(4, -1)

    got = o._project(values(C, m)[None], m, r)[0]
    want = values(C[:, :m - r, :m - r, :m - r], m - r)
    return np.abs(got - want).max() / np.abs(want).max()


def test_projection_pin_catches_interpolation_in_place_of_projection():
    assert _projection_error(5, 2) < 1e-12

    def interpolate(o, m):
        # the reduced values taken by evaluating the m-point interpolant at
        # the (m-2) points instead of projecting: exact only for degree < m-2
        from oracle.basis import basis_3d
        o._tck_level(m)["P"] = basis_3d(gauss_1d(m)[0], tensor_points(gauss_1d(m - 2)[0]))
    assert _projection_error(5, 2, interpolate) > 1e-3


# --- HDG-ADER: one step equals ADER where the DG derivative is collocated ---
def _hdg_vs_ader(mutate=None):
    k, N = 2, 6
    rng = np.random.default_rng(42)
    mesh = synth.cube_mesh(N, q=1, periodic=True, deform=linear_map(SHEAR))
    x = synth.solution_node_positions(mesh, k)
    n3 = (k + 1) ** 3
    o = oracle.Oracle(mesh, k, np.full((N ** 3, n3), 1.3), np.full((N ** 3, n3), 0.7))
    u, _ = _poly_fields(x, rng, k)
    U = np.transpose(u, (0, 2, 1)).copy()
    a = o.ader(U, 0.01, 1, 2)
    if mutate:
        mutate(o)
    h = o.hdg_ader(U, 0.01, 1, 2)
    deep = [e for e in range(N ** 3) if all(2 <= v <= N - 3 for v in (e % N, (e // N) % N, e // (N * N)))]
    return np.abs(h[deep] - a[deep]).max() / np.abs(a[deep]).max()


def test_hdg_pin_catches_a_first_term_built_from_u():
    assert _hdg_vs_ader() < 1e-12
    plain_tck = odg.Oracle.tck

    def tck_ignoring_w(self, U, dt, reduce_every=2, return_terms=False, first=None):
        return plain_tck(self, U, dt, reduce_every, return_terms, first=U)   # T_1 from U, not from W

    def mutate(o):
        o.tck = tck_ignoring_w.__get__(o)
    # the first term enters with dt^2 / 2, so the mutant differs by ~1e-5:
    # far outside the pin's 1e-12
    assert _hdg_vs_ader(mutate) > 1e-8


# --- the 2D oracle: consistency and energy pins on quadrilaterals ---------
def _consistency_2d(mutate=None, k=3):
    from oracle import Oracle2D
    from synth import mesh2d
    N = 5
    A2 = np.array([[1.0, 0.3], [-0.2, 0.9]])
    mesh = mesh2d.square_mesh(N, q=1, periodic=True, deform=lambda x: x @ A2.T)
    x = mesh2d.solution_node_positions_2d(mesh, k)
    rng = np.random.default_rng(k)
    co = rng.normal(size=(3, k + 1, k + 1))
    rho0, c0 = 1.3, 0.7
    terms = [(a, b) for a in range(k + 1) for b in range(k + 1) if a + b <= k]
    f = lambda c: sum(c[a, b] * x[..., 0] ** a * x[..., 1] ** b for a, b in terms)
    dx = lambda c: sum(c[a, b] * a * x[..., 0] ** (a - 1) * x[..., 1] ** b for a, b in terms if a > 0)
    dy = lambda c: sum(c[a, b] * b * x[..., 0] ** a * x[..., 1] ** (b - 1) for a, b in terms if b > 0)
    n2 = (k + 1) ** 2
    o = Oracle2D(mesh, k, np.full((N * N, n2), rho0), np.full((N * N, n2), c0))
    if mutate:
        mutate(o)
    U = np.stack([f(co[i]) for i in range(3)], axis=1)
    R = o.apply(U)
    Rex = np.stack([-rho0 * c0 ** 2 * (dx(co[1]) + dy(co[2])), -dx(co[0]) / rho0, -dy(co[0]) / rho0], axis=1)
    inner = [e for e in range(N * N) if 1 <= e % N <= N - 2 and 1 <= e // N <= N - 2]
    return np.abs(R[inner] - Rex[inner]).max() / np.abs(Rex[inner]).max()


def _energy_rate_2d(alpha, mutate=None):
    from oracle import Oracle2D
    from synth import mesh2d
    k, N = 3, 3
    rng = np.random.default_rng(5)
    A2 = np.array([[1.0, 0.3], [-0.2, 0.9]])
    mesh = mesh2d.square_mesh(N, q=1, periodic=False, deform=lambda x: x @ A2.T,
                              frames=mesh2d.random_frames_2d(N * N, rng))
    n2 = (k + 1) ** 2
    o = Oracle2D(mesh, k, rng.uniform(0.5, 2.0, size=(N * N, n2)), rng.uniform(0.5, 2.0, size=(N * N, n2)), alpha)
    if mutate:
        mutate(o)
    U = rng.uniform(-1, 1, size=(N * N, 3, n2))
    R = o.apply(U)
    return o.mass_inner(U, R) / np.sqrt(o.mass_inner(U, U) * o.mass_inner(R, R))


def test_2d_pins_catch_planted_mistakes():
    assert _consistency_2d() < 1e-11

    def drop_face(o):
        o.s[:, 2] = 0.0
    assert _consistency_2d(drop_face) > 1e-4

    def transpose_cell(o):
        o.B = np.ascontiguousarray(np.swapaxes(o.B, 2, 3))
    assert _consistency_2d(transpose_cell) > 1e-4
    assert _energy_rate_2d(1.0) < -1e-4

    def flip(o):
        o.alpha = -1.0
    assert _energy_rate_2d(1.0, flip) > 1e-4


# --- diagnostics: energy and L2 error closed forms -------------------------
import types

from oracle.basis import basis_3d, tensor_weights
import test_oracle_energy_norms as en


def _energy_closed_form(mutate=None, dim=3, k=2):
    N = 3
    mesh = en._graded_mesh(dim, N)
    x = en._box_nodes(mesh, k, dim)
    E, npts = x.shape[0], x.shape[1]
    U = np.zeros((E, dim + 1, npts))
    U[:, 0] = 1.0 + x[..., 0]
    U[:, 1] = U[:, 2] = 1.0
    o = en._make(dim, mesh, k, 1.0 + x[..., 0], np.full((E, npts), 2.0))
    if mutate:
        mutate(o)
    return abs(o.energy(U) - 27.0 / 16.0)


def _energy_density(o, U, pressure_weight, velocity_weight, half=0.5):
    u = np.einsum("qa,eva->evq", o.Phi, np.asarray(U, float))
    dens = velocity_weight(o) * np.sum(u[:, 1:] ** 2, axis=1) + pressure_weight(o) * u[:, 0] ** 2
    return half * float(np.sum(o.wdet * dens))


def _no_half(o):
    o.energy = types.MethodType(
        lambda self, U: _energy_density(self, U, lambda s: 1 / (s.rho_q * s.c_q ** 2), lambda s: s.rho_q, 1.0), o)


def _pressure_times_impedance(o):
    o.energy = types.MethodType(
        lambda self, U: _energy_density(self, U, lambda s: s.rho_q * s.c_q ** 2, lambda s: s.rho_q), o)


def _velocity_without_density(o):
    o.energy = types.MethodType(
        lambda self, U: _energy_density(self, U, lambda s: 1 / (s.rho_q * s.c_q ** 2), lambda s: 1.0), o)


@pytest.mark.parametrize("mutant", [_no_half, _pressure_times_impedance, _velocity_without_density])
def test_energy_closed_form_pin_catches(mutant):
    assert _energy_closed_form() < 1e-13
    assert _energy_closed_form(mutant) > 1e-2, mutant.__name__


def test_energy_closed_form_pin_catches_2d_dropped_half():
    assert _energy_closed_form(dim=2) < 1e-13
    bad = lambda o: setattr(o, "energy", types.MethodType(lambda self, U: 2 * type(self).energy(self, U), o))
    assert _energy_closed_form(bad, dim=2) > 1e-2


def _l2_closed_form(mutate=None):
    k, N = 2, 3
    mesh = en._graded_mesh(3, N)
    x = en._box_nodes(mesh, k, 3)
    E, npts = x.shape[0], x.shape[1]
    ones = np.ones((E, npts))
    o = oracle.Oracle(mesh, k, ones, ones, 1.0)
    if mutate:
        mutate(o)
    U = np.zeros((E, 4, npts))
    U[:, 0] = 0.5
    U[:, 1] = x[..., 0]

    def exact(xx, t):
        out = np.zeros(xx.shape[:-1] + (4,))
        out[..., 0] = out[..., 1] = xx[..., 0]
        out[..., 2] = xx[..., 1]
        return out
    ep, ev = o.l2_error(U, exact, 0.0)
    return max(abs(ep - 0.5), abs(ev - np.sqrt(0.5)))


def _l2_variant(o, use_detJ=True, mapped=True):
    """l2_error written again with one planted change."""
    def f(self, U, exact, t, extra=2):
        xe, we = gauss_1d(self.n + extra)
        Qe = tensor_points(xe)
        phi = basis_3d(self.xgl, Qe)
        x = self.positions(Qe) if mapped else np.broadcast_to(Qe, (self.E,) + Qe.shape)
        wd = tensor_weights(we)[None, :] * (np.linalg.det(self.jacobian(Qe)) if use_detJ else 1.0)
        uh = np.einsum("qa,eva->eqv", phi, np.asarray(U, float))
        ue = exact(x, t)
        ep = np.sum(wd * (uh[..., 0] - ue[..., 0]) ** 2) / np.sum(wd * ue[..., 0] ** 2)
        ev = np.sum(wd[..., None] * (uh[..., 1:] - ue[..., 1:]) ** 2) / np.sum(wd[..., None] * ue[..., 1:] ** 2)
        return float(np.sqrt(ep)), float(np.sqrt(ev))
    o.l2_error = types.MethodType(f, o)


def test_l2_closed_form_pin_catches():
    assert _l2_closed_form() < 1e-13
    assert _l2_closed_form(lambda o: _l2_variant(o)) < 1e-13          # the restatement itself is right
    assert _l2_closed_form(lambda o: _l2_variant(o, use_detJ=False)) > 1e-3
    assert _l2_closed_form(lambda o: _l2_variant(o, mapped=False)) > 1e-3


# --- the two-register LSRK schemes ----------------------------------------
def test_2r_order_conditions_catch_a_coefficient_typo():
    from oracle import LSRK59_KCL_A, LSRK59_KCL_B
    from test_oracle_lsrk2r import butcher, order_conditions
    res = order_conditions(*butcher(LSRK59_KCL_A, LSRK59_KCL_B))
    assert max(abs(r) for q in res for r in res[q]) < 1e-14
    A = list(LSRK59_KCL_A)
    A[4] *= 1.000001                                     # sixth digit of one coefficient
    res = order_conditions(*butcher(A, LSRK59_KCL_B))
    assert max(abs(r) for q in res for r in res[q]) > 1e-8


def test_2r_step_pin_catches_a_loop_that_restarts_from_u():
    """A two-register loop that builds every stage from u_n instead of the
    running sum S_i fails the step-equals-polynomial pin."""
    from oracle import LSRK59_KCL_A, LSRK59_KCL_B
    from test_oracle_lsrk2r import stability_poly_2r
    cfg = synth.configs.curved_pulse(N=2, k=2)
    o = oracle.Oracle(cfg["mesh"], 2, cfg["rho"], cfg["c"], 1.0)
    U0 = synth.configs.random_state(8, 2, 3)
    dt = 0.01
    g = stability_poly_2r(LSRK59_KCL_A, LSRK59_KCL_B)
    acc, term = g[0] * U0, U0
    for j in range(1, len(g)):
        term = dt * o.apply(term)
        acc = acc + g[j] * term

    def wrong(U):
        s, Y, S = len(LSRK59_KCL_B), U, U.copy()
        for i in range(s):
            R = o.apply(Y)
            if i < s - 1:
                Y = U + dt * LSRK59_KCL_A[i] * R
            S = S + dt * LSRK59_KCL_B[i] * R
        return S
    assert np.abs(o.lsrk2r(U0, dt, 1) - acc).max() / np.abs(U0).max() < 1e-14
    assert np.abs(wrong(U0) - acc).max() / np.abs(U0).max() > 1e-8


# --- curved geometry: free-stream preservation where the quadrature is exact ---
def _refaces(o, nanson):
    """Recompute the oracle's face measures and normals with the given
    version of Nanson's formula (as the oracle's face loop would)."""
    wf = np.outer(o.wg, o.wg).T.reshape(-1)
    for f in range(6):
        Jf = o.jacobian(odg.face_points(f, o.xg))
        detJf, Jinvf = np.linalg.det(Jf), np.linalg.inv(Jf)
        d, side = f // 2, (1.0 if f % 2 else -1.0)
        nw = nanson(wf[None, :, None], detJf[:, :, None], Jinvf, d, side)
        s = np.linalg.norm(nw, axis=2)
        o.s[:, f] = s
        o.nrm[:, f] = nw / s[:, :, None]


def test_free_stream_pin_catches_curved_geometry_mistakes():
    """On a curved mesh with q <= (k+2)/2 a constant state is steady; a
    transposed Jacobian, a face measure without detJ, or the Nanson normal
    taken from a column of J^-1 instead of a row each break that."""
    from test_oracle_curved_geometry import free_stream_residual
    k, q, N = 3, 2, 3

    class Transposed(oracle.Oracle):
        def jacobian(self, pts):
            return np.swapaxes(super().jacobian(pts), -1, -2)

    right = lambda w, det, Ji, d, side: w * det * side * Ji[:, :, d, :]
    no_det = lambda w, det, Ji, d, side: w * side * Ji[:, :, d, :]
    column = lambda w, det, Ji, d, side: w * det * side * Ji[:, :, :, d]
    assert free_stream_residual(k, q, N, 1.0) < 5e-11
    assert free_stream_residual(k, q, N, 1.0, mutate=lambda o: _refaces(o, right)) < 5e-11
    assert free_stream_residual(k, q, N, 1.0, oracle_cls=Transposed) > 1e-3
    assert free_stream_residual(k, q, N, 1.0, mutate=lambda o: _refaces(o, no_det)) > 1e-3
    assert free_stream_residual(k, q, N, 1.0, mutate=lambda o: _refaces(o, column)) > 1e-3


def test_curved_tck_pin_catches_a_transposed_jacobian():
    """The predictor of a linear field on a curved mesh is dt u + dt^2/2 T_1
    in closed form; an oracle that evaluates the Jacobian transposed (which
    the affine symbolic pins on a diagonal map cannot see) misses it."""
    from test_oracle_curved_geometry import curved_linear_case
    k = 3
    mesh, rho, c, U, T1 = curved_linear_case(k)
    ref = 0.01 * U + 0.5 * 0.01 ** 2 * T1

    class Transposed(oracle.Oracle):
        def jacobian(self, pts):
            return np.swapaxes(super().jacobian(pts), -1, -2)

    good = oracle.Oracle(mesh, k, rho, c, 1.0).tck(U, 0.01, 2)
    bad = Transposed(mesh, k, rho, c, 1.0).tck(U, 0.01, 2)
    assert np.abs(good - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(bad - ref).max() > 1e-8 * np.abs(ref).max()
