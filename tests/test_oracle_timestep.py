"""Pins of the oracle's time integrators.

* LSRK (Sec. 2.2): the five-stage 2N scheme's stability polynomial agrees
  with exp(z) through z^4 (fourth order on linear problems), and one step of
  the stage loop equals that polynomial applied through repeated R.
* TCK (Sec. 2.3 Eq. (5), Algorithms 2-3): on an affine element with constant
  coefficients every Taylor term T_j equals (-S)^j u computed symbolically;
  with degree reduction this holds for total-degree data.
* Full schemes: convergence to the analytic standing wave at rate k+1 in
  space (LSRK at a small step) and in space-time (ADER, Sec. 4.7).
* Energy: upwind decays monotonically step by step.
"""
import math

import numpy as np
import pytest
import sympy as sp

import synth
import oracle
from oracle import LSRK54_A, LSRK54_B
from oracle.basis import gauss_1d, tensor_points, gauss_lobatto_1d
from oracle_helpers import single_element_mesh


def stability_poly(A, B):
    """Coefficients of the amplification polynomial of y' = lambda y."""
    P = np.polynomial.Polynomial
    y, dy, z = P([1.0]), P([0.0]), P([0.0, 1.0])
    for a, b in zip(A, B):
        dy = a * dy + z * y
        y = y + b * dy
    return y.coef


def test_lsrk_stability_polynomial():
    g = stability_poly(LSRK54_A, LSRK54_B)
    assert len(g) == 6
    for j in range(5):
        assert abs(g[j] - 1.0 / math.factorial(j)) < 1e-14, (j, g[j])
    assert abs(g[5] - 1.0 / 120) > 1e-4          # fifth order not reached
    assert 0.004 < g[5] < 0.006


def test_lsrk_step_equals_polynomial():
    cfg = synth.configs.standing_wave(N=2, k=2)
    o = oracle.Oracle(cfg["mesh"], 2, cfg["rho"], cfg["c"], 1.0)
    U0 = synth.configs.random_state(8, 2, 3)
    dt = 0.01
    U1 = o.lsrk(U0, dt, 1)
    g = stability_poly(LSRK54_A, LSRK54_B)
    acc, term = g[0] * U0, U0
    for j in range(1, 6):
        term = dt * o.apply(term)
        acc = acc + g[j] * term
    assert np.abs(U1 - acc).max() / np.abs(U0).max() < 1e-14


def _sym_minus_S(fields, Ainv, rho, c, xi):
    p, vx, vy, vz = fields
    grad = lambda f: [sum(Ainv[d, i] * sp.diff(f, xi[d]) for d in range(3)) for i in range(3)]
    gp = grad(p)
    div = sum(grad(v)[i] for i, v in enumerate((vx, vy, vz)))
    return [sp.expand(-rho * c ** 2 * div)] + [sp.expand(-gp[i] / rho) for i in range(3)]


@pytest.mark.parametrize("k,reduce_every", [(2, 0), (3, 0), (3, 2), (4, 2), (5, 2),
                                            (3, 1), (4, 1), (4, 3), (5, 3)])
def test_tck_terms_match_symbolic(k, reduce_every):
    n, n3 = k + 1, (k + 1) ** 3
    A = np.array([[0.31, 0.05, -0.02], [0.03, 0.27, 0.04], [0.06, -0.01, 0.22]])
    Ainv = np.linalg.inv(A)
    rho, c = 1.4, 0.8
    o = oracle.Oracle(single_element_mesh(A), k, np.full((1, n3), rho), np.full((1, n3), c))
    rng = np.random.default_rng(k * 10 + reduce_every)
    xi = sp.symbols("x0 x1 x2")
    flds = []
    for _ in range(4):
        expr = 0
        for a in range(n):
            for b in range(n):
                for cc in range(n):
                    if reduce_every and a + b + cc > k:
                        continue          # total degree <= k when reducing
                    expr += float(rng.normal()) * xi[0] ** a * xi[1] ** b * xi[2] ** cc
        flds.append(expr)
    xgl = gauss_lobatto_1d(n)
    pts = tensor_points(xgl)
    ev = lambda f, P: np.array(sp.lambdify(xi, f, "numpy")(P[:, 0], P[:, 1], P[:, 2]) + 0 * P[:, 0])
    U = np.stack([ev(f, pts) for f in flds])[None]
    dt = 0.03
    Ubar, terms = o.tck(U, dt, reduce_every, return_terms=True)
    cur = flds
    ubar_ex = [dt * f for f in flds]
    scale = np.abs(U).max()
    for j, (m, T) in enumerate(terms):
        if j == 0:
            continue
        cur = _sym_minus_S(cur, Ainv, rho, c, xi)
        if m == 0:
            assert all(sp.simplify(f) == 0 for f in cur) or reduce_every == 2
            break
        Pm = tensor_points(gauss_1d(m)[0])
        ex = np.stack([ev(f, Pm) for f in cur])
        # a term that vanishes exactly is held to the size of the terms before it
        scale = max(np.abs(ex).max(), scale)
        assert np.abs(T[0] - ex).max() / scale < 1e-11, (j, m)
        ubar_ex = [u + dt ** (j + 1) / math.factorial(j + 1) * f for u, f in zip(ubar_ex, cur)]
    ex = np.stack([ev(f, pts) for f in ubar_ex])
    assert np.abs(Ubar[0] - ex).max() / np.abs(ex).max() < 1e-12
    if reduce_every == 2:
        # with reduction the (k+1)-th term vanishes identically (Algorithm 3)
        assert terms[-1][0] in (0, 1) or len(terms) <= k + 2


@pytest.mark.parametrize("m,r", [(2, 1), (3, 1), (5, 1), (8, 1), (3, 2), (4, 2), (6, 2),
                                 (4, 3), (6, 3), (8, 3)])
def test_projection_is_legendre_truncation(m, r):
    """The reference-element L2 projection from m to m - r Gauss points
    (Sec. 3.3) keeps the tensor Legendre modes of degree < m - r in every
    direction and drops the others: Legendre polynomials are L2-orthogonal
    on [-1, 1], and the m-point rule integrates every product involved."""
    from numpy.polynomial import legendre as leg
    k = m - 1 if m > 1 else 1
    A = np.diag([0.5, 0.5, 0.5])
    o = oracle.Oracle(single_element_mesh(A), k, np.ones((1, (k + 1) ** 3)), np.ones((1, (k + 1) ** 3)))
    rng = np.random.default_rng(100 * m + r)
    C = rng.normal(size=(4, m, m, m))             # C[f, i, j, l]: mode P_i(x) P_j(y) P_l(z)

    def values(C, npts):
        x = gauss_1d(npts)[0]
        V = leg.legvander(x, C.shape[1] - 1)      # V[a, i] = P_i(x_a)
        # node index a + npts b + npts^2 c (first axis fastest)
        return np.einsum("fijl,ai,bj,cl->fcba", C, V, V, V).reshape(4, -1)

    T = values(C, m)[None]
    got = o._project(T, m, r)[0]
    want = values(C[:, :m - r, :m - r, :m - r], m - r)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def _errors(method, N, k, cr, t_end, reduce_every=2):
    cfg = synth.configs.standing_wave(N=N, k=k, cr=cr)
    nsteps = int(round(t_end / cfg["dt"]))
    dt = t_end / nsteps
    o = oracle.Oracle(cfg["mesh"], k, cfg["rho"], cfg["c"], 1.0)
    if method == "lsrk":
        U = o.lsrk(cfg["U0"], dt, nsteps)
    else:
        U = o.ader(cfg["U0"], dt, nsteps, reduce_every)
    return o.l2_error(U, cfg["exact"], t_end)[0]


@pytest.mark.parametrize("method,k,cr", [("lsrk", 2, 0.05), ("ader", 2, 0.1), ("ader", 3, 0.1)])
def test_convergence_standing_wave(method, k, cr):
    e = [_errors(method, N, k, cr, 0.1) for N in (2, 4, 8)]
    rate = np.log2(e[1] / e[2])
    assert rate > k + 1 - 0.35, (e, rate)


@pytest.mark.parametrize("method", ["lsrk", "ader"])
def test_upwind_energy_monotone(method):
    cfg = synth.configs.curved_pulse(N=2, k=3, nsteps=20)
    o = oracle.Oracle(cfg["mesh"], 3, cfg["rho"], cfg["c"], 1.0)
    energies = []
    cb = lambda s, U: energies.append(o.energy(U))
    if method == "lsrk":
        o.lsrk(cfg["U0"], cfg["dt"], 20, callback=cb)
    else:
        o.ader(cfg["U0"], cfg["dt"], 20, callback=cb)
    e = np.array([o.energy(cfg["U0"])] + energies)
    assert np.all(np.diff(e) <= 1e-14 * e[0]), np.diff(e)
    assert e[-1] < e[0]
