"""Pins of the 2D oracle (oracle/dg2d.py), the same discrete scheme as the
3D oracle one dimension down: exact quadrature on an affine element,
polynomial consistency, the energy identity, rotated element frames,
convergence to the standing wave, symbolic Taylor terms, and the paper's 2D
critical Courant numbers (Table crit-Cr) by Bloch-wave analysis."""
import itertools
import math
import os

import numpy as np
import pytest
import sympy as sp

from oracle import Oracle2D, LSRK54_A, LSRK54_B
from oracle.basis import gauss_1d, gauss_lobatto_1d
from oracle.dg2d import basis_2d, basis_grad_2d, tensor_points_2d, tensor_weights_2d
from synth import mesh2d
from test_oracle_timestep import stability_poly

SHEAR2 = np.array([[1.0, 0.3], [-0.2, 0.9]])


def _linear_map(A):
    A = np.asarray(A)
    return lambda x: x @ A.T


def _single(A, x0=(0.2, -0.1)):
    """One affine element x = x0 + A xi, walls on every face."""
    m = mesh2d.square_mesh(1, q=1, periodic=False)
    xi = np.array([[i, j] for j in (-1, 1) for i in (-1, 1)], float)
    m["nodes"] = (np.asarray(x0)[None, :] + xi @ np.asarray(A).T)[None]
    return m


@pytest.mark.parametrize("k", [1, 3, 4])
def test_mass_and_cell_matrices_exact_on_affine_element(k):
    A = np.array([[0.4, 0.1], [-0.05, 0.3]])
    n = k + 1
    o = Oracle2D(_single(A), k, np.full((1, n * n), 1.7), np.full((1, n * n), 0.6))
    # independent quadrature with three more points per direction
    xe, we = gauss_1d(n + 3)
    Q, W = tensor_points_2d(xe), tensor_weights_2d(we)
    xgl = gauss_lobatto_1d(n)
    phi, dphi = basis_2d(xgl, Q), basis_grad_2d(xgl, Q)
    det = np.linalg.det(A)
    Ainv = np.linalg.inv(A)
    Mv = 1.7 * det * np.einsum("q,qa,qb->ab", W, phi, phi)
    assert np.allclose(o.Mv[0], Mv, rtol=1e-13, atol=1e-15)
    assert np.allclose(o.Mp[0], Mv / (1.7 ** 2 * 0.6 ** 2), rtol=1e-13, atol=1e-15)
    grad = np.einsum("dqa,di->iqa", dphi, Ainv)
    B = det * np.einsum("q,iqa,qb->iab", W, grad, phi)
    assert np.allclose(o.B[0], B, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("k", [2, 3])
def test_polynomial_consistency_interior(k):
    N = 5
    mesh = mesh2d.square_mesh(N, q=1, periodic=True, deform=_linear_map(SHEAR2))
    x = mesh2d.solution_node_positions_2d(mesh, k)
    rng = np.random.default_rng(k)
    co = rng.normal(size=(3, k + 1, k + 1))
    rho0, c0 = 1.3, 0.7

    def field(c, x):
        return sum(c[a, b] * x[..., 0] ** a * x[..., 1] ** b for a in range(k + 1) for b in range(k + 1)
                   if a + b <= k)

    def dfield(c, x, d):
        out = 0.0
        for a in range(k + 1):
            for b in range(k + 1):
                if a + b > k:
                    continue
                if d == 0 and a > 0:
                    out = out + c[a, b] * a * x[..., 0] ** (a - 1) * x[..., 1] ** b
                if d == 1 and b > 0:
                    out = out + c[a, b] * b * x[..., 0] ** a * x[..., 1] ** (b - 1)
        return out

    n2 = (k + 1) ** 2
    o = Oracle2D(mesh, k, np.full((N * N, n2), rho0), np.full((N * N, n2), c0))
    U = np.stack([field(co[i], x) for i in range(3)], axis=1)
    R = o.apply(U)
    Rex = np.empty_like(U)
    Rex[:, 0] = -rho0 * c0 ** 2 * (dfield(co[1], x, 0) + dfield(co[2], x, 1))
    Rex[:, 1] = -dfield(co[0], x, 0) / rho0
    Rex[:, 2] = -dfield(co[0], x, 1) / rho0
    inner = [e for e in range(N * N) if 1 <= e % N <= N - 2 and 1 <= e // N <= N - 2]
    scale = np.abs(Rex[inner]).max()
    assert np.abs(R[inner] - Rex[inner]).max() < 1e-11 * scale
    assert np.abs(R - Rex).max() > 1e-3 * scale        # the periodic seam is seen


@pytest.mark.parametrize("alpha", [0.0, 1.0])
@pytest.mark.parametrize("periodic", [True, False])
def test_energy_identity(alpha, periodic):
    k, N = 3, 3
    rng = np.random.default_rng(5)
    mesh = mesh2d.square_mesh(N, q=1, periodic=periodic, deform=_linear_map(SHEAR2),
                              frames=mesh2d.random_frames_2d(N * N, rng))
    n2 = (k + 1) ** 2
    rho = rng.uniform(0.5, 2.0, size=(N * N, n2))
    c = rng.uniform(0.5, 2.0, size=(N * N, n2))
    o = Oracle2D(mesh, k, rho, c, alpha)
    U = rng.uniform(-1, 1, size=(N * N, 3, n2))
    R = o.apply(U)
    dE = o.mass_inner(U, R)
    scale = np.sqrt(o.mass_inner(U, U) * o.mass_inner(R, R))
    if alpha == 0.0:
        assert abs(dE) / scale < 1e-13
    else:
        assert dE / scale < -1e-4


def test_rotated_frames_change_nothing_physical():
    k = 3
    a = mesh2d.standing_wave_config_2d(N=3, k=k)
    b = mesh2d.standing_wave_config_2d(N=3, k=k, frames_seed=9)
    t = 0.05
    ea = Oracle2D(a["mesh"], k, a["rho"], a["c"]).lsrk(a["U0"], 0.005, 10)
    ob = Oracle2D(b["mesh"], k, b["rho"], b["c"])
    eb = ob.lsrk(b["U0"], 0.005, 10)
    # compare pointwise at the physical nodes of b: evaluate a's solution there
    oa = Oracle2D(a["mesh"], k, a["rho"], a["c"])
    ra = oa.l2_error(ea, a["exact"], t)
    rb = ob.l2_error(eb, b["exact"], t)
    assert abs(ra[0] - rb[0]) < 1e-10 * max(ra[0], 1e-16) + 1e-14
    assert abs(ra[1] - rb[1]) < 1e-10 * max(ra[1], 1e-16) + 1e-14


def _errors(method, N, k, cr, t_end):
    cfg = mesh2d.standing_wave_config_2d(N=N, k=k, cr=cr)
    nsteps = int(round(t_end / cfg["dt"]))
    dt = t_end / nsteps
    o = Oracle2D(cfg["mesh"], k, cfg["rho"], cfg["c"])
    U = o.lsrk(cfg["U0"], dt, nsteps) if method == "lsrk" else o.ader(cfg["U0"], dt, nsteps, 2)
    return o.l2_error(U, cfg["exact"], t_end)[0]


@pytest.mark.parametrize("method,k", [("lsrk", 2), ("ader", 2), ("ader", 3)])
def test_convergence_standing_wave(method, k):
    e = [_errors(method, N, k, 0.1, 0.1) for N in (4, 8, 16)]
    rate = np.log2(e[1] / e[2])
    assert rate > k + 1 - 0.35, (e, rate)


@pytest.mark.parametrize("k,red", [(2, 0), (3, 2), (4, 2), (4, 1), (4, 3)])
def test_tck_terms_match_symbolic(k, red):
    A = np.array([[0.31, 0.05], [0.03, 0.27]])
    Ainv = np.linalg.inv(A)
    rho, c = 1.4, 0.8
    n = k + 1
    o = Oracle2D(_single(A), k, np.full((1, n * n), rho), np.full((1, n * n), c))
    xi = sp.symbols("x0 x1")
    rng = np.random.default_rng(10 * k + red)
    flds = [sum(float(rng.normal()) * xi[0] ** a * xi[1] ** b for a in range(n) for b in range(n)
                if not red or a + b <= k) for _ in range(3)]
    pts = tensor_points_2d(gauss_lobatto_1d(n))
    ev = lambda f, P: np.array(sp.lambdify(xi, f, "numpy")(P[:, 0], P[:, 1]) + 0 * P[:, 0])
    U = np.stack([ev(f, pts) for f in flds])[None]
    dt = 0.03
    Ubar, terms = o.tck(U, dt, red, return_terms=True)

    def minus_S(f):
        grad = lambda g: [sum(Ainv[d, i] * sp.diff(g, xi[d]) for d in range(2)) for i in range(2)]
        p, vx, vy = f
        gp = grad(p)
        div = grad(vx)[0] + grad(vy)[1]
        return [sp.expand(-rho * c ** 2 * div), sp.expand(-gp[0] / rho), sp.expand(-gp[1] / rho)]

    cur, ubar = flds, [dt * f for f in flds]
    scale = np.abs(U).max()
    for j, (m, T) in enumerate(terms):
        if j == 0:
            continue
        cur = minus_S(cur)
        if m == 0:
            break
        Pm = tensor_points_2d(gauss_1d(m)[0])
        ex = np.stack([ev(f, Pm) for f in cur])
        scale = max(np.abs(ex).max(), scale)
        assert np.abs(T[0] - ex).max() < 1e-11 * scale, (j, m)
        ubar = [u + dt ** (j + 1) / math.factorial(j + 1) * f for u, f in zip(ubar, cur)]
    ex = np.stack([ev(f, pts) for f in ubar])
    assert np.abs(Ubar[0] - ex).max() < 1e-12 * np.abs(ex).max()


# --- the paper's 2D critical Courant numbers (Table crit-Cr) --------------------
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "crit_courant_2d.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, a, b, c = line.split()
            rows[int(k)] = (float(a), float(b), float(c))
    return rows


class Bloch2D:
    """Spectrum of the 2D operator on a periodic Cartesian mesh: union over
    wave numbers theta of the symbols L_00 + sum_d (L_{0,+d} e^{i theta_d} +
    L_{0,-d} e^{-i theta_d}), read off the oracle with unit vectors."""

    def __init__(self, k):
        self.k = k
        n = k + 1
        self.nd = 3 * n * n
        mesh = mesh2d.square_mesh(3, q=1, periodic=True)
        ones = np.ones((9, n * n))
        self.o = Oracle2D(mesh, k, ones, ones, 1.0)
        cols = []
        for i in range(self.nd):
            U = np.zeros((9, self.nd))
            U[0, i] = 1.0
            cols.append(self.o.apply(U.reshape(9, 3, n * n)).reshape(9, self.nd))
        self.L = np.stack(cols, axis=-1)
        th = np.linspace(0, np.pi, 7)
        self.symbols = [self._symbol(t) for t in itertools.product(th, th)]
        self.eigs = np.concatenate([np.linalg.eigvals(S) for S in self.symbols])

    def _symbol(self, theta):
        L = self.L[0].astype(complex)
        for d, s in enumerate((1, 3)):
            L = L + self.L[2 * s] * np.exp(1j * theta[d]) + self.L[s] * np.exp(-1j * theta[d])
        return L

    def dt(self, cr):
        return cr * (1.0 / 3) / self.k ** 1.5

    def lsrk_stable(self, cr, g):
        z = self.dt(cr) * self.eigs
        return np.abs(np.polynomial.polynomial.polyval(z, g)).max() <= 1.0 + 1e-5

    def ader_stable(self, cr, growth=1e-5):
        n2 = (self.k + 1) ** 2
        T = np.zeros((self.nd, self.nd))
        for start in range(0, self.nd, 9):
            U = np.zeros((9, self.nd))
            cols = list(range(start, min(start + 9, self.nd)))
            for e, i in enumerate(cols):
                U[e, i] = 1.0
            out = self.o.tck(U.reshape(9, 3, n2), self.dt(cr), 2).reshape(9, self.nd)
            for e, i in enumerate(cols):
                T[:, i] = out[e]
        I = np.eye(self.nd)
        return max(np.abs(np.linalg.eigvals(I + S @ T)).max() for S in self.symbols) <= 1.0 + growth


def _bisect(stable, lo, hi, tol=2e-3):
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if stable(mid):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("k", [1, 4])
def test_crit_courant_2d(k):
    b = Bloch2D(k)
    ref = _golden()[k]
    cr_ader = _bisect(b.ader_stable, 0.05, 0.6, 4e-3)
    assert abs(cr_ader - ref[2]) <= 0.15 * ref[2], (k, cr_ader, ref[2])
    g = stability_poly(LSRK54_A, LSRK54_B)
    cr_lsrk = _bisect(lambda c: b.lsrk_stable(c, g), 0.05, 1.5)
    assert 0.8 * ref[0] <= cr_lsrk <= 1.02 * ref[0], (k, cr_lsrk, ref[0])


def test_crit_courant_2d_k7_strong_onset():
    """At k = 7 the 2D ADER spectrum has a weak instability well below the
    paper's limit (growth 5e-6 per step at Cr 0.12, 9e-5 at 0.26: a few
    percent over a thousand steps), then a strong one (7e-2 per step at
    0.28).  The paper's simulated limit (0.28) is the strong onset, which
    lies where the growth per step passes 1e-3."""
    b = Bloch2D(7)
    ref = _golden()[7][2]
    cr = _bisect(lambda c: b.ader_stable(c, growth=1e-3), 0.2, 0.34, 4e-3)
    assert abs(cr - ref) <= 0.15 * ref, (cr, ref)
    assert not b.ader_stable(0.16)               # 1% over 1000 steps already exceeded
