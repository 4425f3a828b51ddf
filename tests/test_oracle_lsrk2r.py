"""Pins of the paper's two-register low-storage Runge-Kutta schemes
(Sec. 2.2: LSRK4(5) and LSRK5(9), of Kennedy, Carpenter & Lewis), as the
oracle stores and runs them.

* Their Butcher tableaux, built here from the two-register structure
  (a_{i,j} = b_j for j < i-1, a_{i,i-1} = A_{i-1}), satisfy every order
  condition up to the scheme's order: 8 conditions (order 4) for LSRK4(5),
  all 17 (order 5) for LSRK5(9).  LSRK4(5) misses order 5.
* Their stability polynomials agree with exp(z) through z^4 and z^5.
* One step of the oracle's two-register loop equals that polynomial applied
  through repeated R (a linear autonomous problem).
* Bloch-wave analysis of the oracle's operator with these polynomials gives
  the paper's Table crit-Cr columns, in 3D and 2D: LSRK5(9) within 5%,
  LSRK4(5) within 12%.
"""
import math
import os

import numpy as np
import pytest

import crit_courant as cc
import oracle
import synth
from oracle import LSRK45_KCL_A, LSRK45_KCL_B, LSRK59_KCL_A, LSRK59_KCL_B

SCHEMES = {"lsrk45": (LSRK45_KCL_A, LSRK45_KCL_B, 4), "lsrk59": (LSRK59_KCL_A, LSRK59_KCL_B, 5)}


def butcher(A, B):
    s = len(B)
    a = np.zeros((s, s))
    for i in range(1, s):
        a[i, :i - 1] = B[:i - 1]
        a[i, i - 1] = A[i - 1]
    return a, np.array(B, float)


def order_conditions(a, b):
    """Residuals of the rooted-tree order conditions through order 5,
    grouped by order: sum over the tree's elementary weight minus 1/gamma."""
    c = a.sum(axis=1)
    ac = a @ c
    res = {1: [b.sum() - 1],
           2: [b @ c - 1 / 2],
           3: [b @ c ** 2 - 1 / 3, b @ ac - 1 / 6],
           4: [b @ c ** 3 - 1 / 4, b @ (c * ac) - 1 / 8, b @ (a @ c ** 2) - 1 / 12, b @ (a @ ac) - 1 / 24],
           5: [b @ c ** 4 - 1 / 5, b @ (c ** 2 * ac) - 1 / 10, b @ (c * (a @ c ** 2)) - 1 / 15,
               b @ (c * (a @ ac)) - 1 / 30, b @ ac ** 2 - 1 / 20, b @ (a @ c ** 3) - 1 / 20,
               b @ (a @ (c * ac)) - 1 / 40, b @ (a @ (a @ c ** 2)) - 1 / 60, b @ (a @ (a @ ac)) - 1 / 120]}
    return res


def stability_poly_2r(A, B):
    """gamma_j = b^T a^{j-1} 1 (gamma_0 = 1): the amplification polynomial."""
    a, b = butcher(A, B)
    g, v = [1.0], np.ones(len(b))
    for _ in range(len(b)):
        g.append(b @ v)
        v = a @ v
    return np.array(g)


@pytest.mark.parametrize("name", ["lsrk45", "lsrk59"])
def test_order_conditions(name):
    A, B, p = SCHEMES[name]
    res = order_conditions(*butcher(A, B))
    assert sum(len(res[q]) for q in range(1, 6)) == 17
    for q in range(1, p + 1):
        assert max(abs(r) for r in res[q]) < 1e-14, (name, q, res[q])
    if p < 5:
        assert max(abs(r) for r in res[5]) > 1e-4          # order 5 is not reached


@pytest.mark.parametrize("name", ["lsrk45", "lsrk59"])
def test_stability_polynomial(name):
    A, B, p = SCHEMES[name]
    g = stability_poly_2r(A, B)
    assert len(g) == len(B) + 1
    for j in range(p + 1):
        assert abs(g[j] - 1 / math.factorial(j)) < 1e-14, (name, j, g[j])
    assert abs(g[p + 1] - 1 / math.factorial(p + 1)) > 1e-6


@pytest.mark.parametrize("name", ["lsrk45", "lsrk59"])
def test_step_equals_polynomial(name):
    A, B, _ = SCHEMES[name]
    cfg = synth.configs.curved_pulse(N=2, k=2)
    o = oracle.Oracle(cfg["mesh"], 2, cfg["rho"], cfg["c"], 1.0)
    U0 = synth.configs.random_state(8, 2, 3)
    dt = 0.01
    U1 = o.lsrk2r(U0, dt, 1, A, B)
    g = stability_poly_2r(A, B)
    acc, term = g[0] * U0, U0
    for j in range(1, len(g)):
        term = dt * o.apply(term)
        acc = acc + g[j] * term
    assert np.abs(U1 - acc).max() / np.abs(U0).max() < 1e-14


GOLDEN3 = os.path.join(os.path.dirname(__file__), "golden", "crit_courant_3d.txt")


def _golden(path):
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, a, b, c = line.split()
            rows[int(k)] = (float(a), float(b), float(c))
    return rows


@pytest.fixture(scope="module", params=[1, 4])
def bloch3(request):
    return cc.Bloch(request.param)


def test_crit_courant_3d_paper_table(bloch3):
    ref = _golden(GOLDEN3)[bloch3.k]
    for name, col, tol in (("lsrk45", 0, 0.12), ("lsrk59", 1, 0.05)):
        g = stability_poly_2r(*SCHEMES[name][:2])
        cr = cc.bisect(lambda c: bloch3.lsrk_stable(c, g), lo=0.05, hi=1.5, tol=2e-3)
        assert abs(cr - ref[col]) <= tol * ref[col], (bloch3.k, name, cr, ref[col])


@pytest.mark.parametrize("k", [1, 4])
def test_crit_courant_2d_paper_table(k):
    from test_oracle_2d import Bloch2D, _bisect, _golden as golden2
    b = Bloch2D(k)
    ref = golden2()[k]
    for name, col, tol in (("lsrk45", 0, 0.12), ("lsrk59", 1, 0.05)):
        g = stability_poly_2r(*SCHEMES[name][:2])
        cr = _bisect(lambda c: b.lsrk_stable(c, g), 0.05, 1.8)
        assert abs(cr - ref[col]) <= tol * ref[col], (k, name, cr, ref[col])
