"""Critical Courant numbers of the oracle's schemes by Bloch-wave analysis.

On a periodic Cartesian mesh with constant coefficients the operator is
translation invariant, so its spectrum is the union over wave numbers theta
of the spectra of the 4n^3 x 4n^3 symbols
    L(theta) = L_00 + sum_d (L_{0,+d} e^{i theta_d} + L_{0,-d} e^{-i theta_d}).
The blocks are read off the oracle by applying it to unit vectors of one
element.  LSRK is stable when |g(dt lambda)| <= 1 for its stability
polynomial g; ADER when the spectral radius of I + L(theta) T(dt) is <= 1,
T(dt) being the element-local TCK map.

Stability criterion: growth below 1% over 1000 steps, i.e. |g| or the
spectral radius <= 1 + 1e-5.  The paper finds its limits by running
simulations; a strict |g| <= 1 would flag the slow growth that Taylor
polynomials of order 5 (ADER at k = 4) show for eigenvalues close to the
imaginary axis, which no finite run detects.
"""
import itertools

import numpy as np

import synth
import oracle

GROWTH_TOL = 1e-5


def _unit_responses(fn, E, nd):
    cols = []
    for i in range(nd):
        U = np.zeros((E, nd))
        U[0, i] = 1.0
        cols.append(fn(U).reshape(E, nd))
    return np.stack(cols, axis=-1)          # [E, nd, nd]: response in e to a source in element 0


class Bloch:
    def __init__(self, k):
        self.k = k
        n = k + 1
        self.nd = 4 * n ** 3
        mesh = synth.cube_mesh(3, q=1, periodic=True)
        ones = np.ones((27, n ** 3))
        self.o = oracle.Oracle(mesh, k, ones, ones, 1.0)
        self.h = 1.0 / 3
        shp = (27, 4, n ** 3)
        self.Lcol = _unit_responses(lambda U: self.o.apply(U.reshape(shp)), 27, self.nd)
        th = np.linspace(0, np.pi, 4)
        self.thetas = [t for t in itertools.product(th, th, th) if t[0] >= t[1] >= t[2]]
        self.symbols = [self.symbol(t) for t in self.thetas]
        self.eigs = np.concatenate([np.linalg.eigvals(S) for S in self.symbols])

    def symbol(self, theta):
        L = self.Lcol[0].astype(complex)
        for d, s in enumerate((1, 3, 9)):
            L = L + self.Lcol[2 * s] * np.exp(1j * theta[d]) + self.Lcol[s] * np.exp(-1j * theta[d])
        return L

    def dt(self, cr):
        return cr * self.h / self.k ** 1.5

    def lsrk_stable(self, cr, gamma):
        z = self.dt(cr) * self.eigs
        g = np.polynomial.polynomial.polyval(z, gamma)
        return np.abs(g).max() <= 1.0 + GROWTH_TOL

    def tck_matrix(self, dt, reduce_every=2):
        """Element-local TCK map (GL -> GL), nd x nd.  The predictor acts on
        each element alone, so the 27 elements carry 27 different unit
        vectors per call."""
        n3 = (self.k + 1) ** 3
        T = np.zeros((self.nd, self.nd))
        for start in range(0, self.nd, 27):
            U = np.zeros((27, self.nd))
            cols = list(range(start, min(start + 27, self.nd)))
            for e, i in enumerate(cols):
                U[e, i] = 1.0
            out = self.o.tck(U.reshape(27, 4, n3), dt, reduce_every).reshape(27, self.nd)
            for e, i in enumerate(cols):
                T[:, i] = out[e]
        return T

    def ader_stable(self, cr, reduce_every=2):
        T = self.tck_matrix(self.dt(cr), reduce_every)
        I = np.eye(self.nd)
        rad = max(np.abs(np.linalg.eigvals(I + S @ T)).max() for S in self.symbols)
        return rad <= 1.0 + GROWTH_TOL


def bisect(stable, lo=0.01, hi=1.5, tol=2e-3):
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if stable(mid):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
