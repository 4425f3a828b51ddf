"""Dense-matrix FP64 oracle of the DG acoustic scheme in 2D (test
infrastructure only).

The same discrete scheme as oracle/dg.py one dimension down (the paper
treats d = 2 and d = 3 alike, Sec. 2): state u = (p, v_x, v_y) on
quadrilaterals, tensor-degree-k Lagrange polynomials on Gauss-Lobatto nodes,
(k+1)^2 Gauss points in cells and k+1 on each of the four faces, the
weighted-mass weak form, the impedance-weighted flux (upwind for alpha = 1,
central for alpha = 0) with mirror-state walls, the five-stage 2N-storage
LSRK and ADER with the Taylor terms collocated on shrinking Gauss sets.

Pins (tests/test_oracle_2d.py): exact quadrature of the mass and cell
matrices on an affine element, polynomial consistency R = -S u inside a
periodic mesh, the energy identity, invariance under rotated element frames,
convergence to the analytic standing wave, symbolic Taylor terms, and the
paper's 2D critical Courant numbers (Table crit-Cr) by Bloch-wave analysis.
"""
import math

import numpy as np

from .basis import gauss_1d, gauss_lobatto_1d, lagrange_1d, lagrange_deriv_1d
from .dg import LSRK54_A, LSRK54_B


def tensor_points_2d(x1d):
    """[m^2, 2] tensor-product points, first coordinate fastest."""
    m = len(x1d)
    i = np.arange(m * m)
    return np.stack([x1d[i % m], x1d[i // m]], axis=1)


def tensor_weights_2d(w1d):
    m = len(w1d)
    i = np.arange(m * m)
    return w1d[i % m] * w1d[i // m]


def basis_2d(nodes1d, pts):
    """phi[q, a] = 2D tensor Lagrange basis on nodes1d (a = a0 + n a1) at pts [Q, 2]."""
    n = len(nodes1d)
    L0, L1 = lagrange_1d(nodes1d, pts[:, 0]), lagrange_1d(nodes1d, pts[:, 1])
    a = np.arange(n * n)
    return L0[:, a % n] * L1[:, a // n]


def basis_grad_2d(nodes1d, pts):
    """dphi[d, q, a] = d/dxi_d of the 2D tensor Lagrange basis at pts."""
    n = len(nodes1d)
    L0, L1 = lagrange_1d(nodes1d, pts[:, 0]), lagrange_1d(nodes1d, pts[:, 1])
    D0, D1 = lagrange_deriv_1d(nodes1d, pts[:, 0]), lagrange_deriv_1d(nodes1d, pts[:, 1])
    a = np.arange(n * n)
    return np.stack([D0[:, a % n] * L1[:, a // n], L0[:, a % n] * D1[:, a // n]])


def face_points_2d(f, x1d):
    """Reference points [m, 2] on face f: x1d along the face's tangential axis."""
    d, side = f // 2, (1.0 if f % 2 else -1.0)
    pts = np.zeros((len(x1d), 2))
    pts[:, d] = side
    pts[:, 1 - d] = x1d
    return pts


class Oracle2D:
    """FP64 dense oracle on one 2D mesh (``synth.mesh2d.square_mesh``).
    States [E, 3, (k+1)^2] in the GL basis, fields (p, v_x, v_y)."""

    def __init__(self, mesh, k, rho, c, alpha=1.0):
        self.k = k
        n = self.n = k + 1
        self.alpha = float(alpha)
        self.E = E = int(mesh["n_elem"])
        self.nbr = np.asarray(mesh["nbr"], np.int64)
        self.nbr_face = np.asarray(mesh["nbr_face"], np.int64)
        self.orient = np.asarray(mesh["orient"], np.int64)
        self.X = np.asarray(mesh["nodes"], float)              # [E, (q+1)^2, 2]
        self.xgeo = gauss_lobatto_1d(int(mesh["geom_degree"]) + 1)
        self.xg, self.wg = gauss_1d(n)
        self.xgl = gauss_lobatto_1d(n)
        self.rho = np.asarray(rho, float).reshape(E, n * n)
        self.c = np.asarray(c, float).reshape(E, n * n)

        Q = tensor_points_2d(self.xg)
        W = tensor_weights_2d(self.wg)
        self.Phi = basis_2d(self.xgl, Q)
        dPhi = basis_grad_2d(self.xgl, Q)
        J = self.jacobian(Q)
        detJ = np.linalg.det(J)
        if np.any(detJ <= 0):
            raise ValueError("non-positive Jacobian determinant")
        Jinv = np.linalg.inv(J)
        rho_q, c_q = self.rho @ self.Phi.T, self.c @ self.Phi.T
        wdet = W[None, :] * detJ
        self.wdet, self.rho_q, self.c_q = wdet, rho_q, c_q
        self.Mv = np.einsum("qa,eq,qb->eab", self.Phi, wdet * rho_q, self.Phi)
        self.Mp = np.einsum("qa,eq,qb->eab", self.Phi, wdet / (rho_q * c_q ** 2), self.Phi)
        self.Minv_v = self._chol_inverse(self.Mv)
        self.Minv_p = self._chol_inverse(self.Mp)
        G = np.einsum("jqa,eqji->eiqa", dPhi, Jinv)            # physical gradients
        self.B = np.einsum("eiqa,eq,qb->eiab", G, wdet, self.Phi)

        self.Ef = np.zeros((4, n, n * n))
        self.Enb = np.zeros((E, 4, n, n * n))
        self.s = np.zeros((E, 4, n))
        self.nrm = np.zeros((E, 4, n, 2))
        self.Zm = np.zeros((E, 4, n))
        self.Zp = np.zeros((E, 4, n))
        for f in range(4):
            Fq = face_points_2d(f, self.xg)
            self.Ef[f] = basis_2d(self.xgl, Fq)
            Jf = self.jacobian(Fq)
            detJf, Jinvf = np.linalg.det(Jf), np.linalg.inv(Jf)
            d, side = f // 2, (1.0 if f % 2 else -1.0)
            nw = self.wg[None, :, None] * detJf[:, :, None] * side * Jinvf[:, :, d, :]
            s = np.linalg.norm(nw, axis=2)
            self.s[:, f] = s
            self.nrm[:, f] = nw / s[:, :, None]
            self.Zm[:, f] = (self.rho @ self.Ef[f].T) * (self.c @ self.Ef[f].T)
            for e in range(E):
                en = self.nbr[e, f]
                if en < 0:
                    self.Zp[e, f] = self.Zm[e, f]
                    continue
                pts = face_points_2d(int(self.nbr_face[e, f]), self.xg)
                if self.orient[e, f]:
                    pts = pts[::-1]
                Enb = basis_2d(self.xgl, pts)
                self.Enb[e, f] = Enb
                self.Zp[e, f] = (Enb @ self.rho[en]) * (Enb @ self.c[en])
        self._tck_tables = {}

    @staticmethod
    def _chol_inverse(M):
        L = np.linalg.cholesky(M)
        Linv = np.linalg.inv(L)
        return np.einsum("eka,ekb->eab", Linv, Linv)

    def positions(self, pts):
        psi = basis_2d(self.xgeo, pts)
        return np.einsum("pa,eai->epi", psi, self.X)

    def jacobian(self, pts):
        """J[e, p, i, j] = d x_i / d xi_j."""
        dpsi = basis_grad_2d(self.xgeo, pts)
        return np.einsum("jpa,eai->epij", dpsi, self.X)

    def apply(self, U):
        """R(U) = -M^-1 K U for U [E, 3, n^2]."""
        U = np.asarray(U, float)
        P, V = U[:, 0], U[:, 1:]
        r_v = np.einsum("eiab,eb->eia", self.B, P)
        r_p = np.einsum("eiab,eib->ea", self.B, V)
        a = self.alpha
        nb_all = np.maximum(self.nbr, 0)
        for f in range(4):
            um = np.einsum("qa,eva->evq", self.Ef[f], U)
            up = np.einsum("eqa,eva->evq", self.Enb[:, f], U[nb_all[:, f]])
            n = self.nrm[:, f]
            vm_n = np.einsum("eiq,eqi->eq", um[:, 1:], n)
            vp_n = np.einsum("eiq,eqi->eq", up[:, 1:], n)
            pm, pp = um[:, 0], up[:, 0]
            wall = self.nbr[:, f] < 0
            pp = np.where(wall[:, None], pm, pp)
            vp_n = np.where(wall[:, None], -vm_n, vp_n)
            Zm, Zp = self.Zm[:, f], self.Zp[:, f]
            Zs = Zm + Zp
            pstar = (Zp * pm + Zm * pp) / Zs + a * Zm * Zp * (vm_n - vp_n) / Zs
            vnstar = (Zm * vm_n + Zp * vp_n) / Zs + a * (pm - pp) / Zs
            s = self.s[:, f]
            r_v -= np.einsum("qa,eq,eqi->eia", self.Ef[f], s * pstar, n)
            r_p -= np.einsum("qa,eq->ea", self.Ef[f], s * vnstar)
        R = np.empty_like(U)
        R[:, 0] = np.einsum("eab,eb->ea", self.Minv_p, r_p)
        R[:, 1:] = np.einsum("eab,eib->eia", self.Minv_v, r_v)
        return R

    def energy(self, U):
        u = np.einsum("qa,eva->evq", self.Phi, np.asarray(U, float))
        dens = self.rho_q * np.sum(u[:, 1:] ** 2, axis=1) + u[:, 0] ** 2 / (self.rho_q * self.c_q ** 2)
        return 0.5 * float(np.sum(self.wdet * dens))

    def mass_inner(self, U, R):
        return float(np.einsum("ea,eab,eb->", U[:, 0], self.Mp, R[:, 0])
                     + np.einsum("eia,eab,eib->", U[:, 1:], self.Mv, R[:, 1:]))

    def lsrk(self, U, dt, nsteps, A=LSRK54_A, B=LSRK54_B):
        U = np.array(U, float, copy=True)
        dU = np.zeros_like(U)
        for _ in range(nsteps):
            for s in range(len(A)):
                dU = A[s] * dU + dt * self.apply(U)
                U = U + B[s] * dU
        return U

    def _level(self, m):
        """Collocation derivative, J^-1 and coefficients at the m-point Gauss
        set, and the prolongation to the n-point set."""
        if m in self._tck_tables:
            return self._tck_tables[m]
        xm, _ = gauss_1d(m)
        Qm = tensor_points_2d(xm)
        phim = basis_2d(self.xgl, Qm)
        t = {"D": basis_grad_2d(xm, Qm), "Jinv": np.linalg.inv(self.jacobian(Qm)),
             "rho": self.rho @ phim.T, "c": self.c @ phim.T,
             "I": basis_2d(xm, tensor_points_2d(self.xg))}
        self._tck_tables[m] = t
        return t

    @staticmethod
    def _project(T, m, r):
        """Reference L2 projection from the m-point to the (m-r)-point Gauss
        Lagrange space (dense mass-matrix solve)."""
        xm, wm = gauss_1d(m)
        xr, _ = gauss_1d(m - r)
        Qm = tensor_points_2d(xm)
        Wm = tensor_weights_2d(wm)
        psi = basis_2d(xr, Qm)
        mass = np.einsum("q,qa,qb->ab", Wm, psi, psi)
        P = np.linalg.solve(mass, (Wm[:, None] * psi).T)
        return np.einsum("ab,evb->eva", P, T)

    def tck(self, U, dt, reduce_every=2, return_terms=False, first=None):
        """Predictor Ubar (GL) = sum_{j=0}^{k+1} dt^{j+1}/(j+1)! T_j, T_j = -S
        T_{j-1} collocated at the current Gauss set, which shrinks by
        reduce_every points after every reduce_every-th derivative."""
        U = np.asarray(U, float)
        T = np.einsum("qa,eva->evq", self.Phi, U)
        Ubar = dt * T
        terms = [(self.n, T)]
        m = self.n
        for j in range(1, self.k + 2):
            if m <= 0:
                break
            t = self._level(m)
            if j == 1 and first is not None:
                Tn = np.einsum("qa,eva->evq", self.Phi, np.asarray(first, float))
            else:
                gp = np.einsum("dqb,eb->edq", t["D"], T[:, 0])
                gv = np.einsum("dqb,eib->eidq", t["D"], T[:, 1:])
                dp = np.einsum("eqdi,edq->eiq", t["Jinv"], gp)
                divv = np.einsum("eqdi,eidq->eq", t["Jinv"], gv)
                Tn = np.empty((self.E, 3, m * m))
                Tn[:, 1:] = -dp / t["rho"][:, None, :]
                Tn[:, 0] = -t["rho"] * t["c"] ** 2 * divv
            if reduce_every > 0 and j % reduce_every == 0:
                if m - reduce_every >= 1:
                    Tn = self._project(Tn, m, reduce_every)
                    m -= reduce_every
                else:
                    terms.append((0, None))
                    break
            Ubar = Ubar + dt ** (j + 1) / math.factorial(j + 1) * np.einsum(
                "qb,evb->evq", self._level(m)["I"], Tn)
            terms.append((m, Tn))
            T = Tn
        Ubar_gl = np.linalg.solve(self.Phi[None, None], Ubar[..., None])[..., 0]
        return (Ubar_gl, terms) if return_terms else Ubar_gl

    def ader(self, U, dt, nsteps, reduce_every=2):
        U = np.array(U, float, copy=True)
        for _ in range(nsteps):
            U = U + self.apply(self.tck(U, dt, reduce_every))
        return U

    def l2_error(self, U, exact, t, extra=2):
        """Relative continuous L2 errors (p, v) against exact(x, t) -> [..., 3]."""
        xe, we = gauss_1d(self.n + extra)
        Qe = tensor_points_2d(xe)
        W = tensor_weights_2d(we)
        phi = basis_2d(self.xgl, Qe)
        x = self.positions(Qe)
        detJ = np.linalg.det(self.jacobian(Qe))
        uh = np.einsum("qa,eva->eqv", phi, np.asarray(U, float))
        ue = exact(x, t)
        wd = W[None, :] * detJ
        ep = np.sum(wd * (uh[..., 0] - ue[..., 0]) ** 2) / np.sum(wd * ue[..., 0] ** 2)
        ev = np.sum(wd[..., None] * (uh[..., 1:] - ue[..., 1:]) ** 2) / max(np.sum(wd[..., None] * ue[..., 1:] ** 2), 1e-300)
        return float(np.sqrt(ep)), float(np.sqrt(ev))
