"""Dense-matrix FP64 oracle of the DG acoustic scheme (test infrastructure).

Scheme (the paper's Sec. 2 with the readings listed in the design notes):

* PDE, Sec. 2 Eq. (1): dv/dt + rho^-1 grad p = 0, dp/dt + rho c^2 div v = 0,
  state u = (p, v_x, v_y, v_z).
* Weak form, Sec. 2.1 Eq. (2), written with the coefficients on the mass
  terms so that the cell integrals are coefficient free:
      (rho w, dv/dt) - (div w, p) + <w.n, p*> = 0,
      ((rho c^2)^-1 q, dp/dt) - (grad q, v) + <q, (v.n)*> = 0,
  tensor-degree-k Lagrange polynomials on Gauss-Lobatto nodes (storage basis
  GL, Sec. 3.1), (k+1)^3 Gauss points in cells and (k+1)^2 on faces (Sec. 3).
  Semi-discrete form, Eq. (3): M dU/dt + K U = 0, and R(U) = -M^-1 K U.
* Flux, Sec. 2.4: with Z = rho c on each side, [[p]] = p- - p+,
  [[v.n]] = (v- - v+).n (n outward from the element):
      p*     = (Z+ p- + Z- p+)/(Z- + Z+) + alpha Z- Z+ [[v.n]]/(Z- + Z+)
      (v.n)* = (Z- v-.n + Z+ v+.n)/(Z- + Z+) + alpha [[p]]/(Z- + Z+)
  alpha = 1 is the upwind flux, which equals the HDG flux with
  tau = 1/(rho c) when Z- = Z+; alpha = 0 is the central flux.
  Walls use the mirror state p+ = p-, v+ = v- - 2 (v-.n) n, Z+ = Z-.
* LSRK: 2N-storage five-stage fourth-order scheme (Sec. 2.2),
      dU <- A_s dU + dt R(U);  U <- U + B_s dU,  s = 1..5;
  and the paper's two-register schemes LSRK4(5) and LSRK5(9) (Sec. 2.2):
      Y_{i+1} = S_i + dt A_i R(Y_i),  S_{i+1} = S_i + dt B_i R(Y_i),
  Y_1 = S_1 = u_n, u_{n+1} = S_{s+1}.
* ADER, Sec. 2.3 Eqs. (5)-(6): Ubar = sum_{j=0}^{k+1} dt^{j+1}/(j+1)! T_j with
  T_0 = u, T_j = -S T_{j-1} evaluated by collocation in the Gauss points
  (Algorithm 2), the degree reduced every second derivative by the
  reference-element L2 projection (Sec. 3.3, Algorithm 3), then
  U <- U + R(Ubar).

Parity pins (tests/test_oracle_*.py): exact quadrature of M and B on affine
elements against exact integrals; polynomial consistency R = -S u in interior
elements; the semi-discrete energy identity (central: 0, upwind: <= 0);
invariance under relabelled element axes; LSRK stability polynomials and,
for the two-register schemes, all Butcher order conditions up to their order
and the paper's critical Courant numbers; TCK terms against symbolic
(-S)^j u; convergence of both schemes to the analytic standing wave at the
expected rates; the energy 1/2 U^T M U and the L2 errors against closed
forms on graded meshes; on curved meshes, free-stream preservation (a
constant state is steady) wherever the Gauss rule integrates the metric
terms exactly (geometry degree q <= (k + 2) / 2), the same operator for
an affine map described by nodes of any degree, and the predictor of a
linear field of the discrete map in closed form.  Curved meshes with
variable coefficients are covered by the same code path; beyond these
identities and convergence, no value printed in the paper fixes them.
"""
import math
import numpy as np

from .basis import (gauss_1d, gauss_lobatto_1d, tensor_points,
                    tensor_weights, basis_3d, basis_grad_3d)

# Five-stage fourth-order 2N-storage Runge-Kutta (Carpenter & Kennedy, 1994).
LSRK54_A = [0.0,
            -567301805773.0 / 1357537059087.0,
            -2404267990393.0 / 2016746695238.0,
            -3550918686646.0 / 2091501179385.0,
            -1275806237668.0 / 842570457699.0]
LSRK54_B = [1432997174477.0 / 9575080441755.0,
            5161836677717.0 / 13612068292357.0,
            1720146321549.0 / 2090206949498.0,
            3134564353537.0 / 4481467310338.0,
            2277821191437.0 / 14882151754819.0]


# The two-register (2R) schemes of Kennedy, Carpenter & Lewis (2000), the
# paper's LSRK4(5) and LSRK5(9) (Sec. 2.2): RK4(3)5[2R+]C, five stages of
# order four, and RK5(4)9[2R+]S, nine stages of order five.  In Butcher form
# a_{i,j} = b_j for j < i-1 and a_{i,i-1} = A_{i-1}: stage i+1 starts from
# u_n plus all earlier increments weighted by b, except the newest, which
# is weighted by A_i.  Published coefficients (rationals).
LSRK45_KCL_A = [970286171893.0 / 4311952581923.0, 6584761158862.0 / 12103376702013.0,
                2251764453980.0 / 15575788980749.0, 26877169314380.0 / 34165994151039.0]
LSRK45_KCL_B = [1153189308089.0 / 22510343858157.0, 1772645290293.0 / 4653164025191.0,
                -1672844663538.0 / 4480602732383.0, 2114624349019.0 / 3568978502595.0,
                5198255086312.0 / 14908931495163.0]
LSRK59_KCL_A = [1107026461565.0 / 5417078080134.0, 38141181049399.0 / 41724347789894.0,
                493273079041.0 / 11940823631197.0, 1851571280403.0 / 6147804934346.0,
                11782306865191.0 / 62590030070788.0, 9452544825720.0 / 13648368537481.0,
                4435885630781.0 / 26285702406235.0, 2357909744247.0 / 11371140753790.0]
LSRK59_KCL_B = [2274579626619.0 / 23610510767302.0, 693987741272.0 / 12394497460941.0,
                -347131529483.0 / 15096185902911.0, 1144057200723.0 / 32081666971178.0,
                1562491064753.0 / 11797114684756.0, 13113619727965.0 / 44346030145118.0,
                393957816125.0 / 7825732611452.0, 720647959663.0 / 6565743875477.0,
                3559252274877.0 / 14424734981077.0]


def face_tangential_axes(f):
    d = f // 2
    return [a for a in range(3) if a != d]


def face_points(f, x1d):
    """Reference points [m^2, 3] on face f, tensor product of x1d along the
    face's two tangential axes (first tangential axis fastest)."""
    m = len(x1d)
    d, side = f // 2, (1.0 if f % 2 else -1.0)
    t0, t1 = face_tangential_axes(f)
    i = np.arange(m * m)
    pts = np.zeros((m * m, 3))
    pts[:, d] = side
    pts[:, t0] = x1d[i % m]
    pts[:, t1] = x1d[i // m]
    return pts


def orient_perm(o, m):
    """Index map own face point i + m j -> neighbour face point i' + m j'."""
    out = np.empty(m * m, np.int64)
    for j in range(m):
        for i in range(m):
            u, v = (j, i) if (o & 1) else (i, j)
            ip = m - 1 - u if (o & 2) else u
            jp = m - 1 - v if (o & 4) else v
            out[i + m * j] = ip + m * jp
    return out


class Oracle:
    """FP64 dense oracle on one mesh.

    mesh: dict as produced by ``synth.cube_mesh``; k: polynomial degree;
    rho, c: [E, (k+1)^3] nodal values at the GL solution nodes; alpha: flux
    parameter.  States are arrays [E, 4, (k+1)^3] in the GL basis, fields
    (p, v_x, v_y, v_z), nodes lexicographic with the first axis fastest.
    """

    def __init__(self, mesh, k, rho, c, alpha=1.0):
        self.k = k
        n = k + 1
        self.n = n
        self.alpha = float(alpha)
        self.E = E = int(mesh["n_elem"])
        self.nbr = np.asarray(mesh["nbr"], np.int64)
        self.nbr_face = np.asarray(mesh["nbr_face"], np.int64)
        self.orient = np.asarray(mesh["orient"], np.int64)
        self.X = np.asarray(mesh["nodes"], float)             # [E, Nq, 3]
        self.xgeo = gauss_lobatto_1d(int(mesh["geom_degree"]) + 1)
        self.xg, self.wg = gauss_1d(n)
        self.xgl = gauss_lobatto_1d(n)
        self.rho = np.asarray(rho, float).reshape(E, n ** 3)
        self.c = np.asarray(c, float).reshape(E, n ** 3)

        # ---- cell quadrature -------------------------------------------
        Q = tensor_points(self.xg)
        W = tensor_weights(self.wg)
        self.Phi = basis_3d(self.xgl, Q)                       # [nq, np]
        dPhi = basis_grad_3d(self.xgl, Q)                      # [3, nq, np]
        J = self.jacobian(Q)                                   # [E, nq, 3, 3]
        detJ = np.linalg.det(J)
        if np.any(detJ <= 0):
            raise ValueError("non-positive Jacobian determinant")
        Jinv = np.linalg.inv(J)
        rho_q = self.rho @ self.Phi.T
        c_q = self.c @ self.Phi.T
        wdet = W[None, :] * detJ
        self.wdet, self.rho_q, self.c_q = wdet, rho_q, c_q
        # mass matrices M[a, b] = sum_q w detJ chi phi_a phi_b, chi = rho (v)
        # or 1/(rho c^2) (p); inverted through a dense Cholesky factor
        Mv = np.einsum("qa,eq,qb->eab", self.Phi, wdet * rho_q, self.Phi)
        Mp = np.einsum("qa,eq,qb->eab", self.Phi, wdet / (rho_q * c_q ** 2), self.Phi)
        self.Mv, self.Mp = Mv, Mp
        self.Minv_v = self._chol_inverse(Mv)
        self.Minv_p = self._chol_inverse(Mp)
        # physical gradients of the basis G[e, i, q, a] and the cell matrices
        # B[e, i, a, b] = sum_q w detJ (d phi_a / d x_i) phi_b
        G = np.einsum("jqa,eqji->eiqa", dPhi, Jinv)
        self.B = np.einsum("eiqa,eq,qb->eiab", G, wdet, self.Phi)
        del G

        # ---- faces -------------------------------------------------------
        nf = n * n
        wf = np.outer(self.wg, self.wg).T.reshape(-1)          # w_i w_j, i fastest
        self.Ef = np.zeros((6, nf, n ** 3))
        self.Enb = np.zeros((E, 6, nf, n ** 3))
        self.s = np.zeros((E, 6, nf))
        self.nrm = np.zeros((E, 6, nf, 3))
        self.Zm = np.zeros((E, 6, nf))
        self.Zp = np.zeros((E, 6, nf))
        nb_cache = {}
        for f in range(6):
            Fq = face_points(f, self.xg)
            self.Ef[f] = basis_3d(self.xgl, Fq)
            Jf = self.jacobian(Fq)
            detJf = np.linalg.det(Jf)
            Jinvf = np.linalg.inv(Jf)
            d, side = f // 2, (1.0 if f % 2 else -1.0)
            # Nanson: n |J_f| = detJ J^-T n_ref, n_ref = side e_d
            nw = wf[None, :, None] * detJf[:, :, None] * side * Jinvf[:, :, d, :]
            s = np.linalg.norm(nw, axis=2)
            self.s[:, f] = s
            self.nrm[:, f] = nw / s[:, :, None]
            self.Zm[:, f] = (self.rho @ self.Ef[f].T) * (self.c @ self.Ef[f].T)
            for e in range(E):
                en = self.nbr[e, f]
                if en < 0:
                    self.Zp[e, f] = self.Zm[e, f]
                    continue
                key = (int(self.nbr_face[e, f]), int(self.orient[e, f]))
                if key not in nb_cache:
                    pts = face_points(key[0], self.xg)[orient_perm(key[1], n)]
                    nb_cache[key] = basis_3d(self.xgl, pts)
                Enb = nb_cache[key]
                self.Enb[e, f] = Enb
                self.Zp[e, f] = (Enb @ self.rho[en]) * (Enb @ self.c[en])
        self._tck_tables = {}

    # ------------------------------------------------------------------
    @staticmethod
    def _chol_inverse(M):
        L = np.linalg.cholesky(M)
        Linv = np.linalg.inv(L)
        return np.einsum("eka,ekb->eab", Linv, Linv)

    def positions(self, pts):
        """x[e, p, i] = sum_a X[e, a, i] psi_a(pts_p), psi = geometry basis."""
        psi = basis_3d(self.xgeo, pts)
        return np.einsum("pa,eai->epi", psi, self.X)

    def jacobian(self, pts):
        """J[e, p, i, j] = d x_i / d xi_j at reference points pts [P, 3]."""
        dpsi = basis_grad_3d(self.xgeo, pts)
        return np.einsum("jpa,eai->epij", dpsi, self.X)

    # ------------------------------------------------------------------
    def traces(self, U, f):
        """Own and neighbour traces [E, 4, n^2] at the Gauss points of face f,
        each evaluated from all coefficients of the element."""
        um = np.einsum("qa,eva->evq", self.Ef[f], U)
        nb = np.maximum(self.nbr[:, f], 0)
        up = np.einsum("eqa,eva->evq", self.Enb[:, f], U[nb])
        return um, up

    def apply(self, U):
        """R(U) = -M^-1 K U for a state U [E, 4, n^3] (GL coefficients)."""
        U = np.asarray(U, float)
        P, V = U[:, 0], U[:, 1:]
        r_v = np.einsum("eiab,eb->eia", self.B, P)
        r_p = np.einsum("eiab,eib->ea", self.B, V)
        a = self.alpha
        for f in range(6):
            um, up = self.traces(U, f)
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
        """Discrete energy 1/2 U^T M U = 1/2 sum_q w detJ (rho |v|^2 + p^2/(rho c^2))."""
        u = np.einsum("qa,eva->evq", self.Phi, np.asarray(U, float))
        dens = self.rho_q * np.sum(u[:, 1:] ** 2, axis=1) + u[:, 0] ** 2 / (self.rho_q * self.c_q ** 2)
        return 0.5 * float(np.sum(self.wdet * dens))

    def mass_inner(self, U, R):
        """U^T M R with the dense mass matrices."""
        return float(np.einsum("ea,eab,eb->", U[:, 0], self.Mp, R[:, 0])
                     + np.einsum("eia,eab,eib->", U[:, 1:], self.Mv, R[:, 1:]))

    # ------------------------------------------------------------------
    def lsrk(self, U, dt, nsteps, A=LSRK54_A, B=LSRK54_B, callback=None):
        """nsteps of the 2N-storage Runge-Kutta scheme (A_1 = 0)."""
        U = np.array(U, float, copy=True)
        dU = np.zeros_like(U)
        for step in range(nsteps):
            for s in range(len(A)):
                R = self.apply(U)
                dU = A[s] * dU + dt * R
                U = U + B[s] * dU
            if callback is not None:
                callback(step, U)
        return U

    def lsrk2r(self, U, dt, nsteps, A=LSRK59_KCL_A, B=LSRK59_KCL_B, callback=None):
        """nsteps of a two-register low-storage Runge-Kutta scheme: with
        k_i = R(Y_i), Y_1 = u_n and S_i = u_n + dt sum_{j<i} B_j k_j,
        Y_{i+1} = S_i + dt A_i k_i and u_{n+1} = S_{s+1}."""
        U = np.array(U, float, copy=True)
        s = len(B)
        for step in range(nsteps):
            acc = U.copy()
            Y = U
            for i in range(s):
                R = self.apply(Y)
                if i < s - 1:
                    Y = acc + dt * A[i] * R
                acc = acc + dt * B[i] * R
            U = acc
            if callback is not None:
                callback(step, U)
        return U

    def _tck_level(self, m):
        """Dense tables of the m-point Gauss set: collocation derivative
        D[d, q, b] = d psi_b / d xi_d (xi_q), geometry J^-1 and coefficients
        at the m^3 points, prolongation to the n-point set, and the reference
        L2 projection onto degree m-3 (m-2 points)."""
        if m in self._tck_tables:
            return self._tck_tables[m]
        n = self.n
        xm, wm = gauss_1d(m)
        Qm = tensor_points(xm)
        t = {"D": basis_grad_3d(xm, Qm)}
        Jm = self.jacobian(Qm)
        t["Jinv"] = np.linalg.inv(Jm)                          # [E, m3, 3, 3]
        phim = basis_3d(self.xgl, Qm)
        t["rho"] = self.rho @ phim.T
        t["c"] = self.c @ phim.T
        t["I"] = basis_3d(xm, tensor_points(self.xg))          # [n3, m3]
        if m - 2 >= 1:
            xr, _ = gauss_1d(m - 2)
            Wm = tensor_weights(wm)
            psi_r = basis_3d(xr, Qm)                           # [m3, (m-2)^3]
            mass = np.einsum("q,qa,qb->ab", Wm, psi_r, psi_r)
            rhs = np.einsum("q,qa,qb->ab", Wm, psi_r, np.eye(m ** 3))
            t["P"] = np.linalg.solve(mass, rhs)                # [(m-2)^3, m3]
        self._tck_tables[m] = t
        return t

    def _project(self, T, m, r):
        """Reference-element L2 projection of T (m-point Gauss values) onto
        the (m-r)-point Gauss Lagrange space; r = 2 uses the cached table."""
        if r == 2:
            return np.einsum("ab,evb->eva", self._tck_level(m)["P"], T)
        xm, wm = gauss_1d(m)
        xr, _ = gauss_1d(m - r)
        Qm = tensor_points(xm)
        Wm = tensor_weights(wm)
        psi_r = basis_3d(xr, Qm)
        mass = np.einsum("q,qa,qb->ab", Wm, psi_r, psi_r)
        P = np.linalg.solve(mass, (Wm[:, None] * psi_r).T)
        return np.einsum("ab,evb->eva", P, T)

    def tck(self, U, dt, reduce_every=2, return_terms=False, first=None):
        """Taylor-Cauchy-Kowalevski predictor Ubar (GL basis) of Eq. (6):
        sum_{j=0}^{k+1} dt^{j+1}/(j+1)! T_j, T_j = -S T_{j-1} by collocation
        at the current Gauss set, the set shrunk by ``reduce_every`` points
        after every ``reduce_every``-th derivative (0 = never).  ``first``
        (GL basis) replaces T_1 = -S U, as HDG-ADER does with the DG
        derivative (Eq. hdg-ader)."""
        U = np.asarray(U, float)
        n = self.n
        T = np.einsum("qa,eva->evq", self.Phi, U)              # values in G
        Ubar = dt * T
        terms = [(n, T)]
        m = n
        for j in range(1, self.k + 2):
            if m <= 0:
                break
            t = self._tck_level(m)
            if j == 1 and first is not None:
                Tn = np.einsum("qa,eva->evq", self.Phi, np.asarray(first, float))
            else:
                gp = np.einsum("dqb,eb->edq", t["D"], T[:, 0])
                gv = np.einsum("dqb,eib->eidq", t["D"], T[:, 1:])
                dp = np.einsum("eqdi,edq->eiq", t["Jinv"], gp)
                divv = np.einsum("eqdi,eidq->eq", t["Jinv"], gv)
                Tn = np.empty((self.E, 4, m ** 3))
                Tn[:, 1:] = -dp / t["rho"][:, None, :]
                Tn[:, 0] = -t["rho"] * t["c"] ** 2 * divv
            if reduce_every > 0 and j % reduce_every == 0:
                if m - reduce_every >= 1:
                    Tn = self._project(Tn, m, reduce_every)
                    m -= reduce_every
                else:
                    m = 0
                    terms.append((0, None))
                    break
            Ubar = Ubar + dt ** (j + 1) / math.factorial(j + 1) * np.einsum(
                "qb,evb->evq", self._tck_level(m)["I"], Tn)
            terms.append((m, Tn))
            T = Tn
        Ubar_gl = np.linalg.solve(self.Phi[None, None], Ubar[..., None])[..., 0]
        if return_terms:
            return Ubar_gl, terms
        return Ubar_gl

    def hdg_ader(self, U, dt, nsteps, reduce_every=2):
        """nsteps of HDG-ADER (Eq. hdg-ader): with W = -M^-1 K U the DG
        derivative, U <- U + dt W - M^-1 K sum_{j=1}^{k+1} dt^{j+1}/(j+1)!
        (-S)^{j-1} W.  Since -M^-1 K is linear this is U + R(Ubar) with the
        predictor's T_1 replaced by W."""
        U = np.array(U, float, copy=True)
        for _ in range(nsteps):
            W = self.apply(U)
            U = U + self.apply(self.tck(U, dt, reduce_every, first=W))
        return U

    def ader(self, U, dt, nsteps, reduce_every=2, callback=None):
        """nsteps of ADER: U <- U + R(Ubar), Eq. (6)."""
        U = np.array(U, float, copy=True)
        for step in range(nsteps):
            U = U + self.apply(self.tck(U, dt, reduce_every))
            if callback is not None:
                callback(step, U)
        return U

    # ------------------------------------------------------------------
    def l2_error(self, U, exact, t, extra=2):
        """Relative continuous L2 errors (pressure, velocity) against
        exact(x, t) -> [..., 4], with (n + extra)-point Gauss integration on
        the mapped elements."""
        xe, we = gauss_1d(self.n + extra)
        Qe = tensor_points(xe)
        W = tensor_weights(xe * 0 + we)
        phi = basis_3d(self.xgl, Qe)
        x = self.positions(Qe)
        detJ = np.linalg.det(self.jacobian(Qe))
        uh = np.einsum("qa,eva->eqv", phi, np.asarray(U, float))
        ue = exact(x, t)
        wd = W[None, :] * detJ
        ep = np.sum(wd * (uh[..., 0] - ue[..., 0]) ** 2) / np.sum(wd * ue[..., 0] ** 2)
        ev_den = np.sum(wd[..., None] * ue[..., 1:] ** 2)
        ev = np.sum(wd[..., None] * (uh[..., 1:] - ue[..., 1:]) ** 2) / max(ev_den, 1e-300)
        return float(np.sqrt(ep)), float(np.sqrt(ev))
