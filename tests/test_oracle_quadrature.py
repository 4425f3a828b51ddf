"""Pin: the oracle's element matrices equal exact integrals on affine
elements (Sec. 3: k+1 Gauss points per direction integrate the bilinear forms
exactly for element-wise constant coefficients on affine elements)."""
import numpy as np
import pytest

import oracle
from oracle import gauss_lobatto_1d
from oracle_helpers import single_element_mesh, poly1d_lagrange, exact_int


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_mass_and_cell_matrices_exact(k):
    n = k + 1
    A = np.array([[0.31, 0.05, -0.02], [0.03, 0.27, 0.04], [0.06, -0.01, 0.22]])
    mesh = single_element_mesh(A)
    rho, c = 1.7, 0.6
    o = oracle.Oracle(mesh, k, np.full((1, n ** 3), rho), np.full((1, n ** 3), c))
    nodes = gauss_lobatto_1d(n)
    L = [poly1d_lagrange(nodes, a) for a in range(n)]
    mm = np.array([[exact_int(L[a] * L[b]) for b in range(n)] for a in range(n)])
    dm = np.array([[exact_int(L[a].deriv() * L[b]) for b in range(n)] for a in range(n)])
    detA = np.linalg.det(A)
    Ainv = np.linalg.inv(A)
    idx = np.arange(n ** 3)
    a0, a1, a2 = idx % n, (idx // n) % n, idx // (n * n)
    M1 = mm[a0][:, a0] * mm[a1][:, a1] * mm[a2][:, a2]
    # int d phi_a / d xi_j * phi_b
    Dref = [dm[a0][:, a0] * mm[a1][:, a1] * mm[a2][:, a2],
            mm[a0][:, a0] * dm[a1][:, a1] * mm[a2][:, a2],
            mm[a0][:, a0] * mm[a1][:, a1] * dm[a2][:, a2]]
    assert np.allclose(o.Mv[0], rho * detA * M1, rtol=0, atol=1e-14 * abs(detA) * 8)
    assert np.allclose(o.Mp[0], detA * M1 / (rho * c * c), rtol=0, atol=1e-13 * abs(detA) * 8)
    for i in range(3):
        Bex = detA * sum(Ainv[j, i] * Dref[j] for j in range(3))
        assert np.allclose(o.B[0, i], Bex, rtol=0, atol=1e-12 * np.abs(Bex).max())


def test_face_measure_and_normal_affine():
    """Face quadrature weights sum to the face area; normals are the
    outward unit normals of the parallelepiped."""
    A = np.array([[0.31, 0.05, -0.02], [0.03, 0.27, 0.04], [0.06, -0.01, 0.22]])
    o = oracle.Oracle(single_element_mesh(A), 2, np.ones((1, 27)), np.ones((1, 27)))
    for f in range(6):
        d, side = f // 2, (1 if f % 2 else -1)
        t = [a for a in range(3) if a != d]
        area = np.linalg.norm(np.cross(A[:, t[0]], A[:, t[1]])) * 4.0
        assert abs(o.s[0, f].sum() - area) < 1e-14
        nexp = side * np.linalg.inv(A)[d]
        nexp /= np.linalg.norm(nexp)
        assert np.allclose(o.nrm[0, f], nexp[None, :], atol=1e-14)
