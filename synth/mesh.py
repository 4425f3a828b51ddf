"""Structured cube meshes of hexahedra, described the way the C ABI expects.

Mesh description (a dict of numpy arrays):

* ``nodes``    float64 [E, (q+1)^3, 3]: physical positions of the element's
  geometry nodes, placed at the tensor-product Gauss-Lobatto points of degree
  ``q`` of the reference cube [-1, 1]^3, lexicographic with the first
  reference axis fastest.
* ``nbr``      int32 [E, 6]: neighbour element across local face f, -1 = wall.
  Faces: 0 = -xi, 1 = +xi, 2 = -eta, 3 = +eta, 4 = -zeta, 5 = +zeta.
* ``nbr_face`` int8 [E, 6]: the neighbour's local face index (-1 at walls).
* ``orient``   int8 [E, 6]: how a point of this face is found on the
  neighbour's face.  The two tangential axes of face f are the two reference
  axes other than f // 2, in increasing order; a face point has indices (i, j)
  along them.  Code o maps (i, j) to the neighbour's (i', j'): first
  (u, v) = (j, i) if o & 1 else (i, j); then i' = n-1-u if o & 2 else u and
  j' = n-1-v if o & 4 else v.  Both the Gauss and the Gauss-Lobatto point sets
  are symmetric, so the same code serves either set.

Periodicity is expressed only through ``nbr``.  Each element may carry its own
right-handed relabelling of the reference axes (a signed permutation with
determinant +1), which exercises the orientation codes.
"""
import numpy as np


def gll_points_1d(q):
    """Gauss-Lobatto points of degree q (q+1 points) on [-1, 1], ascending.

    Used only to place geometry and solution nodes of the synthetic meshes.
    """
    if q < 1:
        raise ValueError("degree must be >= 1")
    if q == 1:
        return np.array([-1.0, 1.0])
    leg = np.polynomial.legendre.Legendre.basis(q)
    dleg = leg.deriv()
    r = np.sort(dleg.roots().real)
    # a few Newton steps on P'_q polish the companion-matrix roots
    d2 = dleg.deriv()
    for _ in range(3):
        r = r - dleg(r) / d2(r)
    x = np.concatenate(([-1.0], r, [1.0]))
    return 0.5 * (x - x[::-1])  # exact symmetry


def _tensor_points(x1d):
    n = len(x1d)
    idx = np.arange(n ** 3)
    return np.stack([x1d[idx % n], x1d[(idx // n) % n], x1d[idx // (n * n)]], axis=1)


_EVEN_PERMS = [(0, 1, 2), (1, 2, 0), (2, 0, 1)]
_ODD_PERMS = [(1, 0, 2), (0, 2, 1), (2, 1, 0)]


def random_frames(n_elem, rng):
    """Random right-handed signed permutation matrices, one per element."""
    frames = np.zeros((n_elem, 3, 3))
    for e in range(n_elem):
        while True:
            perm = [_EVEN_PERMS, _ODD_PERMS][rng.integers(2)][rng.integers(3)]
            signs = rng.choice([-1.0, 1.0], size=3)
            R = np.zeros((3, 3))
            for col, row in enumerate(perm):
                R[row, col] = signs[col]
            if np.linalg.det(R) > 0:
                frames[e] = R
                break
    return frames


def _undeformed(mesh_info, e, xi):
    """Undeformed physical position of reference points xi [m, 3] in element e."""
    N, h = mesh_info["N"], mesh_info["h"]
    ex, ey, ez = e % N, (e // N) % N, e // (N * N)
    centre = np.array([ex + 0.5, ey + 0.5, ez + 0.5]) * h
    R = mesh_info["frames"][e]
    return centre[None, :] + 0.5 * h * (xi @ R.T)


def cube_mesh(N, q=1, periodic=True, deform=None, frames=None):
    """Unit cube split into N^3 hexahedra.

    ``deform`` is an optional callable x[..., 3] -> x'[..., 3] applied to the
    geometry nodes (curving); ``frames`` optional [E, 3, 3] signed permutations
    relabelling each element's reference axes (identity when None).
    """
    E = N ** 3
    h = 1.0 / N
    if frames is None:
        return _cube_mesh_aligned(N, q, periodic, deform)
    info = {"N": N, "h": h, "frames": frames, "deform": deform}
    xg = _tensor_points(gll_points_1d(q))
    nodes = np.empty((E, (q + 1) ** 3, 3))
    for e in range(E):
        x0 = _undeformed(info, e, xg)
        nodes[e] = deform(x0) if deform is not None else x0
    nbr = np.full((E, 6), -1, np.int32)
    nbr_face = np.full((E, 6), -1, np.int8)
    orient = np.zeros((E, 6), np.int8)
    per = (periodic,) * 3 if isinstance(periodic, bool) else tuple(periodic)
    for e in range(E):
        ijk = np.array([e % N, (e // N) % N, e // (N * N)])
        R = frames[e]
        for f in range(6):
            d, s = f // 2, (1.0 if f % 2 else -1.0)
            out = s * R[:, d]                       # outward direction, global
            D = int(np.argmax(np.abs(out)))
            step = int(round(out[D]))
            nb = ijk.copy()
            nb[D] += step
            if nb[D] < 0 or nb[D] >= N:
                if not per[D]:
                    continue
                nb[D] %= N
            en = int(nb[0] + N * nb[1] + N * N * nb[2])
            Rn = frames[en]
            # neighbour face whose outward direction is opposite
            fn = None
            for g in range(6):
                dn, sn = g // 2, (1.0 if g % 2 else -1.0)
                if np.allclose(sn * Rn[:, dn], -out):
                    fn = g
                    break
            t = [a for a in range(3) if a != d]
            tn = [a for a in range(3) if a != fn // 2]
            c00 = R[:, t[0]] @ Rn[:, tn[0]]
            if abs(c00) > 0.5:
                code = 0
                if R[:, t[0]] @ Rn[:, tn[0]] < 0:
                    code |= 2
                if R[:, t[1]] @ Rn[:, tn[1]] < 0:
                    code |= 4
            else:
                code = 1
                if R[:, t[1]] @ Rn[:, tn[0]] < 0:
                    code |= 2
                if R[:, t[0]] @ Rn[:, tn[1]] < 0:
                    code |= 4
            nbr[e, f], nbr_face[e, f], orient[e, f] = en, fn, code
    return {
        "n_elem": E, "geom_degree": q, "nodes": nodes, "nbr": nbr,
        "nbr_face": nbr_face, "orient": orient, "N": N, "h": h,
        "frames": frames, "deform": deform, "periodic": per,
    }


def _element_ijk(N):
    e = np.arange(N ** 3)
    return np.stack([e % N, (e // N) % N, e // (N * N)], axis=1)


def _cube_mesh_aligned(N, q, periodic, deform):
    """cube_mesh with every element's reference axes along the global axes
    (vectorised; orientation codes are all 0)."""
    E, h = N ** 3, 1.0 / N
    ijk = _element_ijk(N)
    xg = _tensor_points(gll_points_1d(q))
    x0 = (ijk[:, None, :] + 0.5) * h + 0.5 * h * xg[None, :, :]
    nodes = deform(x0) if deform is not None else x0
    per = (periodic,) * 3 if isinstance(periodic, bool) else tuple(periodic)
    nbr = np.full((E, 6), -1, np.int32)
    nbr_face = np.full((E, 6), -1, np.int8)
    for f in range(6):
        d, step = f // 2, (1 if f % 2 else -1)
        nb = ijk.copy()
        nb[:, d] += step
        inside = (nb[:, d] >= 0) & (nb[:, d] < N)
        if per[d]:
            nb[:, d] %= N
            inside[:] = True
        en = nb[:, 0] + N * nb[:, 1] + N * N * nb[:, 2]
        nbr[inside, f] = en[inside]
        nbr_face[inside, f] = f ^ 1
    return {
        "n_elem": E, "geom_degree": q, "nodes": np.ascontiguousarray(nodes), "nbr": nbr,
        "nbr_face": nbr_face, "orient": np.zeros((E, 6), np.int8), "N": N, "h": h,
        "frames": None, "deform": deform, "periodic": per,
    }


def solution_node_positions(mesh, k):
    """Physical positions [E, (k+1)^3, 3] of the degree-k Gauss-Lobatto
    solution nodes, through the exact (analytic) deformation map."""
    xg = _tensor_points(gll_points_1d(k))
    E = mesh["n_elem"]
    if mesh["frames"] is None:
        N, h = mesh["N"], mesh["h"]
        x0 = (_element_ijk(N)[:, None, :] + 0.5) * h + 0.5 * h * xg[None, :, :]
        return mesh["deform"](x0) if mesh["deform"] is not None else x0
    out = np.empty((E, xg.shape[0], 3))
    for e in range(E):
        x0 = _undeformed(mesh, e, xg)
        out[e] = mesh["deform"](x0) if mesh["deform"] is not None else x0
    return out


def curving(a):
    """x_i <- x_i + a * prod_j sin(2 pi x_j), the same scalar for each i."""
    def f(x):
        s = np.sin(2 * np.pi * x[..., 0]) * np.sin(2 * np.pi * x[..., 1]) * np.sin(2 * np.pi * x[..., 2])
        return x + a * s[..., None]
    return f
