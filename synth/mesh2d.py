"""Synthetic 2D meshes: the unit square split into N^2 quadrilaterals.

Same conventions as the 3D meshes, one dimension down:

* element e = i + N j; reference square [-1, 1]^2, node order first axis
  fastest;
* faces (edges) 0: xi = -1, 1: xi = +1, 2: eta = -1, 3: eta = +1;
* ``nbr[e][f]`` the neighbour element across face f (-1 = wall),
  ``nbr_face[e][f]`` the neighbour's face index, ``orient[e][f]`` 1 when the
  neighbour's face coordinate runs opposite to this element's (face point i
  of e meets face point n-1-i of the neighbour), else 0.

Each element may carry its own rotation of the reference axes (a signed
permutation with determinant +1), which exercises the orientation codes.
"""
import numpy as np

from .mesh import gll_points_1d

_ROTATIONS = [np.array([[1.0, 0.0], [0.0, 1.0]]), np.array([[0.0, -1.0], [1.0, 0.0]]),
              np.array([[-1.0, 0.0], [0.0, -1.0]]), np.array([[0.0, 1.0], [-1.0, 0.0]])]


def _tensor_points_2d(x1d):
    n = len(x1d)
    idx = np.arange(n * n)
    return np.stack([x1d[idx % n], x1d[idx // n]], axis=1)


def random_frames_2d(n_elem, rng):
    """Random rotations by multiples of 90 degrees, one per element."""
    return np.stack([_ROTATIONS[rng.integers(4)] for _ in range(n_elem)])


def _undeformed(N, h, R, e, xi):
    centre = np.array([e % N + 0.5, e // N + 0.5]) * h
    return centre[None, :] + 0.5 * h * (xi @ R.T)


def square_mesh(N, q=1, periodic=True, deform=None, frames=None):
    """Unit square split into N^2 quadrilaterals; ``deform`` maps x[..., 2]
    to x'[..., 2] (curving), ``frames`` [E, 2, 2] rotations of the
    reference axes (identity when None)."""
    E, h = N * N, 1.0 / N
    if frames is None:
        frames = np.broadcast_to(_ROTATIONS[0], (E, 2, 2))
    xg = _tensor_points_2d(gll_points_1d(q))
    nodes = np.empty((E, (q + 1) ** 2, 2))
    for e in range(E):
        x0 = _undeformed(N, h, frames[e], e, xg)
        nodes[e] = deform(x0) if deform is not None else x0
    per = (periodic,) * 2 if isinstance(periodic, bool) else tuple(periodic)
    nbr = np.full((E, 4), -1, np.int32)
    nbr_face = np.full((E, 4), -1, np.int8)
    orient = np.zeros((E, 4), np.int8)
    for e in range(E):
        ij = np.array([e % N, e // N])
        R = frames[e]
        for f in range(4):
            d, s = f // 2, (1.0 if f % 2 else -1.0)
            out = s * R[:, d]                           # outward direction, global
            D = int(np.argmax(np.abs(out)))
            step = int(round(out[D]))
            nb = ij.copy()
            nb[D] += step
            if nb[D] < 0 or nb[D] >= N:
                if not per[D]:
                    continue
                nb[D] %= N
            en = int(nb[0] + N * nb[1])
            Rn = frames[en]
            fn = next(g for g in range(4) if np.allclose((1.0 if g % 2 else -1.0) * Rn[:, g // 2], -out))
            t, tn = 1 - d, 1 - fn // 2                  # tangential reference axes
            nbr[e, f], nbr_face[e, f] = en, fn
            orient[e, f] = 1 if R[:, t] @ Rn[:, tn] < 0 else 0
    return {"n_elem": E, "geom_degree": q, "nodes": nodes, "nbr": nbr, "nbr_face": nbr_face,
            "orient": orient, "N": N, "h": h, "frames": np.array(frames), "deform": deform,
            "periodic": per, "dim": 2}


def solution_node_positions_2d(mesh, k):
    """Physical positions [E, (k+1)^2, 2] of the degree-k Gauss-Lobatto
    solution nodes, through the exact deformation map."""
    xg = _tensor_points_2d(gll_points_1d(k))
    N, h = mesh["N"], mesh["h"]
    out = np.empty((mesh["n_elem"], xg.shape[0], 2))
    for e in range(mesh["n_elem"]):
        x0 = _undeformed(N, h, mesh["frames"][e], e, xg)
        out[e] = mesh["deform"](x0) if mesh["deform"] is not None else x0
    return out


def curving_2d(a):
    """x_i <- x_i + a sin(2 pi x) sin(2 pi y), the same scalar for each i."""
    def deform(x):
        s = a * np.sin(2 * np.pi * x[..., 0]) * np.sin(2 * np.pi * x[..., 1])
        return x + s[..., None]
    return deform


def standing_wave_2d(x, t):
    """Standing wave on the periodic unit square for rho = c = 1:
    p = cos(2 pi x) cos(2 pi y) cos(w t), w = 2 pi sqrt(2),
    v_x = (2 pi / w) sin(2 pi x) cos(2 pi y) sin(w t), v_y likewise."""
    w = 2 * np.pi * np.sqrt(2.0)
    cx, cy = np.cos(2 * np.pi * x[..., 0]), np.cos(2 * np.pi * x[..., 1])
    sx, sy = np.sin(2 * np.pi * x[..., 0]), np.sin(2 * np.pi * x[..., 1])
    amp = 2 * np.pi / w * np.sin(w * t)
    return np.stack([cx * cy * np.cos(w * t), amp * sx * cy, amp * cx * sy], axis=-1)


def membrane_modes_2d(x, t, modes=((1, 1), (1, 2), (2, 1), (2, 2), (1, 3), (3, 1), (3, 3))):
    """Sum of standing modes of the square with rho = c = 1 on the periodic
    unit square: p = sum_m cos(2 pi a_m x) cos(2 pi b_m y) cos(w_m t),
    w_m = 2 pi sqrt(a_m^2 + b_m^2), with the matching velocities."""
    out = 0.0
    for a, b in modes:
        w = 2 * np.pi * np.sqrt(a * a + b * b)
        cx, cy = np.cos(2 * np.pi * a * x[..., 0]), np.cos(2 * np.pi * b * x[..., 1])
        sx, sy = np.sin(2 * np.pi * a * x[..., 0]), np.sin(2 * np.pi * b * x[..., 1])
        out = out + np.stack([cx * cy * np.cos(w * t), (2 * np.pi * a / w) * sx * cy * np.sin(w * t),
                              (2 * np.pi * b / w) * cx * sy * np.sin(w * t)], axis=-1)
    return out


def pack_state_2d(vals):
    """vals [E, n^2, 3] -> U [E, 3, n^2]."""
    return np.ascontiguousarray(np.transpose(vals, (0, 2, 1)))


def standing_wave_config_2d(N=4, k=3, cr=0.2, frames_seed=None, exact=standing_wave_2d):
    """Periodic affine square, rho = c = 1, a standing solution."""
    frames = None
    if frames_seed is not None:
        frames = random_frames_2d(N * N, np.random.default_rng(frames_seed))
    mesh = square_mesh(N, q=1, periodic=True, frames=frames)
    x = solution_node_positions_2d(mesh, k)
    E, n2 = x.shape[0], x.shape[1]
    return {"mesh": mesh, "k": k, "rho": np.ones((E, n2)), "c": np.ones((E, n2)),
            "U0": pack_state_2d(exact(x, 0.0)), "alpha": 1.0,
            "dt": cr * mesh["h"] / k ** 1.5, "exact": exact, "xnodes": x}


def curved_config_2d(N=4, k=3, seed=2, a=0.05, cr=0.1, frames_seed=None, periodic=False):
    """Curved square with variable coefficients (c = 1 + 0.5 sin 2 pi x cos 2 pi y,
    rho = 1 + 0.3 cos 2 pi y) and a seeded Gaussian pressure pulse (width 0.05)."""
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0.25, 0.75, size=2)
    frames = None
    if frames_seed is not None:
        frames = random_frames_2d(N * N, np.random.default_rng(frames_seed))
    mesh = square_mesh(N, q=k, periodic=periodic, deform=curving_2d(a), frames=frames)
    x = solution_node_positions_2d(mesh, k)
    c = 1.0 + 0.5 * np.sin(2 * np.pi * x[..., 0]) * np.cos(2 * np.pi * x[..., 1])
    rho = 1.0 + 0.3 * np.cos(2 * np.pi * x[..., 1])
    p = np.exp(-np.sum((x - x0) ** 2, axis=-1) / (2 * 0.05 ** 2))
    z = np.zeros_like(p)
    return {"mesh": mesh, "k": k, "rho": rho, "c": c, "U0": pack_state_2d(np.stack([p, z, z], axis=-1)),
            "alpha": 1.0, "dt": cr * mesh["h"] / (1.5 * k ** 1.5), "exact": None, "xnodes": x}


def random_state_2d(E, k, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(E, 3, (k + 1) ** 2))
