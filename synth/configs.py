"""The five workloads of the wave solver, as seeded synthetic instances.

Each builder returns a dict with the mesh description, the degree ``k``, the
nodal coefficient fields ``rho`` and ``c`` ([E, (k+1)^3] at the solution's
Gauss-Lobatto nodes), the initial state ``U0`` ([E, 4, (k+1)^3], fields
p, v_x, v_y, v_z), the flux parameter ``alpha`` (1 upwind, 0 central), the
time step ``dt`` from the Courant number ``Cr = c_max dt k^1.5 / h`` and the
step count.  ``exact`` is the analytic solution x, t -> [..., 4] when known.

Sizes are parameters so that the same recipe yields small instances the CPU
oracle finishes in seconds and the full sizes the GPU runs.
"""
import numpy as np

from .mesh import cube_mesh, solution_node_positions, curving, random_frames
from . import fields


def dt_from_courant(cr, h, c_max, k):
    """Time step from the Courant number Cr = c dt k^1.5 / h."""
    return cr * h / (c_max * k ** 1.5)


def _nodal(mesh, k, fn):
    x = solution_node_positions(mesh, k)
    return x, fn(x)


def _pack_state(vals):
    # vals [E, n^3, 4] -> U [E, 4, n^3]
    return np.ascontiguousarray(np.transpose(vals, (0, 2, 1)))


def standing_wave(N=4, k=3, cr=0.2, nsteps=100, alpha=1.0, frames_seed=None):
    """Plain method: periodic affine cube, rho = c = 1, standing wave."""
    frames = None
    if frames_seed is not None:
        frames = random_frames(N ** 3, np.random.default_rng(frames_seed))
    mesh = cube_mesh(N, q=1, periodic=True, frames=frames)
    x, u0 = _nodal(mesh, k, lambda x: fields.standing_wave(x, 0.0))
    E, n3 = x.shape[0], x.shape[1]
    return {
        "name": f"standing_wave_N{N}_k{k}", "mesh": mesh, "k": k,
        "rho": np.ones((E, n3)), "c": np.ones((E, n3)), "U0": _pack_state(u0),
        "alpha": alpha, "dt": dt_from_courant(cr, mesh["h"], 1.0, k),
        "nsteps": nsteps, "exact": fields.standing_wave, "xnodes": x,
    }


def curved_pulse(N=32, k=5, cr=0.1, nsteps=200, seed=2, a=0.05, alpha=1.0):
    """Plain method at scale: curved cube with walls, variable rho and c,
    Gaussian pressure pulse (width 0.05) at a seeded centre."""
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0.25, 0.75, size=3)
    mesh = cube_mesh(N, q=k, periodic=False, deform=curving(a))
    x = solution_node_positions(mesh, k)
    rho, c = fields.cfg2_coefficients(x)
    u0 = fields.gaussian_pulse(x, x0, 0.05)
    return {
        "name": f"curved_pulse_N{N}_k{k}", "mesh": mesh, "k": k,
        "rho": rho, "c": c, "U0": _pack_state(u0), "alpha": alpha,
        "dt": dt_from_courant(cr, mesh["h"], 1.5, k), "nsteps": nsteps,
        "exact": None, "xnodes": x, "pulse_centre": x0,
    }


def plane_wave(N=64, k=4, cr=0.1, nsteps=1000, alpha=1.0):
    """Precision form: periodic affine cube, rho = c = 1, plane wave along
    (1,1,1) with wave vector 4 pi (1,1,1)."""
    mesh = cube_mesh(N, q=1, periodic=True)
    x, u0 = _nodal(mesh, k, lambda x: fields.plane_wave(x, 0.0))
    E, n3 = x.shape[0], x.shape[1]
    return {
        "name": f"plane_wave_N{N}_k{k}", "mesh": mesh, "k": k,
        "rho": np.ones((E, n3)), "c": np.ones((E, n3)), "U0": _pack_state(u0),
        "alpha": alpha, "dt": dt_from_courant(cr, mesh["h"], 1.0, k),
        "nsteps": nsteps, "exact": fields.plane_wave, "xnodes": x,
    }


def random_instance(seed, N=None, k=None, curved=True, cr=0.1, nsteps=500,
                    n_range=(4, 24), k_choices=(2, 3, 4, 5, 6, 7)):
    """One instance of the batched/served mix: walls, seeded smooth rho and
    c in [0.55, 1.95], mild random curving, seeded Gaussian pulse."""
    rng = np.random.default_rng(seed)
    if N is None:
        N = int(rng.integers(n_range[0], n_range[1] + 1))
    if k is None:
        k = int(rng.choice(k_choices))
    a = float(rng.uniform(0.0, 0.05)) if curved else 0.0
    sigma = float(rng.uniform(0.05, 0.1))
    x0 = rng.uniform(0.25, 0.75, size=3)
    frho = fields.random_smooth_field(rng)
    fc = fields.random_smooth_field(rng)
    mesh = cube_mesh(N, q=(k if curved else 1), periodic=False,
                     deform=(curving(a) if curved and a > 0 else None))
    x = solution_node_positions(mesh, k)
    rho, c = frho(x), fc(x)
    u0 = fields.gaussian_pulse(x, x0, sigma)
    return {
        "name": f"random_{seed}", "mesh": mesh, "k": k, "rho": rho, "c": c,
        "U0": _pack_state(u0), "alpha": 1.0,
        "dt": dt_from_courant(cr, mesh["h"], float(np.max(c)), k),
        "nsteps": nsteps, "exact": None, "xnodes": x,
    }


def random_state(mesh_E, k, seed):
    """Seeded random state [E, 4, (k+1)^3] with entries in [-1, 1]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(mesh_E, 4, (k + 1) ** 3))
