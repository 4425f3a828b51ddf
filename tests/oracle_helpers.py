"""Small helpers shared by the oracle pin tests (no DG arithmetic)."""
import numpy as np

import synth


def linear_map(A, shift=(0.0, 0.0, 0.0)):
    A = np.asarray(A, float)
    b = np.asarray(shift, float)

    def f(x):
        return x @ A.T + b
    return f


SHEAR = np.array([[1.0, 0.2, 0.1], [0.05, 0.9, 0.15], [-0.1, 0.07, 1.1]])

# phases of the generic curving below (one row per displaced coordinate)
CURVE_PHASES = np.array([[0.3, 1.1, 2.0], [0.7, 0.2, 1.4], [1.9, 0.5, 0.9]])


def generic_curving(a):
    """x_i <- x_i + a prod_j sin(2 pi x_j + phi_ij): a periodic curving whose
    three displacements differ, so that the Jacobian has no special
    structure (the bench's curving adds the same scalar to every
    coordinate)."""
    def f(x):
        s = [np.prod([np.sin(2 * np.pi * x[..., j] + CURVE_PHASES[i, j]) for j in range(3)], axis=0)
             for i in range(3)]
        return x + a * np.stack(s, axis=-1)
    return f


def single_element_mesh(A, x0=(0.3, -0.2, 0.5)):
    """One affine element x = x0 + A xi (xi in [-1,1]^3), all faces walls."""
    m = synth.cube_mesh(1, q=1, periodic=False)
    # cube_mesh(1) maps xi to 0.5 + 0.5 xi; rebuild nodes directly
    xi = np.array([[i, j, k] for k in (-1, 1) for j in (-1, 1) for i in (-1, 1)], float)
    m["nodes"] = (np.asarray(x0)[None, :] + xi @ np.asarray(A).T)[None]
    return m


def poly1d_lagrange(nodes, a):
    """Lagrange polynomial l_a on ``nodes`` as a numpy Polynomial, built from
    its roots (a route independent of the oracle's product formula)."""
    others = np.delete(nodes, a)
    p = np.polynomial.Polynomial.fromroots(others)
    return p / p(nodes[a])


def exact_int(p):
    P = p.integ()
    return P(1.0) - P(-1.0)


def generic_curving_2d(a):
    """2D counterpart of generic_curving: x_i <- x_i + a prod_j sin(2 pi x_j + phi_ij)."""
    def f(x):
        s = [np.prod([np.sin(2 * np.pi * x[..., j] + CURVE_PHASES[i, j]) for j in range(2)], axis=0)
             for i in range(2)]
        return x + a * np.stack(s, axis=-1)
    return f
