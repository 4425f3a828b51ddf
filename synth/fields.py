"""Analytic fields: initial states, coefficient fields and exact solutions.

All functions take physical positions x[..., 3] and return numpy arrays.
Field order everywhere is (p, v_x, v_y, v_z).
"""
import numpy as np

TWO_PI = 2.0 * np.pi


def standing_wave(x, t):
    """Standing wave on the periodic unit cube for rho = c = 1.

    p = cos(2 pi x) cos(2 pi y) cos(2 pi z) cos(w t), w = 2 pi sqrt(3);
    v_x = (2 pi / w) sin(2 pi x) cos(2 pi y) cos(2 pi z) sin(w t), cyclically.
    """
    w = TWO_PI * np.sqrt(3.0)
    cx, cy, cz = (np.cos(TWO_PI * x[..., i]) for i in range(3))
    sx, sy, sz = (np.sin(TWO_PI * x[..., i]) for i in range(3))
    amp = TWO_PI / w * np.sin(w * t)
    return np.stack([cx * cy * cz * np.cos(w * t), amp * sx * cy * cz,
                     amp * cx * sy * cz, amp * cx * cy * sz], axis=-1)


def plane_wave(x, t, kvec=(4 * np.pi, 4 * np.pi, 4 * np.pi), rho=1.0, c=1.0):
    """Plane wave p = cos(k.x - w t), v = p/(rho c) k/|k|, w = c |k|.

    The default wave vector 4 pi (1, 1, 1) is periodic on the unit cube.
    """
    k = np.asarray(kvec, float)
    kn = np.linalg.norm(k)
    p = np.cos(x @ k - c * kn * t)
    v = (p / (rho * c))[..., None] * (k / kn)
    return np.concatenate([p[..., None], v], axis=-1)


def gaussian_pulse(x, x0, sigma):
    """p = exp(-|x - x0|^2 / (2 sigma^2)), v = 0."""
    r2 = np.sum((x - np.asarray(x0)) ** 2, axis=-1)
    p = np.exp(-r2 / (2.0 * sigma ** 2))
    z = np.zeros_like(p)
    return np.stack([p, z, z, z], axis=-1)


def cfg2_coefficients(x):
    """c = 1 + 0.5 sin(2 pi x) cos(2 pi y), rho = 1 + 0.3 cos(2 pi z)."""
    c = 1.0 + 0.5 * np.sin(TWO_PI * x[..., 0]) * np.cos(TWO_PI * x[..., 1])
    rho = 1.0 + 0.3 * np.cos(TWO_PI * x[..., 2])
    return rho, c


def random_smooth_field(rng, n_modes=4, mean=1.25, total_amp=0.7):
    """A seeded sum of sinusoids, mean + sum_m a_m sin(2 pi kappa_m . x + phi_m),
    kappa_m in {-2..2}^3 \\ {0}, sum |a_m| = total_amp."""
    kap = []
    while len(kap) < n_modes:
        k = rng.integers(-2, 3, size=3)
        if np.any(k != 0):
            kap.append(k)
    kap = np.array(kap, float)
    a = rng.uniform(0.2, 1.0, size=n_modes) * rng.choice([-1.0, 1.0], size=n_modes)
    a *= total_amp / np.sum(np.abs(a))
    phi = rng.uniform(0, TWO_PI, size=n_modes)

    def f(x):
        out = np.full(x.shape[:-1], mean)
        for m in range(n_modes):
            out = out + a[m] * np.sin(TWO_PI * (x @ kap[m]) + phi[m])
        return out
    return f
