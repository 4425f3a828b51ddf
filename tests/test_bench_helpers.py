"""Host-side measurement helpers of bench.py, checked against the oracle."""
import numpy as np

import synth
import oracle
import bench


def test_l2_pressure_error_matches_oracle():
    """The bench's continuous L2 pressure error (tensor interpolation to
    k+3 Gauss points) equals the oracle's over-integrated L2 error."""
    for k, N in ((1, 3), (3, 2), (4, 2)):
        cfg = synth.configs.standing_wave(N=N, k=k, frames_seed=5)
        rng = np.random.default_rng(k)
        U = cfg["U0"] + 1e-3 * rng.normal(size=cfg["U0"].shape)
        E, n3 = cfg["U0"].shape[0], (k + 1) ** 3
        o = oracle.Oracle(cfg["mesh"], k, np.ones((E, n3)), np.ones((E, n3)))
        t = 0.13
        want = o.l2_error(U, cfg["exact"], t)[0]
        got = bench._l2_pressure_error(U, cfg["xnodes"], cfg["exact"], t, k)
        assert abs(got - want) <= 1e-10 * want, (k, got, want)


def test_l2_pressure_error_2d_matches_oracle():
    from synth import mesh2d
    for k, N in ((1, 3), (3, 2), (4, 3)):
        cfg = mesh2d.standing_wave_config_2d(N=N, k=k, frames_seed=4, exact=mesh2d.membrane_modes_2d)
        rng = np.random.default_rng(k)
        U = cfg["U0"] + 1e-3 * rng.normal(size=cfg["U0"].shape)
        o = oracle.Oracle2D(cfg["mesh"], k, cfg["rho"], cfg["c"])
        want = o.l2_error(U, cfg["exact"], 0.07)[0]
        got = bench._l2_pressure_error_2d(U, cfg["xnodes"], cfg["exact"], 0.07, k)
        assert abs(got - want) <= 1e-10 * want, (k, got, want)
