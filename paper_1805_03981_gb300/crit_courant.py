"""Critical Courant numbers of the GPU schemes by simulation (the paper's
Sec. 4.7 "iterative procedure", Table crit-Cr).

On a periodic Cartesian mesh with rho = c = 1 and the upwind flux, a seeded
random state is advanced for ``steps`` steps at Cr = c dt k^1.5 / h; the run
is unstable when the discrete energy grows by more than ``growth`` (default
1% over 1000 steps).  Bisection on Cr brackets the limit.

    python -m paper_1805_03981_gb300.crit_courant --k 1,4,7
"""
import argparse
import json

import numpy as np


def _setup(k, N, prec, dim=3):
    import synth
    from . import _lib
    if dim == 2:
        from synth import mesh2d
        mesh = mesh2d.square_mesh(N, q=1, periodic=True)
        ones = np.ones((N * N, (k + 1) ** 2))
        return _lib.Solver2D(mesh, k, prec, 1.0, ones, ones), mesh2d.random_state_2d(N * N, k, 1234), 1.0 / N
    mesh = synth.cube_mesh(N, q=1, periodic=True)
    n3 = (k + 1) ** 3
    ones = np.ones((N ** 3, n3))
    s = _lib.Solver(mesh, k, prec, 1.0, ones, ones)
    U0 = synth.configs.random_state(N ** 3, k, 1234)
    return s, U0, 1.0 / N


def stable(s, U0, h, k, cr, method, steps, growth):
    import torch
    U = s.to_device(U0)
    e0 = s.energy(U)
    dt = cr * h / k ** 1.5
    if method in ("lsrk", "lsrk45", "lsrk59"):
        s.step_lsrk(U, dt, steps)
    elif method == "hdg_ader":
        s.step_hdg_ader(U, dt, steps, 2)
    else:
        s.step_ader(U, dt, steps, 2)
    torch.cuda.synchronize()
    e1 = s.energy(U)
    return bool(np.isfinite(e1) and e1 <= e0 * (1.0 + growth))


def critical(k, method, N=4, steps=1000, growth=0.01, lo=0.02, hi=1.2, tol=2e-3, prec=None, dim=3):
    from . import _lib
    s, U0, h = _setup(k, N, _lib.DG_FP64 if prec is None else prec, dim)
    # lsrk: the 2N five-stage scheme; lsrk45 / lsrk59: the paper's
    # two-register LSRK4(5) / LSRK5(9) (Sec. 2.2)
    s_scheme = {"lsrk45": _lib.LSRK45, "lsrk59": _lib.LSRK59}.get(method)
    if s_scheme is not None:
        s.set_lsrk_scheme(s_scheme)
    if method in ("ader", "hdg_ader"):
        hi = min(hi, 0.6)
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if stable(s, U0, h, k, mid, method, steps, growth):
            lo = mid
        else:
            hi = mid
    s.close()
    return 0.5 * (lo + hi)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--k", default="1,4,7")
    ap.add_argument("--N", type=int, default=4)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--dim", type=int, default=3, choices=[2, 3])
    a = ap.parse_args()
    out = {}
    methods = ("lsrk", "lsrk45", "lsrk59", "ader", "hdg_ader") if a.dim == 3 else ("lsrk", "ader")
    for k in (int(x) for x in a.k.split(",")):
        out[k] = {m: critical(k, m, a.N, a.steps, dim=a.dim) for m in methods}
    print(json.dumps({"crit_courant_%dd" % a.dim: out,
                      "mesh": f"{a.N}^{a.dim} periodic Cartesian, rho=c=1, upwind",
                      "criterion": f"energy growth <= 1 percent over {a.steps} steps from a seeded random state"}))


if __name__ == "__main__":
    main()
