"""The precision form's accuracy bar: FP32 operator and state, FP32
accumulation, FP64 geometry set-up, relative l2 error <= 1e-5 after 1000
steps of each method.

Recipe: the plane wave along (1, 1, 1) with wave vector 4 pi (1, 1, 1) on the
periodic unit cube, k = 4, rho = c = 1, upwind flux, Cr = 0.1; the GPU runs
with the bench's configuration (Gauss-point state inside the steppers, the
default predictor form: the column form in FP32).  Two references:

* the FP64 CPU oracle on the 4^3 mesh (1000 LSRK and 1000 ADER steps, run in
  two spawned processes side by side);
* the FP64 GPU path, itself at 1e-12 oracle parity, on the 16^3 mesh.

Both FP32 errors are also reported against the analytic solution, beside
the FP64 path's, to show that rounding stays below the discretisation error.
"""
import multiprocessing as mp

import numpy as np
import pytest

import synth
import paper_1805_03981_gb300 as dgw
from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

STEPS = 1000
TOL = 1e-5


def _oracle_run(method):
    import oracle
    cfg = synth.configs.plane_wave(N=4, k=4, nsteps=STEPS)
    o = oracle.Oracle(cfg["mesh"], cfg["k"], cfg["rho"], cfg["c"], cfg["alpha"])
    if method == "lsrk":
        return o.lsrk(cfg["U0"], cfg["dt"], STEPS)
    return o.ader(cfg["U0"], cfg["dt"], STEPS, 2)


@pytest.fixture(scope="module")
def oracle_refs():
    with mp.get_context("spawn").Pool(2) as pool:
        out = pool.map(_oracle_run, ["lsrk", "ader"])
    return dict(zip(["lsrk", "ader"], out))


def _gpu_run(cfg, prec, method):
    import torch
    s = dgw.Solver(cfg["mesh"], cfg["k"], prec, cfg["alpha"], cfg["rho"], cfg["c"])
    s.set_basis(dgw.BASIS_G)
    U = s.to_device(cfg["U0"])
    if method == "lsrk":
        s.step_lsrk(U, cfg["dt"], STEPS)
    else:
        s.step_ader(U, cfg["dt"], STEPS, 2)
    torch.cuda.synchronize()
    s.check_device()
    out = U.double().cpu().numpy()
    s.close()
    return out


def _nodal_error(cfg, U, t):
    ex = cfg["exact"](cfg["xnodes"], t)
    return rel_l2(U, np.transpose(ex, (0, 2, 1)))


@pytest.mark.parametrize("method", ["lsrk", "ader"])
def test_fp32_1000_steps_against_fp64_oracle(oracle_refs, method):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = synth.configs.plane_wave(N=4, k=4, nsteps=STEPS)
    U32 = _gpu_run(cfg, dgw.DG_FP32, method)
    err = rel_l2(U32, oracle_refs[method])
    print(f"\n{method} FP32 vs FP64 oracle, 4^3 k=4, {STEPS} steps: {err:.3e}")
    assert err <= TOL, err


@pytest.mark.parametrize("method", ["lsrk", "ader"])
def test_fp32_1000_steps_against_fp64_gpu_16cubed(method):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = synth.configs.plane_wave(N=16, k=4, nsteps=STEPS)
    U32 = _gpu_run(cfg, dgw.DG_FP32, method)
    U64 = _gpu_run(cfg, dgw.DG_FP64, method)
    err = rel_l2(U32, U64)
    t = STEPS * cfg["dt"]
    e32, e64 = _nodal_error(cfg, U32, t), _nodal_error(cfg, U64, t)
    print(f"\n{method} 16^3 k=4, {STEPS} steps: FP32 vs FP64 {err:.3e}; "
          f"vs exact (nodal): FP32 {e32:.3e}, FP64 {e64:.3e}")
    assert err <= TOL, err
    assert e32 <= e64 + 2 * TOL
