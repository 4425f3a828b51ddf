"""The 2D path on the GPU (dg_mesh_setup_2d) against the 2D oracle.

Tolerances as in 3D: FP64 operator and predictor <= 1e-13 relative l2, FP64
after a few steps <= 1e-12, FP32 operator <= 2e-6 and after a few steps
<= 2e-5."""
import numpy as np
import pytest

import oracle
import paper_1805_03981_gb300 as dgw
from synth import mesh2d
from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _pair(cfg, prec=dgw.DG_FP64, alpha=1.0):
    s = dgw.Solver2D(cfg["mesh"], cfg["k"], prec, alpha, cfg["rho"], cfg["c"])
    o = oracle.Oracle2D(cfg["mesh"], cfg["k"], cfg["rho"], cfg["c"], alpha)
    return s, o


def _curved(N, k, seed, periodic):
    cfg = mesh2d.curved_config_2d(N=N, k=k, seed=seed, frames_seed=seed + 100, periodic=periodic)
    cfg["U0"] = mesh2d.random_state_2d(N * N, k, seed + 1)
    return cfg


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
def test_operator_2d(k, prec):
    torch = _cuda()
    cfg = _curved(4, k, 3 + k, periodic=(k % 2 == 0))
    s, o = _pair(cfg, prec)
    R = s.apply(s.to_device(cfg["U0"]))
    torch.cuda.synchronize()
    assert rel_l2(R.cpu().numpy(), o.apply(cfg["U0"])) < (1e-13 if prec == dgw.DG_FP64 else 2e-6)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("red", [0, 2])
def test_tck_2d(k, red):
    torch = _cuda()
    cfg = _curved(3, k, 20 + k, periodic=False)
    s, o = _pair(cfg)
    Ub = s.tck(s.to_device(cfg["U0"]), 0.02, red)
    torch.cuda.synchronize()
    assert rel_l2(Ub.cpu().numpy(), o.tck(cfg["U0"], 0.02, red)) < 1e-13


@pytest.mark.parametrize("k", [1, 3, 5, 7])
@pytest.mark.parametrize("method", ["lsrk", "ader"])
def test_steppers_2d(k, method):
    torch = _cuda()
    cfg = _curved(4, k, 40 + k, periodic=(k % 2 == 1))
    dt = 0.003
    s, o = _pair(cfg)
    U = s.to_device(cfg["U0"])
    if method == "lsrk":
        s.step_lsrk(U, dt, 3)
        ref = o.lsrk(cfg["U0"], dt, 3)
    else:
        s.step_ader(U, dt, 3, 2)
        ref = o.ader(cfg["U0"], dt, 3, 2)
    torch.cuda.synchronize()
    assert rel_l2(U.cpu().numpy(), ref) < 1e-12
    s32 = dgw.Solver2D(cfg["mesh"], k, dgw.DG_FP32, 1.0, cfg["rho"], cfg["c"])
    V = s32.to_device(cfg["U0"])
    if method == "lsrk":
        s32.step_lsrk(V, dt, 3)
    else:
        s32.step_ader(V, dt, 3, 2)
    torch.cuda.synchronize()
    assert rel_l2(V.cpu().numpy(), ref) < 2e-5


@pytest.mark.parametrize("method", ["lsrk", "ader"])
def test_standing_wave_100_steps_2d(method):
    torch = _cuda()
    cfg = mesh2d.standing_wave_config_2d(N=6, k=3, cr=0.1, frames_seed=7)
    s, o = _pair(cfg)
    U = s.to_device(cfg["U0"])
    dt = cfg["dt"]
    if method == "lsrk":
        s.step_lsrk(U, dt, 100)
        ref = o.lsrk(cfg["U0"], dt, 100)
    else:
        s.step_ader(U, dt, 100, 2)
        ref = o.ader(cfg["U0"], dt, 100, 2)
    torch.cuda.synchronize()
    assert rel_l2(U.cpu().numpy(), ref) < 1e-12
    assert o.l2_error(U.cpu().numpy(), cfg["exact"], 100 * dt)[0] < 1e-2


def test_energy_and_solve_host_2d():
    torch = _cuda()
    cfg = _curved(3, 4, 60, periodic=False)
    s, o = _pair(cfg)
    U = s.to_device(cfg["U0"])
    e = s.energy(U)
    assert abs(e - o.energy(cfg["U0"])) < 1e-12 * abs(e)
    Uh = torch.from_numpy(np.ascontiguousarray(cfg["U0"]))
    out = torch.empty_like(Uh)
    s.solve_host(1, Uh, out, 0.003, 2, 2)
    assert rel_l2(out.numpy(), o.ader(cfg["U0"], 0.003, 2, 2)) < 1e-12


def test_unsupported_calls_2d():
    _cuda()
    cfg = _curved(2, 2, 70, periodic=True)
    s, _ = _pair(cfg)
    U = s.to_device(cfg["U0"])
    with pytest.raises(dgw.DGError):
        s.set_basis(dgw.BASIS_GL)
    with pytest.raises(dgw.DGError):
        s.step_hdg_ader(U, 0.01, 1)
    with pytest.raises(dgw.DGError):
        s.step_ader(U, 0.01, 1, reduce_every=1)
    with pytest.raises(dgw.DGError):
        dgw.Batch([s], [U], [0.01])
