"""Checkpoint and restart on the GPU (dg_get_state / dg_set_state and
paper_1805_03981_gb300.checkpoint): the copies are exact, and a solve
restarted from a file in a fresh context gives, bit for bit, what the same
step calls give without the checkpoint."""
import numpy as np
import pytest

import synth
import paper_1805_03981_gb300 as dgw
from paper_1805_03981_gb300 import checkpoint as ck
from synth import mesh2d

pytestmark = pytest.mark.gpu


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _curved(N, k, seed):
    rng = np.random.default_rng(seed)
    fr = synth.mesh.random_frames(N ** 3, rng)
    mesh = synth.cube_mesh(N, q=k, periodic=False, deform=synth.mesh.curving(0.05), frames=fr)
    x = synth.solution_node_positions(mesh, k)
    rho, c = synth.fields.cfg2_coefficients(x)
    return mesh, rho, c, synth.configs.random_state(N ** 3, k, seed + 1)


@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
def test_state_copies_exact(prec):
    torch = _cuda()
    mesh, rho, c, U0 = _curved(3, 3, 5)
    s = dgw.Solver(mesh, 3, prec, 1.0, rho, c)
    U = s.to_device(U0)
    h = s.get_state(U)
    assert h.dtype == np.float64 and h.shape == (27, 4, 64)
    assert np.array_equal(h, U.cpu().double().numpy())
    W = s.set_state(U0)
    torch.cuda.synchronize()
    assert torch.equal(W.cpu(), torch.from_numpy(np.ascontiguousarray(U0)).to(s.dtype))  # round to nearest
    V = s.set_state(h, s.empty_state())
    assert torch.equal(V, U)


def _steps(s, U, method, dt, m):
    if method == "lsrk":
        s.step_lsrk(U, dt, m)
    elif method == "ader":
        s.step_ader(U, dt, m, 2)
    else:
        s.step_hdg_ader(U, dt, m, 2)


@pytest.mark.parametrize("method", ["lsrk", "ader", "hdg_ader"])
@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
@pytest.mark.parametrize("basis", [dgw.BASIS_GL, dgw.BASIS_G])
def test_restart_bitwise(tmp_path, method, prec, basis):
    torch = _cuda()
    k, dt, m = 4, 0.004, 3
    mesh, rho, c, U0 = _curved(3, k, 11)
    a = dgw.Solver(mesh, k, prec, 1.0, rho, c)
    a.set_basis(basis)
    ref = a.to_device(U0)
    _steps(a, ref, method, dt, m)
    _steps(a, ref, method, dt, m)
    one = a.to_device(U0)
    _steps(a, one, method, dt, 2 * m)
    U = a.to_device(U0)
    _steps(a, U, method, dt, m)
    path = str(tmp_path / "solve.ckpt")
    ck.save(path, a, U, t=m * dt, step=m, extra={"method": method, "dt": dt})
    a.close()
    b = dgw.Solver(mesh, k, prec, 1.0, rho, c)
    b.set_basis(basis)
    V, t, step, meta = ck.restore(path, b)
    assert step == m and t == m * dt and meta["extra"]["method"] == method
    _steps(b, V, method, dt, m)
    torch.cuda.synchronize()
    assert torch.equal(V, ref)
    if basis == dgw.BASIS_GL:
        assert torch.equal(V, one)
    else:
        d = (V.double() - one.double()).norm() / one.double().norm()
        assert d < (1e-13 if prec == dgw.DG_FP64 else 1e-6)


def test_restore_rejects_other_problem(tmp_path):
    _cuda()
    mesh, rho, c, U0 = _curved(2, 2, 21)
    a = dgw.Solver(mesh, 2, dgw.DG_FP64, 1.0, rho, c)
    path = str(tmp_path / "x.ckpt")
    ck.save(path, a, a.to_device(U0), t=0.0, step=0)
    b = dgw.Solver(mesh, 2, dgw.DG_FP64, 1.0, rho, c * 1.01)
    with pytest.raises(ValueError):
        ck.restore(path, b)
    central = dgw.Solver(mesh, 2, dgw.DG_FP64, 0.0, rho, c)
    with pytest.raises(ValueError):
        ck.restore(path, central)


@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
def test_restart_2d(tmp_path, prec):
    torch = _cuda()
    cfg = mesh2d.curved_config_2d(N=4, k=3, seed=8, frames_seed=108, periodic=False)
    U0 = mesh2d.random_state_2d(16, 3, 9)
    mk = lambda: dgw.Solver2D(cfg["mesh"], 3, prec, 1.0, cfg["rho"], cfg["c"])
    a = mk()
    ref = a.to_device(U0)
    a.step_ader(ref, 0.003, 2, 2)
    a.step_ader(ref, 0.003, 2, 2)
    U = a.to_device(U0)
    a.step_ader(U, 0.003, 2, 2)
    assert np.array_equal(a.get_state(U), U.cpu().double().numpy())
    path = str(tmp_path / "s2.ckpt")
    ck.save(path, a, U, t=0.006, step=2)
    b = mk()
    V, *_ = ck.restore(path, b)
    b.step_ader(V, 0.003, 2, 2)
    torch.cuda.synchronize()
    assert torch.equal(V, ref)
