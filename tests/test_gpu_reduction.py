"""Degree reduction every 1, 2 or 3 derivatives in the predictor (Sec. 3.3,
Fig. reduc-comp) on the GPU, against the FP64 oracle.

Tolerances as in test_gpu_parity: FP64 predictor <= 1e-13, FP64 after a few
ADER steps <= 1e-12, FP32 predictor <= 5e-6 relative l2.
"""
import numpy as np
import pytest

import synth
import paper_1805_03981_gb300 as dgw
from gpu_helpers import rel_l2, pair

pytestmark = pytest.mark.gpu


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _curved(N, k, seed, periodic=False):
    rng = np.random.default_rng(seed)
    fr = synth.mesh.random_frames(N ** 3, rng)
    mesh = synth.cube_mesh(N, q=k, periodic=periodic, deform=synth.mesh.curving(0.05), frames=fr)
    x = synth.solution_node_positions(mesh, k)
    rho, c = synth.fields.cfg2_coefficients(x)
    return {"mesh": mesh, "k": k, "rho": rho, "c": c, "alpha": 1.0,
            "U0": synth.configs.random_state(N ** 3, k, seed + 1)}


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("red", [1, 3])
def test_tck_odd_reduction_curved(k, red):
    torch = _cuda()
    cfg = _curved(2, k, seed=60 + k)
    s, o = pair(cfg)
    dt = 0.02
    Ub = s.tck(s.to_device(cfg["U0"]), dt, red)
    torch.cuda.synchronize()
    ref = o.tck(cfg["U0"], dt, red)
    assert rel_l2(Ub.cpu().numpy(), ref) < 1e-13
    s32 = dgw.Solver(cfg["mesh"], k, dgw.DG_FP32, 1.0, cfg["rho"], cfg["c"])
    V = s32.tck(s32.to_device(cfg["U0"]), dt, red)
    torch.cuda.synchronize()
    assert rel_l2(V.cpu().numpy(), ref) < 5e-6


@pytest.mark.parametrize("red", [1, 3])
@pytest.mark.parametrize("basis", ["g", "gl"])
def test_ader_odd_reduction_steps(red, basis):
    torch = _cuda()
    for k in (3, 6):
        cfg = _curved(3 if k < 5 else 2, k, seed=70 + k + red, periodic=True)
        s, o = pair(cfg)
        s.set_basis(dgw.BASIS_G if basis == "g" else dgw.BASIS_GL)
        dt = 0.004
        U = s.to_device(cfg["U0"])
        s.step_ader(U, dt, 3, red)
        torch.cuda.synchronize()
        ref = o.ader(cfg["U0"], dt, 3, red)
        assert rel_l2(U.cpu().numpy(), ref) < 1e-12, k


@pytest.mark.parametrize("red", [1, 3])
def test_affine_odd_reduction(red):
    """Affine elements with element-wise constant coefficients: the compact
    predictor data serve every Gauss set, no rebuild needed."""
    torch = _cuda()
    from oracle_helpers import SHEAR, linear_map
    k, N = 5, 2
    mesh = synth.cube_mesh(N, q=1, periodic=True, deform=linear_map(SHEAR))
    rng = np.random.default_rng(80 + red)
    n3 = (k + 1) ** 3
    rho = rng.uniform(0.6, 1.6, size=(N ** 3, 1)) * np.ones((1, n3))
    c = rng.uniform(0.6, 1.6, size=(N ** 3, 1)) * np.ones((1, n3))
    cfg = {"mesh": mesh, "k": k, "rho": rho, "c": c, "alpha": 1.0,
           "U0": synth.configs.random_state(N ** 3, k, 81)}
    s, o = pair(cfg)
    assert s.is_affine()
    before = s.device_bytes()
    Ub = s.tck(s.to_device(cfg["U0"]), 0.02, red)
    torch.cuda.synchronize()
    assert s.device_bytes() == before
    assert rel_l2(Ub.cpu().numpy(), o.tck(cfg["U0"], 0.02, red)) < 1e-13


def test_levels_rebuilt_once_and_results_unchanged():
    """The first reduction by 1 on a curved mesh rebuilds the predictor data
    at every Gauss set; reduction by 2 reads the same values afterwards, so
    its result is bitwise unchanged."""
    torch = _cuda()
    k = 5
    cfg = _curved(2, k, seed=90)
    s, _ = pair(cfg)
    U0 = s.to_device(cfg["U0"])
    before = s.device_bytes()
    A = s.tck(U0, 0.02, 2).clone()
    s.tck(U0, 0.02, 1)
    grown = s.device_bytes()
    E, rs = 8, 8
    extra = 11 * (sum(m ** 3 for m in range(k + 1, 1, -1)) - sum(m ** 3 for m in range(k + 1, 1, -2)))
    assert grown - before == extra * E * rs
    B = s.tck(U0, 0.02, 2)
    s.tck(U0, 0.02, 3)
    torch.cuda.synchronize()
    assert s.device_bytes() == grown
    assert torch.equal(A, B)


def test_reduction_arguments():
    torch = _cuda()
    cfg = _curved(2, 2, seed=95)
    s, _ = pair(cfg)
    U = s.to_device(cfg["U0"])
    for bad in (-1, 4, 5):
        with pytest.raises(dgw.DGError):
            s.step_ader(U, 0.01, 1, reduce_every=bad)
    b = dgw.Batch([s], [U], [0.01])
    with pytest.raises(dgw.DGError):
        b.step_ader(1, reduce_every=1)
    b.step_ader(1, reduce_every=2)
    torch.cuda.synchronize()
    b.close()
