"""The predictor without the basis change (Sec. 3.2, Alg. 1;
DG_PRED_GL_PROJECTION) against the FP64 oracle.  It equals the collocated
predictor in exact arithmetic (the n-point Gauss rule makes the GL
projection of Gauss-point values their interpolant), so the oracle's
predictor without reduction is its reference.  Its longer chain of
contractions (interpolation, integration, two inverse interpolations per
derivative) rounds more: FP64 <= 1e-12, FP32 <= 2e-5 relative l2."""
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


def _affine(N, k, seed):
    from oracle_helpers import SHEAR, linear_map
    mesh = synth.cube_mesh(N, q=1, periodic=True, deform=linear_map(SHEAR))
    rng = np.random.default_rng(seed)
    n3 = (k + 1) ** 3
    rho = rng.uniform(0.6, 1.6, size=(N ** 3, 1)) * np.ones((1, n3))
    c = rng.uniform(0.6, 1.6, size=(N ** 3, 1)) * np.ones((1, n3))
    return {"mesh": mesh, "k": k, "rho": rho, "c": c, "alpha": 1.0,
            "U0": synth.configs.random_state(N ** 3, k, seed + 1)}


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
def test_alg1_predictor_curved(k):
    torch = _cuda()
    cfg = _curved(2, k, seed=500 + k)
    s, o = pair(cfg)
    s.set_predictor_kernel(dgw.PRED_GL_PROJECTION)
    dt = 0.02
    Ub = s.tck(s.to_device(cfg["U0"]), dt, 0)
    torch.cuda.synchronize()
    ref = o.tck(cfg["U0"], dt, 0)
    assert rel_l2(Ub.cpu().numpy(), ref) < 1e-12
    s32 = dgw.Solver(cfg["mesh"], k, dgw.DG_FP32, 1.0, cfg["rho"], cfg["c"])
    s32.set_predictor_kernel(dgw.PRED_GL_PROJECTION)
    V = s32.tck(s32.to_device(cfg["U0"]), dt, 0)
    torch.cuda.synchronize()
    assert rel_l2(V.cpu().numpy(), ref) < 2e-5


@pytest.mark.parametrize("k", [2, 5])
def test_alg1_predictor_affine(k):
    torch = _cuda()
    cfg = _affine(2, k, seed=520 + k)
    s, o = pair(cfg)
    assert s.is_affine()
    s.set_predictor_kernel(dgw.PRED_GL_PROJECTION)
    Ub = s.tck(s.to_device(cfg["U0"]), 0.02, 0)
    torch.cuda.synchronize()
    assert rel_l2(Ub.cpu().numpy(), o.tck(cfg["U0"], 0.02, 0)) < 1e-12


@pytest.mark.parametrize("k", [3, 6])
def test_alg1_ader_steps(k):
    """ADER steps in the GL basis with the Alg. 1 predictor, blocks of 1 and 2
    elements over 27 elements (a ragged last block)."""
    torch = _cuda()
    cfg = _curved(3, k, seed=540 + k, periodic=True)
    s, o = pair(cfg)
    s.set_basis(dgw.BASIS_GL)
    s.set_predictor_kernel(dgw.PRED_GL_PROJECTION)
    ref = o.ader(cfg["U0"], 0.004, 2, 0)
    for epb in (1, 2):
        s.set_tiling(0, epb)
        U = s.to_device(cfg["U0"])
        s.step_ader(U, 0.004, 2, 0)
        torch.cuda.synchronize()
        assert rel_l2(U.cpu().numpy(), ref) < 1e-12, epb


def test_alg1_unsupported():
    _cuda()
    cfg = _curved(2, 3, seed=560)
    s, _ = pair(cfg)
    s.set_predictor_kernel(dgw.PRED_GL_PROJECTION)
    U = s.to_device(cfg["U0"])
    with pytest.raises(dgw.DGError):
        s.tck(U, 0.01, 2)  # degree reduction is the other forms' business
    s.set_basis(dgw.BASIS_G)
    with pytest.raises(dgw.DGError):
        s.step_ader(U, 0.01, 1, 0)  # Gauss-point states
    s.set_basis(dgw.BASIS_GL)
    with pytest.raises(dgw.DGError):
        s.step_hdg_ader(U, 0.01, 1, 0)
    s.set_predictor_kernel(dgw.PRED_AUTO)
    s.step_ader(U, 0.01, 1, 0)
