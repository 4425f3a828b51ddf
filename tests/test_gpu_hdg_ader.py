"""HDG-ADER (Eq. hdg-ader) on the GPU against the oracle, alone and on
parts.  Tolerances as for ADER: FP64 <= 1e-12, FP32 <= 2e-5 relative l2
after three steps."""
import numpy as np
import pytest

import synth
import paper_1805_03981_gb300 as dgw
from paper_1805_03981_gb300 import partition
from gpu_helpers import rel_l2, pair

pytestmark = pytest.mark.gpu


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _curved(N, k, seed, periodic):
    rng = np.random.default_rng(seed)
    fr = synth.mesh.random_frames(N ** 3, rng)
    mesh = synth.cube_mesh(N, q=k, periodic=periodic, deform=synth.mesh.curving(0.05), frames=fr)
    x = synth.solution_node_positions(mesh, k)
    rho, c = synth.fields.cfg2_coefficients(x)
    return {"mesh": mesh, "k": k, "rho": rho, "c": c, "alpha": 1.0,
            "U0": synth.configs.random_state(N ** 3, k, seed + 1)}


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("basis", [dgw.BASIS_GL, dgw.BASIS_G])
def test_hdg_ader_matches_oracle(k, basis):
    torch = _cuda()
    cfg = _curved(2 if k >= 5 else 3, k, 50 + k, periodic=(k % 2 == 0))
    s, o = pair(cfg)
    s.set_basis(basis)
    dt = 0.003
    U = s.to_device(cfg["U0"])
    s.step_hdg_ader(U, dt, 3, 2)
    torch.cuda.synchronize()
    ref = o.hdg_ader(cfg["U0"], dt, 3, 2)
    assert rel_l2(U.cpu().numpy(), ref) < 1e-12
    s32 = dgw.Solver(cfg["mesh"], k, dgw.DG_FP32, 1.0, cfg["rho"], cfg["c"])
    s32.set_basis(basis)
    V = s32.to_device(cfg["U0"])
    s32.step_hdg_ader(V, dt, 3, 2)
    torch.cuda.synchronize()
    assert rel_l2(V.cpu().numpy(), ref) < 2e-5


def test_hdg_ader_reduction_variants():
    torch = _cuda()
    cfg = _curved(2, 4, 70, periodic=True)
    s, o = pair(cfg)
    for red in (0, 1, 3):
        U = s.to_device(cfg["U0"])
        s.step_hdg_ader(U, 0.004, 2, red)
        torch.cuda.synchronize()
        assert rel_l2(U.cpu().numpy(), o.hdg_ader(cfg["U0"], 0.004, 2, red)) < 1e-12, red


@pytest.mark.parametrize("basis", [dgw.BASIS_GL, dgw.BASIS_G])
def test_hdg_ader_parts_bitwise_equal_whole(basis):
    torch = _cuda()
    cfg = _curved(3, 3, 80, periodic=False)
    whole = dgw.Solver(cfg["mesh"], 3, dgw.DG_FP64, 1.0, cfg["rho"], cfg["c"])
    whole.set_basis(basis)
    U = whole.to_device(cfg["U0"])
    whole.step_hdg_ader(U, 0.003, 3, 2)
    pt = partition.Partitioned(cfg["mesh"], 3, 3, dgw.DG_FP64, 1.0, cfg["rho"], cfg["c"], basis)
    states = pt.to_device(cfg["U0"])
    pt.step_hdg_ader(0.003, 3, 2)
    torch.cuda.synchronize()
    assert np.array_equal(pt.gather(states), U.double().cpu().numpy())
    assert pt.info()["exchanges"] == 2 * 3
    pt.close()
