"""The column-form predictor kernel (tckc.cuh, DG_PRED_COLUMNS) inside ADER
steps with Gauss-point states, against the FP64 oracle and against the
line-form kernel it replaces by default.

Tolerances: FP64 ADER steps <= 1e-12 relative l2 against the oracle (as in
test_gpu_parity); the two FP64 kernels differ only in rounding order,
<= 1e-13; FP32 <= 2e-5 against the oracle after the steps.
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


def _affine(N, k, seed):
    """Sheared affine elements with element-wise constant coefficients: the
    compact predictor data."""
    from oracle_helpers import SHEAR, linear_map
    mesh = synth.cube_mesh(N, q=1, periodic=True, deform=linear_map(SHEAR),
                           frames=synth.mesh.random_frames(N ** 3, np.random.default_rng(seed)))
    rng = np.random.default_rng(seed + 1)
    n3 = (k + 1) ** 3
    rho = rng.uniform(0.6, 1.6, size=(N ** 3, 1)) * np.ones((1, n3))
    c = rng.uniform(0.6, 1.6, size=(N ** 3, 1)) * np.ones((1, n3))
    return {"mesh": mesh, "k": k, "rho": rho, "c": c, "alpha": 1.0,
            "U0": synth.configs.random_state(N ** 3, k, seed + 2)}


def _ader(s, U0, kind, dt, nsteps, red, hdg=False, tiling=0):
    s.set_basis(dgw.BASIS_G)
    s.set_predictor_kernel(kind)
    if tiling:
        s.set_tiling(0, tiling)
    U = s.to_device(U0)
    (s.step_hdg_ader if hdg else s.step_ader)(U, dt, nsteps, red)
    return U


@pytest.mark.parametrize("k", [1, 4, 7])
@pytest.mark.parametrize("red", [0, 1, 2, 3])
def test_columns_curved_vs_oracle(k, red):
    torch = _cuda()
    cfg = _curved(2, k, seed=100 + 10 * k + red)
    s, o = pair(cfg)
    dt = 0.004
    U = _ader(s, cfg["U0"], dgw.PRED_COLUMNS, dt, 2, red)
    torch.cuda.synchronize()
    ref = o.ader(cfg["U0"], dt, 2, red)
    assert rel_l2(U.cpu().numpy(), ref) < 1e-12
    s32 = dgw.Solver(cfg["mesh"], k, dgw.DG_FP32, 1.0, cfg["rho"], cfg["c"])
    V = _ader(s32, cfg["U0"], dgw.PRED_COLUMNS, dt, 2, red)
    torch.cuda.synchronize()
    assert rel_l2(V.cpu().numpy(), ref) < 2e-5


@pytest.mark.parametrize("k", [2, 5])
@pytest.mark.parametrize("red", [0, 1, 2, 3])
def test_columns_affine_vs_oracle(k, red):
    torch = _cuda()
    cfg = _affine(2, k, seed=200 + 10 * k + red)
    s, o = pair(cfg)
    assert s.is_affine()
    dt = 0.004
    U = _ader(s, cfg["U0"], dgw.PRED_COLUMNS, dt, 2, red)
    torch.cuda.synchronize()
    ref = o.ader(cfg["U0"], dt, 2, red)
    assert rel_l2(U.cpu().numpy(), ref) < 1e-12
    s32 = dgw.Solver(cfg["mesh"], k, dgw.DG_FP32, 1.0, cfg["rho"], cfg["c"])
    V = _ader(s32, cfg["U0"], dgw.PRED_COLUMNS, dt, 2, red)
    torch.cuda.synchronize()
    assert rel_l2(V.cpu().numpy(), ref) < 2e-5


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("geometry", ["curved", "affine"])
def test_columns_equal_lines(k, geometry):
    """Every degree and reduction, blocks of 1, 2 and 3 elements over a
    27-element mesh (a ragged last block): the column and line kernels agree
    to rounding."""
    torch = _cuda()
    cfg = _curved(3, k, seed=300 + k, periodic=True) if geometry == "curved" else _affine(3, k, seed=300 + k)
    dt = 0.003
    for red in (0, 1, 2, 3):
        s, _ = pair(cfg)
        A = _ader(s, cfg["U0"], dgw.PRED_LINES, dt, 2, red)
        for epb in (1, 2, 3):
            B = _ader(s, cfg["U0"], dgw.PRED_COLUMNS, dt, 2, red, tiling=epb)
            torch.cuda.synchronize()
            assert rel_l2(B.cpu().numpy(), A.cpu().numpy()) < 1e-13, (red, epb)
        s.close()


@pytest.mark.parametrize("k", [3, 5])
@pytest.mark.parametrize("red", [1, 2, 3])
def test_columns_hdg_ader_vs_oracle(k, red):
    torch = _cuda()
    cfg = _curved(2, k, seed=400 + k)
    s, o = pair(cfg)
    dt = 0.003
    U = _ader(s, cfg["U0"], dgw.PRED_COLUMNS, dt, 2, red, hdg=True)
    torch.cuda.synchronize()
    assert rel_l2(U.cpu().numpy(), o.hdg_ader(cfg["U0"], dt, 2, red)) < 1e-12


def test_predictor_kernel_argument():
    _cuda()
    cfg = _curved(2, 2, seed=450)
    s, _ = pair(cfg)
    assert s.predictor_kernel() == dgw.PRED_AUTO
    for kind in (dgw.PRED_LINES, dgw.PRED_COLUMNS, dgw.PRED_INTERLEAVED, dgw.PRED_AUTO):
        s.set_predictor_kernel(kind)
        assert s.predictor_kernel() == kind
    for bad in (-1, 5):
        with pytest.raises(dgw.DGError):
            s.set_predictor_kernel(bad)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("red", [0, 2])
@pytest.mark.parametrize("N", [2, 3])
def test_interleaved_matches_columns(k, red, N):
    """FP32 affine elements with constant coefficients: the interleaved
    column form (tcki.cuh, DG_PRED_INTERLEAVED, the FP32 default there),
    which forms each reduced Taylor term directly on the smaller Gauss set,
    agrees with the column form to FP32 rounding, on full blocks and on a
    ragged last block (N^3 = 8 or 27 elements, 8 or 4 per block), and is at
    oracle parity."""
    torch = _cuda()
    cfg = _affine(N, k, seed=300 + 10 * k + red + N)
    s = dgw.Solver(cfg["mesh"], k, dgw.DG_FP32, 1.0, cfg["rho"], cfg["c"])
    assert s.is_affine()
    dt = 0.004
    Ui = _ader(s, cfg["U0"], dgw.PRED_INTERLEAVED, dt, 2, red)
    Ua = _ader(s, cfg["U0"], dgw.PRED_AUTO, dt, 2, red)
    Uc = _ader(s, cfg["U0"], dgw.PRED_COLUMNS, dt, 2, red)
    torch.cuda.synchronize()
    s.check_device()
    assert torch.equal(Ua, Ui)                 # the default is the interleaved form
    assert rel_l2(Ui.cpu().numpy(), Uc.cpu().numpy()) < 2e-6
    import oracle
    o = oracle.Oracle(cfg["mesh"], k, cfg["rho"], cfg["c"], 1.0)
    assert rel_l2(Ui.cpu().numpy(), o.ader(cfg["U0"], dt, 2, red)) < 2e-5
    s.close()
