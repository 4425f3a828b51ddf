"""Parity of the two-register LSRK schemes on the GPU (Sec. 2.2: the
paper's LSRK4(5) and LSRK5(9)) with the oracle's two-register loop.

Each stage runs the operator with the two-register epilogue fused in; the
tests cover both storage bases (GL, and Gauss-point states inside the
stepper), both precisions, curved meshes with variable coefficients and
rotated element frames (general kernels) and the affine compact kernels,
k = 1..7.  Tolerances as for the 2N scheme: FP64 <= 1e-12 after the steps,
FP32 <= 2e-5 after a few steps.  The GPU's critical Courant number of
LSRK5(9) at k = 1 matches the oracle's Bloch analysis and the paper's Table
crit-Cr.  Batches, parts and 2D contexts refuse the two-register schemes.
"""
import numpy as np
import pytest

import synth
import paper_1805_03981_gb300 as dgw
from gpu_helpers import rel_l2, pair
from oracle import LSRK45_KCL_A, LSRK45_KCL_B, LSRK59_KCL_A, LSRK59_KCL_B

pytestmark = pytest.mark.gpu

TABLES = {dgw.LSRK45: (LSRK45_KCL_A, LSRK45_KCL_B), dgw.LSRK59: (LSRK59_KCL_A, LSRK59_KCL_B)}
DG_EUNSUPPORTED = -4


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
    U0 = synth.configs.random_state(N ** 3, k, seed + 1)
    return {"mesh": mesh, "k": k, "rho": rho, "c": c, "alpha": 1.0, "U0": U0,
            "dt": synth.configs.dt_from_courant(0.1, 1.0 / N, 1.5, k)}


def _run(cfg, prec, basis, scheme, nsteps):
    torch = _cuda()
    s, o = pair(cfg, prec)
    s.set_basis(basis)
    s.set_lsrk_scheme(scheme)
    assert s.lsrk_scheme() == scheme
    U = s.to_device(cfg["U0"])
    s.step_lsrk(U, cfg["dt"], nsteps)
    torch.cuda.synchronize()
    s.check_device()
    got = U.double().cpu().numpy()
    s.close()
    ref = o.lsrk2r(cfg["U0"], cfg["dt"], nsteps, *TABLES[scheme])
    return rel_l2(got, ref)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("scheme", [dgw.LSRK45, dgw.LSRK59])
def test_curved_variable_fp64_gauss_basis(k, scheme):
    cfg = _curved(3 if k <= 3 else 2, k, seed=30 + k)
    assert _run(cfg, dgw.DG_FP64, dgw.BASIS_G, scheme, 2) < 1e-12


@pytest.mark.parametrize("basis", [dgw.BASIS_GL, dgw.BASIS_G])
@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
@pytest.mark.parametrize("scheme", [dgw.LSRK45, dgw.LSRK59])
def test_curved_both_bases_both_precisions(basis, prec, scheme):
    cfg = _curved(3, 3, seed=41)
    err = _run(cfg, prec, basis, scheme, 3)
    assert err < (1e-12 if prec == dgw.DG_FP64 else 2e-5), err


@pytest.mark.parametrize("basis", [dgw.BASIS_GL, dgw.BASIS_G])
@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
def test_affine_compact_kernels(basis, prec):
    cfg = synth.configs.standing_wave(N=3, k=4, cr=0.1)
    cfg["U0"] = synth.configs.random_state(27, 4, 5)
    err = _run(cfg, prec, basis, dgw.LSRK59, 3)
    assert err < (1e-12 if prec == dgw.DG_FP64 else 2e-5), err


def test_standing_wave_100_steps_lsrk59_fp64():
    cfg = synth.configs.standing_wave(N=4, k=3, cr=0.1, nsteps=100)
    assert _run(cfg, dgw.DG_FP64, dgw.BASIS_G, dgw.LSRK59, 100) < 1e-12


def test_other_paths_refuse_two_register_schemes():
    torch = _cuda()
    from synth import mesh2d
    m2 = mesh2d.square_mesh(2, q=1, periodic=True)
    ones2 = np.ones((4, 16))
    s2 = dgw.Solver2D(m2, 3, dgw.DG_FP64, 1.0, ones2, ones2)
    with pytest.raises(dgw.DGError) as ei:
        s2.set_lsrk_scheme(dgw.LSRK59)
    assert ei.value.status == DG_EUNSUPPORTED
    s2.close()
    cfg = synth.configs.standing_wave(N=2, k=2)
    s = dgw.Solver(cfg["mesh"], 2, dgw.DG_FP32, 1.0, cfg["rho"], cfg["c"])
    s.set_lsrk_scheme(dgw.LSRK59)
    U = s.to_device(cfg["U0"])
    b = dgw.Batch([s], [U], [cfg["dt"]])
    with pytest.raises(dgw.DGError) as ei:
        b.step_lsrk(1)
    assert ei.value.status == DG_EUNSUPPORTED
    b.close()
    with pytest.raises(dgw.DGError):
        s.set_lsrk_scheme(7)
    s.close()


def test_crit_courant_lsrk59_k1_matches_oracle_and_paper():
    _cuda()
    import crit_courant as cc
    from test_oracle_lsrk2r import stability_poly_2r
    from test_oracle_crit_courant import golden
    from paper_1805_03981_gb300 import crit_courant
    b = cc.Bloch(1)
    g = stability_poly_2r(LSRK59_KCL_A, LSRK59_KCL_B)
    o_cr = cc.bisect(lambda c: b.lsrk_stable(c, g), lo=0.05, hi=1.5, tol=2e-3)
    gpu = crit_courant.critical(1, "lsrk59", N=4, steps=1000)
    assert abs(gpu - o_cr) < 0.012, (gpu, o_cr)
    paper = golden()[1][1]
    assert abs(gpu - paper) <= 0.05 * paper, (gpu, paper)
