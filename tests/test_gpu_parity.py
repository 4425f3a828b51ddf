"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 operator and predictor <= 1e-13 relative l2; FP64 after 100
LSRK or ADER steps <= 1e-12 (the target for the FP64 path); FP32 operator
<= 2e-6 and FP32 after 100 steps <= 1e-5 (single-precision rounding of a
sum-factorised evaluation, about 1e-7 per operation, grown over the steps).
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


def _curved(N, k, seed=0, frames=True, periodic=False):
    rng = np.random.default_rng(seed)
    fr = synth.mesh.random_frames(N ** 3, rng) if frames else None
    mesh = synth.cube_mesh(N, q=k, periodic=periodic, deform=synth.mesh.curving(0.05), frames=fr)
    x = synth.solution_node_positions(mesh, k)
    rho, c = synth.fields.cfg2_coefficients(x)
    U0 = synth.configs.random_state(N ** 3, k, seed + 1)
    return {"mesh": mesh, "k": k, "rho": rho, "c": c, "alpha": 1.0, "U0": U0}


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
def test_operator_curved_variable(k, prec):
    torch = _cuda()
    N = 3 if k <= 4 else 2
    cfg = _curved(N, k, seed=k, periodic=(k % 2 == 0))
    s, o = pair(cfg, prec)
    R = s.apply(s.to_device(cfg["U0"]))
    torch.cuda.synchronize()
    ref = o.apply(cfg["U0"])
    err = rel_l2(R.cpu().numpy(), ref)
    assert err < (1e-13 if prec == dgw.DG_FP64 else 2e-6), err


@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_operator_affine_periodic(alpha):
    torch = _cuda()
    cfg = synth.configs.standing_wave(N=4, k=3)
    cfg["U0"] = synth.configs.random_state(64, 3, 9)
    s, o = pair(cfg, dgw.DG_FP64, alpha)
    R = s.apply(s.to_device(cfg["U0"]))
    torch.cuda.synchronize()
    assert rel_l2(R.cpu().numpy(), o.apply(cfg["U0"])) < 1e-13


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("red", [0, 2])
def test_tck_curved_variable(k, red):
    torch = _cuda()
    cfg = _curved(2, k, seed=10 + k)
    s, o = pair(cfg)
    dt = 0.02
    Ub = s.tck(s.to_device(cfg["U0"]), dt, red)
    torch.cuda.synchronize()
    ref = o.tck(cfg["U0"], dt, red)
    assert rel_l2(Ub.cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("method", ["lsrk", "ader"])
def test_standing_wave_100_steps_fp64(method):
    torch = _cuda()
    cfg = synth.configs.standing_wave(N=4, k=3, cr=0.1, nsteps=100)
    s, o = pair(cfg)
    U = s.to_device(cfg["U0"])
    if method == "lsrk":
        s.step_lsrk(U, cfg["dt"], 100)
        ref = o.lsrk(cfg["U0"], cfg["dt"], 100)
    else:
        s.step_ader(U, cfg["dt"], 100, 2)
        ref = o.ader(cfg["U0"], cfg["dt"], 100, 2)
    torch.cuda.synchronize()
    assert rel_l2(U.cpu().numpy(), ref) < 1e-12
    # and it is the standing wave
    assert o.l2_error(U.cpu().numpy(), cfg["exact"], 100 * cfg["dt"])[0] < 2e-2


@pytest.mark.parametrize("method", ["lsrk", "ader"])
def test_curved_pulse_steps(method):
    torch = _cuda()
    cfg = synth.configs.curved_pulse(N=3, k=4, nsteps=20)
    s, o = pair(cfg)
    for prec, tol in ((dgw.DG_FP64, 1e-12), (dgw.DG_FP32, 1e-5)):
        s = dgw.Solver(cfg["mesh"], cfg["k"], prec, 1.0, cfg["rho"], cfg["c"])
        U = s.to_device(cfg["U0"])
        if method == "lsrk":
            s.step_lsrk(U, cfg["dt"], 20)
        else:
            s.step_ader(U, cfg["dt"], 20, 2)
        torch.cuda.synchronize()
        ref = o.lsrk(cfg["U0"], cfg["dt"], 20) if method == "lsrk" else o.ader(cfg["U0"], cfg["dt"], 20, 2)
        assert rel_l2(U.cpu().numpy(), ref) < tol, prec


def test_energy_and_norms():
    torch = _cuda()
    cfg = _curved(3, 3, seed=4)
    s, o = pair(cfg)
    U = s.to_device(cfg["U0"])
    e = s.energy(U)
    assert abs(e - o.energy(cfg["U0"])) / o.energy(cfg["U0"]) < 1e-13
    V = s.to_device(cfg["U0"] * 0.5)
    aa, dd = s.norms(U, V)
    assert abs(aa - np.sum(cfg["U0"] ** 2)) / aa < 1e-13
    assert abs(dd - np.sum((0.5 * cfg["U0"]) ** 2)) / dd < 1e-13


@pytest.mark.parametrize("case", ["single_wall", "single_periodic", "ragged"])
def test_edge_meshes(case):
    torch = _cuda()
    k = 3
    if case == "single_wall":
        mesh = synth.cube_mesh(1, q=2, periodic=False, deform=synth.mesh.curving(0.03))
    elif case == "single_periodic":
        mesh = synth.cube_mesh(1, q=1, periodic=True)
    else:  # 5^3 = 125 elements: not a multiple of the elements per block
        mesh = synth.cube_mesh(5, q=1, periodic=(True, False, True))
    E = mesh["n_elem"]
    x = synth.solution_node_positions(mesh, k)
    rho, c = synth.fields.cfg2_coefficients(x)
    cfg = {"mesh": mesh, "k": k, "rho": rho, "c": c, "alpha": 1.0,
           "U0": synth.configs.random_state(E, k, 3)}
    s, o = pair(cfg)
    R = s.apply(s.to_device(cfg["U0"]))
    Ub = s.tck(s.to_device(cfg["U0"]), 0.01, 2)
    torch.cuda.synchronize()
    assert rel_l2(R.cpu().numpy(), o.apply(cfg["U0"])) < 1e-13
    assert rel_l2(Ub.cpu().numpy(), o.tck(cfg["U0"], 0.01, 2)) < 1e-13


def test_solve_host_matches_device():
    torch = _cuda()
    cfg = _curved(2, 3, seed=8)
    s, o = pair(cfg)
    Uh = torch.from_numpy(cfg["U0"]).pin_memory()
    out = torch.empty_like(Uh).pin_memory()
    s.solve_host(1, Uh, out, 0.005, 3, 2)
    U = s.to_device(cfg["U0"])
    s.step_ader(U, 0.005, 3, 2)
    torch.cuda.synchronize()
    assert torch.equal(out, U.cpu())


@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("scheme", [dgw.LSRK_CK54, dgw.LSRK59])
def test_solve_host_fused_transfers(prec, method, scheme):
    """Gauss-point states with pinned host buffers: the transfers are fused
    with the changes of basis (kernels read and write the host buffers).
    Bitwise the same as pageable buffers (plain copies, the steppers change
    basis) and as stepping a device state; at oracle parity."""
    torch = _cuda()
    if method == 1 and scheme != dgw.LSRK_CK54:
        pytest.skip("the LSRK scheme does not apply to ADER")
    cfg = _curved(3, 3, seed=12)
    s, o = pair(cfg, prec)
    s.set_basis(dgw.BASIS_G)
    s.set_lsrk_scheme(scheme)
    dt = 0.004
    Uh = torch.from_numpy(cfg["U0"]).to(s.dtype)
    pinned_in, pinned_out = Uh.pin_memory(), torch.empty_like(Uh).pin_memory()
    page_in, page_out = Uh.clone(), torch.empty_like(Uh)
    s.solve_host(method, pinned_in, pinned_out, dt, 2, 2)
    s.solve_host(method, page_in, page_out, dt, 2, 2)
    U = s.to_device(cfg["U0"])
    if method == 0:
        s.step_lsrk(U, dt, 2)
    else:
        s.step_ader(U, dt, 2, 2)
    torch.cuda.synchronize()
    assert torch.equal(pinned_out, page_out)
    assert torch.equal(pinned_out, U.cpu())
    if method == 1:
        ref = o.ader(cfg["U0"], dt, 2, 2)
    elif scheme == dgw.LSRK_CK54:
        ref = o.lsrk(cfg["U0"], dt, 2)
    else:
        from oracle import LSRK59_KCL_A, LSRK59_KCL_B
        ref = o.lsrk2r(cfg["U0"], dt, 2, LSRK59_KCL_A, LSRK59_KCL_B)
    err = rel_l2(pinned_out.double().numpy(), ref)
    assert err < (1e-12 if prec == dgw.DG_FP64 else 2e-5), err


def test_errors_are_reported():
    torch = _cuda()
    cfg = _curved(2, 2, seed=1)
    s, _ = pair(cfg)
    U = s.to_device(cfg["U0"])
    with pytest.raises(dgw.DGError):
        s.step_ader(U, 0.01, 1, reduce_every=5)
    with pytest.raises(dgw.DGError):
        s.step_lsrk(U, -1.0, 1)
    bad = np.array(cfg["rho"])
    bad[0, 0] = -1.0
    with pytest.raises(dgw.DGError):
        s.set_coefficients(bad, cfg["c"])
    # a curved mesh folded onto itself is rejected at set-up
    mesh = synth.cube_mesh(2, q=2, periodic=False, deform=synth.mesh.curving(0.5))
    with pytest.raises(dgw.DGError):
        dgw.Solver(mesh, 2)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("method", ["lsrk", "ader"])
def test_gauss_basis_steppers_match_oracle(k, method):
    """The steppers with the state kept at the Gauss points (DG_BASIS_G) run
    the same discrete scheme: same oracle parity as the GL storage."""
    torch = _cuda()
    cfg = _curved(2 if k >= 5 else 3, k, seed=30 + k, periodic=(k % 2 == 1))
    dt = 0.004
    s, o = pair(cfg)
    s.set_basis(dgw.BASIS_G)
    assert s.basis() == dgw.BASIS_G
    U = s.to_device(cfg["U0"])
    if method == "lsrk":
        s.step_lsrk(U, dt, 3)
        ref = o.lsrk(cfg["U0"], dt, 3)
    else:
        s.step_ader(U, dt, 3, 2)
        ref = o.ader(cfg["U0"], dt, 3, 2)
    torch.cuda.synchronize()
    assert rel_l2(U.cpu().numpy(), ref) < 1e-12
    s32 = dgw.Solver(cfg["mesh"], k, dgw.DG_FP32, 1.0, cfg["rho"], cfg["c"])
    s32.set_basis(dgw.BASIS_G)
    V = s32.to_device(cfg["U0"])
    if method == "lsrk":
        s32.step_lsrk(V, dt, 3)
    else:
        s32.step_ader(V, dt, 3, 2)
    torch.cuda.synchronize()
    s32.check_device()
    assert rel_l2(V.cpu().numpy(), ref) < 2e-5


def test_misaligned_state_rejected():
    torch = _cuda()
    cfg = _curved(2, 2, seed=3)
    s, _ = pair(cfg)
    n = cfg["U0"].size
    buf = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    view = buf[1:].view(cfg["U0"].shape)          # 8-byte offset
    with pytest.raises(dgw.DGError):
        s.step_lsrk(view, 0.001, 1)


def _affine_piecewise(N, k, seed, periodic=True):
    from oracle_helpers import SHEAR, linear_map
    mesh = synth.cube_mesh(N, q=1, periodic=periodic, deform=linear_map(SHEAR))
    rng = np.random.default_rng(seed)
    E, n3 = N ** 3, (k + 1) ** 3
    rho = rng.uniform(0.6, 1.6, size=(E, 1)) * np.ones((1, n3))   # constant per element, jumps between
    c = rng.uniform(0.6, 1.6, size=(E, 1)) * np.ones((1, n3))
    return {"mesh": mesh, "k": k, "rho": rho, "c": c, "alpha": 1.0,
            "U0": synth.configs.random_state(E, k, seed + 1)}


def test_affine_detection():
    _cuda()
    cfg = _affine_piecewise(2, 3, 1)
    s, _ = pair(cfg)
    assert s.is_affine()
    x = synth.solution_node_positions(cfg["mesh"], 3)
    rho, c = synth.fields.cfg2_coefficients(x)
    s.set_coefficients(rho, c)                    # varies inside elements
    assert not s.is_affine()
    s.set_coefficients(cfg["rho"], cfg["c"])
    assert s.is_affine()
    curved = _curved(2, 3, seed=2)
    sc, _ = pair(curved)
    assert not sc.is_affine()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("basis", ["g", "gl"])
def test_affine_steppers_match_oracle(k, basis):
    """Affine elements with element-wise constant coefficients (impedance
    jumps across faces) run the compact-data kernels: same parity."""
    torch = _cuda()
    cfg = _affine_piecewise(3 if k <= 4 else 2, k, seed=40 + k, periodic=(k % 2 == 0))
    s, o = pair(cfg)
    assert s.is_affine()
    s.set_basis(dgw.BASIS_G if basis == "g" else dgw.BASIS_GL)
    dt = 0.003
    for method in ("lsrk", "ader"):
        U = s.to_device(cfg["U0"])
        if method == "lsrk":
            s.step_lsrk(U, dt, 3)
            ref = o.lsrk(cfg["U0"], dt, 3)
        else:
            s.step_ader(U, dt, 3, 2)
            ref = o.ader(cfg["U0"], dt, 3, 2)
        torch.cuda.synchronize()
        assert rel_l2(U.cpu().numpy(), ref) < 1e-12, method
        s32 = dgw.Solver(cfg["mesh"], k, dgw.DG_FP32, 1.0, cfg["rho"], cfg["c"])
        s32.set_basis(s.basis())
        V = s32.to_device(cfg["U0"])
        if method == "lsrk":
            s32.step_lsrk(V, dt, 3)
        else:
            s32.step_ader(V, dt, 3, 2)
        torch.cuda.synchronize()
        s32.check_device()
        assert rel_l2(V.cpu().numpy(), ref) < 2e-5, method


@pytest.mark.parametrize("geometry", ["affine", "curved"])
@pytest.mark.parametrize("k", [2, 4])
def test_operator_tilings_fp32(geometry, k):
    """The FP32 Gauss-point operators (staged tiles) with 1 to 4 elements per
    block over a 27-element periodic mesh: neighbours that are block-mates
    (x-neighbours, and y-neighbours where a block wraps a row, the periodic
    seam included) take their traces from the staged tiles, the others from
    global memory; the last block is ragged.  LSRK and ADER steps against
    the oracle."""
    torch = _cuda()
    cfg = (_affine_piecewise(3, k, seed=70 + k, periodic=True) if geometry == "affine"
           else _curved(3, k, seed=70 + k, periodic=True))
    s, o = pair(cfg)
    refs = {"lsrk": o.lsrk(cfg["U0"], 0.003, 2), "ader": o.ader(cfg["U0"], 0.003, 2, 2)}
    s32 = dgw.Solver(cfg["mesh"], k, dgw.DG_FP32, 1.0, cfg["rho"], cfg["c"])
    s32.set_basis(dgw.BASIS_G)
    assert s32.is_affine() == (geometry == "affine")
    for epb in (1, 2, 3, 4):
        s32.set_tiling(epb, 0)
        for method, ref in refs.items():
            V = s32.to_device(cfg["U0"])
            if method == "lsrk":
                s32.step_lsrk(V, 0.003, 2)
            else:
                s32.step_ader(V, 0.003, 2, 2)
            torch.cuda.synchronize()
            s32.check_device()
            assert rel_l2(V.cpu().numpy(), ref) < 2e-5, (epb, method)
