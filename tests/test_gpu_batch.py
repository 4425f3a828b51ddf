"""Batched form: independent solves (mixed degrees and sizes) advanced by
persistent launches give, for every solve, exactly (bitwise) the state the
single-solve path gives, and that state matches the oracle."""
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


def _mix(seed, count, prec):
    rng = np.random.default_rng(seed)
    cfgs = []
    ks = [2, 3, 4, 5, 6, 7]
    for i in range(count):
        k = ks[i % len(ks)]
        N = int(rng.integers(2, 5 if k >= 6 else 6))
        cfgs.append(synth.configs.random_instance(seed * 1000 + i, N=N, k=k, nsteps=10))
    solvers = [dgw.Solver(c["mesh"], c["k"], prec, c["alpha"], c["rho"], c["c"]) for c in cfgs]
    return cfgs, solvers


@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
@pytest.mark.parametrize("method", ["ader", "lsrk"])
def test_batch_bitwise_equals_alone(prec, method):
    torch = _cuda()
    cfgs, solvers = _mix(3, 9, prec)
    steps = 11                                     # one captured chunk of 8 and 3 direct steps
    alone = []
    for c, s in zip(cfgs, solvers):
        U = s.to_device(c["U0"])
        if method == "ader":
            s.step_ader(U, c["dt"], steps, 2)
        else:
            s.step_lsrk(U, c["dt"], steps)
        alone.append(U)
    states = [s.to_device(c["U0"]) for c, s in zip(cfgs, solvers)]
    b = dgw.Batch(solvers, states, [c["dt"] for c in cfgs])
    if method == "ader":
        b.step_ader(steps, 2)
    else:
        b.step_lsrk(steps)
    torch.cuda.synchronize()
    for i, (u, v) in enumerate(zip(states, alone)):
        assert torch.equal(u, v), (i, cfgs[i]["k"], (u - v).abs().max().item())
    info = b.info()
    assert info["instances"] == 9 and info["launches"] > 0
    b.close()


def test_batch_matches_oracle_and_tiling_invariance():
    torch = _cuda()
    cfgs, solvers = _mix(5, 3, dgw.DG_FP64)
    c0, s0 = cfgs[0], solvers[0]
    s0.set_tiling(1, 1)                            # a different tiling changes nothing
    states = [s.to_device(c["U0"]) for c, s in zip(cfgs, solvers)]
    b = dgw.Batch(solvers, states, [c["dt"] for c in cfgs])
    b.step_ader(3, 2)
    torch.cuda.synchronize()
    _, o = pair(c0)
    ref = o.ader(c0["U0"], c0["dt"], 3, 2)
    assert rel_l2(states[0].cpu().numpy(), ref) < 1e-12
    b.close()


def test_autotune_table_records_tiling_and_predictor_form():
    """autotune.tune times the Gauss-basis kernels and both predictor forms;
    the recorded form is the faster one, and apply sets it on a curved
    solver but not on an affine one."""
    _cuda()
    from paper_1805_03981_gb300 import autotune
    table = autotune.tune(("fp32",), [3], reps=1)
    for cls in autotune.SIZE_CLASSES:
        r = table["fp32"]["3"][cls]
        assert r["pred"] in ("lines", "columns")
        other = "lines" if r["pred"] == "columns" else "columns"
        assert r["tck"]["ms"] == r["tck_" + r["pred"]]["ms"] <= r["tck_" + other]["ms"]
        assert r["epb_tck"] == r["tck_" + r["pred"]]["epb"]
    cfg = synth.configs.curved_pulse(N=4, k=3)
    s = dgw.Solver(cfg["mesh"], 3, dgw.DG_FP32, 1.0, cfg["rho"], cfg["c"])
    autotune.apply(s, table)
    want = dgw.PRED_COLUMNS if table["fp32"]["3"]["small"]["pred"] == "columns" else dgw.PRED_LINES
    assert s.predictor_kernel() == want
    s.close()
    c = synth.configs.standing_wave(N=4, k=3)
    s = dgw.Solver(c["mesh"], 3, dgw.DG_FP32, 1.0, c["rho"], c["c"])
    autotune.apply(s, table)
    assert s.predictor_kernel() == dgw.PRED_AUTO
    s.close()


def test_tune_sets_a_valid_tiling():
    torch = _cuda()
    cfg = synth.configs.curved_pulse(N=4, k=4)
    s = dgw.Solver(cfg["mesh"], 4, dgw.DG_FP32, 1.0, cfg["rho"], cfg["c"])
    ms = s.tune(dgw.KIND_LSRK, [1, 2, 3, 5, 40], reps=2)
    assert ms[-1] == -1.0                          # 40 x 25 threads > 1024: impossible
    assert all(m > 0 for m in ms[:-1])
    assert s.tiling()[0] == [1, 2, 3, 5][int(np.argmin(ms[:-1]))]


@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
@pytest.mark.parametrize("method", ["ader", "ader_red0", "lsrk"])
def test_batch_gauss_basis_bitwise_equals_alone(prec, method):
    """Gauss-basis batches (general and affine solves mixed) give each solve
    exactly the state of its own Gauss-basis stepping.  Batches run the
    column-form predictor for FP32 Gauss-point states; stepped alone, an FP32
    solve on affine elements with constant coefficients runs the interleaved
    form (the same arithmetic, other rounding), so for those the batch is
    compared bitwise with the column form alone and to FP32 rounding with
    the interleaved form."""
    torch = _cuda()
    cfgs, solvers = _mix(7, 6, prec)
    for k in (3, 5):                                    # affine, constant coefficients
        c = synth.configs.standing_wave(N=3, k=k)
        cfgs.append(c)
        solvers.append(dgw.Solver(c["mesh"], k, prec, 1.0, c["rho"], c["c"]))
    assert solvers[-1].is_affine() and not solvers[0].is_affine()
    steps = 11

    def step(s, U, dt):
        if method.startswith("ader"):
            s.step_ader(U, dt, steps, 0 if method == "ader_red0" else 2)
        else:
            s.step_lsrk(U, dt, steps)

    alone, interleaved = [], {}
    for i, (c, s) in enumerate(zip(cfgs, solvers)):
        s.set_basis(dgw.BASIS_G)
        if prec == dgw.DG_FP32 and s.is_affine() and method.startswith("ader"):
            U = s.to_device(c["U0"])
            step(s, U, c["dt"])                         # DG_PRED_AUTO: the interleaved form
            interleaved[i] = U
            s.set_predictor_kernel(dgw.PRED_COLUMNS)
        U = s.to_device(c["U0"])
        step(s, U, c["dt"])
        alone.append(U)
    assert len(interleaved) == (2 if prec == dgw.DG_FP32 and method.startswith("ader") else 0)
    states = [s.to_device(c["U0"]) for c, s in zip(cfgs, solvers)]
    b = dgw.Batch(solvers, states, [c["dt"] for c in cfgs])
    b.set_basis(dgw.BASIS_G, convert_each_call=True)
    if method.startswith("ader"):
        b.step_ader(steps, 0 if method == "ader_red0" else 2)
    else:
        b.step_lsrk(steps)
    torch.cuda.synchronize()
    for i, (u, v) in enumerate(zip(states, alone)):
        assert torch.equal(u, v), (i, (u - v).abs().max().item())
    for i, v in interleaved.items():
        assert rel_l2(states[i].cpu().numpy(), v.cpu().numpy()) < 1e-5, i
    b.close()
