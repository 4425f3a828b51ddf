"""Parity at the bench's full sizes and launch configuration, on sampled
elements: the GPU runs the whole mesh (curved pulse 32^3 at k = 5 in FP64
and FP32, plane wave 64^3 at k = 4 in FP32) with the bench's state basis,
predictor form and autotuned tiling; the oracle computes the seeded sample
elements exactly on patches cut around them (tests/patch_helpers.py: one
layer for the operator and an ADER step, five for an LSRK step).

States are seeded random values on the bench's mesh and coefficients, so
every sampled element carries O(1) data; one check uses the bench's own
pulse.  Samples include the first and last element (mesh corners, walls or
the periodic seam).  Tolerances as at small sizes: FP64 <= 1e-12, FP32
<= 2e-5 relative l2 over the sampled elements."""
import numpy as np
import pytest

import oracle
import synth
import paper_1805_03981_gb300 as dgw
from paper_1805_03981_gb300 import autotune
from gpu_helpers import rel_l2
from patch_helpers import patch

pytestmark = pytest.mark.gpu


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


_CFG = {}


def _config(name):
    if name not in _CFG:
        _CFG[name] = (synth.configs.curved_pulse(N=32, k=5) if name == "curved_pulse"
                      else synth.configs.plane_wave(N=64, k=4))
    return _CFG[name]


def _solver(cfg, prec):
    """The bench's solver: Gauss-point states and autotuned tiling."""
    s = dgw.Solver(cfg["mesh"], cfg["k"], prec, cfg["alpha"], cfg["rho"], cfg["c"])
    s.set_basis(dgw.BASIS_G)
    for kind in (dgw.KIND_LSRK, dgw.KIND_TCK):
        s.tune(kind, autotune.CANDIDATES, reps=1)
    return s


def _seeds(E, seed):
    rng = np.random.default_rng(seed)
    return sorted({0, E - 1, *(int(e) for e in rng.choice(E, 3, replace=False))})


def _oracle_at(cfg, U0, seeds, radius, run):
    """The oracle's result at each seed, from a patch of that radius."""
    out = []
    for s in seeds:
        sub, ids, rho, c, V, loc = patch(cfg["mesh"], cfg["rho"], cfg["c"], U0, [s], radius)
        o = oracle.Oracle(sub, cfg["k"], rho, c, cfg["alpha"])
        out.append(run(o, V)[loc[0]])
    return np.stack(out)


@pytest.mark.parametrize("name,prec", [("curved_pulse", dgw.DG_FP64), ("curved_pulse", dgw.DG_FP32),
                                       ("plane_wave", dgw.DG_FP32)])
def test_fullsize_ader_step(name, prec):
    torch = _cuda()
    cfg = _config(name)
    E, k, dt = cfg["mesh"]["n_elem"], cfg["k"], cfg["dt"]
    U0 = synth.configs.random_state(E, k, 600)
    s = _solver(cfg, prec)
    U = s.to_device(U0)
    s.step_ader(U, dt, 1, 2)
    torch.cuda.synchronize()
    seeds = _seeds(E, 601)
    got = U[seeds].double().cpu().numpy()
    s.close()
    ref = _oracle_at(cfg, U0, seeds, 1, lambda o, V: o.ader(V, dt, 1, 2))
    assert rel_l2(got, ref) < (1e-12 if prec == dgw.DG_FP64 else 2e-5)


@pytest.mark.parametrize("name,prec", [("curved_pulse", dgw.DG_FP64), ("curved_pulse", dgw.DG_FP32),
                                       ("plane_wave", dgw.DG_FP32)])
def test_fullsize_lsrk_step(name, prec):
    torch = _cuda()
    cfg = _config(name)
    E, k, dt = cfg["mesh"]["n_elem"], cfg["k"], cfg["dt"]
    U0 = synth.configs.random_state(E, k, 610)
    s = _solver(cfg, prec)
    U = s.to_device(U0)
    s.step_lsrk(U, dt, 1)
    torch.cuda.synchronize()
    seeds = _seeds(E, 611)[:3]
    got = U[seeds].double().cpu().numpy()
    s.close()
    ref = _oracle_at(cfg, U0, seeds, 5, lambda o, V: o.lsrk(V, dt, 1))
    assert rel_l2(got, ref) < (1e-12 if prec == dgw.DG_FP64 else 2e-5)


def test_fullsize_operator():
    torch = _cuda()
    cfg = _config("curved_pulse")
    E, k = cfg["mesh"]["n_elem"], cfg["k"]
    U0 = synth.configs.random_state(E, k, 620)
    s = dgw.Solver(cfg["mesh"], k, dgw.DG_FP64, cfg["alpha"], cfg["rho"], cfg["c"])
    R = s.apply(s.to_device(U0))
    torch.cuda.synchronize()
    seeds = _seeds(E, 621)
    got = R[seeds].cpu().numpy()
    s.close()
    assert rel_l2(got, _oracle_at(cfg, U0, seeds, 1, lambda o, V: o.apply(V))) < 1e-12


def test_fullsize_pulse_steps():
    """The bench's own state (the Gaussian pulse) through one ADER and one
    LSRK step, sampled where the pulse is (the element holding its largest
    value and its neighbours) and at the corners.  The comparison is of the
    state after the step, as for the small sizes: the raw operator on this
    steep pulse (width 1.6 elements) is the sum of terms far larger than
    itself, and two rounding orders of it differ by about 1e-11 relative."""
    torch = _cuda()
    cfg = _config("curved_pulse")
    E, k, dt = cfg["mesh"]["n_elem"], cfg["k"], cfg["dt"]
    U0 = cfg["U0"]
    peak = int(np.argmax(np.abs(U0[:, 0]).max(axis=1)))
    s = _solver(cfg, dgw.DG_FP64)
    Ua = s.to_device(U0)
    s.step_ader(Ua, dt, 1, 2)
    Ul = s.to_device(U0)
    s.step_lsrk(Ul, dt, 1)
    torch.cuda.synchronize()
    seeds = sorted({0, E - 1, peak, *(int(e) for e in cfg["mesh"]["nbr"][peak] if e >= 0)})
    got_a = Ua[seeds].cpu().numpy()
    got_l = Ul[[peak]].cpu().numpy()
    s.close()
    ref_a = _oracle_at(cfg, U0, seeds, 1, lambda o, V: o.ader(V, dt, 1, 2))
    assert rel_l2(got_a, ref_a) < 1e-12
    assert np.abs(ref_a - U0[seeds]).max() > 1e-3  # the step moves the sampled state
    assert rel_l2(got_l, _oracle_at(cfg, U0, [peak], 5, lambda o, V: o.lsrk(V, dt, 1))) < 1e-12
