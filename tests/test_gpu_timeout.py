"""The give-up path of the bounded device waits.

The FP32 Gauss-basis operators stage their inputs by bulk copies completed
on an mbarrier and wait for them with a bounded poll loop.  With the test
setting dg_test_expire_waits, the first wait gives up at once: each block
sets the device status, drains its own copies with the second bounded wait
and returns without results.  dg_check_device must then report DG_ETIMEOUT
once, and after the setting is cleared the same context must step to oracle
parity with a clean status.  No kernel hangs or faults here: the copies are
valid and always complete.
"""
import numpy as np
import pytest

import synth
import oracle
import paper_1805_03981_gb300 as dgw

pytestmark = pytest.mark.gpu

DG_ETIMEOUT = -6


@pytest.mark.parametrize("recipe", ["curved", "affine"])
def test_expired_wait_reports_timeout_then_recovers(recipe):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if recipe == "curved":
        cfg = synth.configs.curved_pulse(N=3, k=3, nsteps=1)
    else:
        cfg = synth.configs.standing_wave(N=3, k=3, nsteps=1)
    s = dgw.Solver(cfg["mesh"], cfg["k"], dgw.DG_FP32, cfg["alpha"], cfg["rho"], cfg["c"])
    s.set_basis(dgw.BASIS_G)
    s.test_expire_waits(True)
    U = s.to_device(cfg["U0"])
    s.step_lsrk(U, cfg["dt"], 1)
    with pytest.raises(dgw.DGError) as ei:
        s.check_device()
    assert ei.value.status == DG_ETIMEOUT
    s.check_device()                       # reported once, then cleared
    s.test_expire_waits(False)
    U = s.to_device(cfg["U0"])
    s.step_lsrk(U, cfg["dt"], 1)
    s.check_device()
    o = oracle.Oracle(cfg["mesh"], cfg["k"], cfg["rho"], cfg["c"], cfg["alpha"])
    ref = o.lsrk(cfg["U0"], cfg["dt"], 1)
    err = np.linalg.norm(U.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < 2e-5, err
    s.close()
