"""dg_energy_noalloc: the allocation-free energy, for callers that must not
allocate device memory while running (for example a server that has
committed its whole HBM budget).  Its partial sums live in a fixed device
array owned by the library instead of context scratch.  Called through the C
ABI twice in a row on different states, it must agree with dg_energy.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process,
where its first call is the one that resolves the array's device address.
"""
import numpy as np
import pytest

import synth
import paper_1805_03981_gb300 as dgw

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
def test_energy_noalloc_matches_energy(prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = synth.configs.curved_pulse(N=5, k=3)
    s = dgw.Solver(cfg["mesh"], cfg["k"], prec, 1.0, cfg["rho"], cfg["c"])
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    states = [cfg["U0"], synth.configs.random_state(cfg["mesh"]["n_elem"], cfg["k"], 11)]
    for U0 in states:                      # two calls in a row, different data
        U = s.to_device(U0)
        s.energy_noalloc(U, out)
        torch.cuda.synchronize()
        ref = s.energy(U)
        assert abs(out.item() - ref) <= 1e-13 * abs(ref), (out.item(), ref)
    s.close()
