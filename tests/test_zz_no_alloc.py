"""dg_energy_noalloc: the allocation-free energy, for callers that must not
allocate device memory while running (for example a server that has
committed its whole HBM budget).  Its partial sums live in a fixed device
array owned by the library instead of context scratch.  Called through the C
ABI twice in a row on different states, it must agree with dg_energy, and
repeated calls must leave the device's free memory and the context's own
allocation count unchanged.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process,
where its first call is the one that resolves the array's device address.
"""
import numpy as np
import pytest

import synth
import paper_1805_03981_gb300 as dgw

pytestmark = pytest.mark.gpu

DG_EINVAL = -1


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
def test_energy_noalloc_matches_energy(prec):
    torch = _torch()
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


def test_energy_noalloc_allocates_nothing():
    torch = _torch()
    cfg = synth.configs.curved_pulse(N=4, k=4)
    s = dgw.Solver(cfg["mesh"], cfg["k"], dgw.DG_FP64, 1.0, cfg["rho"], cfg["c"])
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    U = s.to_device(cfg["U0"])
    s.energy_noalloc(U, out)               # the first call on this device resolves the array's address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ctx0 = s.device_bytes()
    torch0 = torch.cuda.memory_allocated()
    vals = []
    for _ in range(5):
        s.energy_noalloc(U, out)
        torch.cuda.synchronize()
        vals.append(out.item())
    assert torch.cuda.mem_get_info()[0] == free0
    assert s.device_bytes() == ctx0
    assert torch.cuda.memory_allocated() == torch0
    assert len(set(vals)) == 1             # fixed summation order: the same bits every call
    s.close()


def test_energy_noalloc_rejects_bad_arguments():
    torch = _torch()
    cfg = synth.configs.curved_pulse(N=3, k=2)
    s = dgw.Solver(cfg["mesh"], cfg["k"], dgw.DG_FP64, 1.0, cfg["rho"], cfg["c"])
    U = s.to_device(cfg["U0"])
    host = torch.zeros(1, dtype=torch.float64)
    with pytest.raises(dgw.DGError):
        s.energy_noalloc(U, host)          # the binding refuses a CPU tensor
    # the library itself refuses a host address (checked before any launch)
    assert s.energy_noalloc_raw(U, host.data_ptr()) == DG_EINVAL
    s.check_device()
    s.close()


def test_energy_noalloc_rejects_meshes_beyond_its_array():
    """At k = 5 the energy kernel takes 3 elements per block, so the fixed
    array of 16384 partial sums covers 49152 elements; 37^3 = 50653 is too
    many, and the call must say so instead of writing past the array."""
    torch = _torch()
    N, k = 37, 5
    mesh = synth.cube_mesh(N, q=1, periodic=True)
    ones = np.ones((N ** 3, (k + 1) ** 3))
    s = dgw.Solver(mesh, k, dgw.DG_FP32, 1.0, ones, ones)
    U = torch.zeros((N ** 3, 4, (k + 1) ** 3), dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(dgw.DGError) as ei:
        s.energy_noalloc(U, out)
    assert ei.value.status == DG_EINVAL
    assert "partial sums" in str(ei.value)
    s.close()
