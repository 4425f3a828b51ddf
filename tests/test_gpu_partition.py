"""Partitioned solve on the GPU (dg_set_owned, dg_part_*): several parts
with ghost exchanges give owned states bitwise equal to one context on the
whole mesh running the same kernels."""
import numpy as np
import pytest

import synth
import paper_1805_03981_gb300 as dgw
from paper_1805_03981_gb300 import partition

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
    return mesh, rho, c, synth.configs.random_state(N ** 3, k, seed + 1)


@pytest.mark.parametrize("P", [2, 3])
@pytest.mark.parametrize("basis", [dgw.BASIS_GL, dgw.BASIS_G])
@pytest.mark.parametrize("prec", [dgw.DG_FP64, dgw.DG_FP32])
def test_parts_bitwise_equal_whole(P, basis, prec):
    torch = _cuda()
    for k, N, periodic in ((2, 4, True), (5, 3, False)):
        mesh, rho, c, U0 = _curved(N, k, 30 + k, periodic)
        whole = dgw.Solver(mesh, k, prec, 1.0, rho, c)
        whole.set_basis(basis)
        pt = partition.Partitioned(mesh, k, P, prec, 1.0, rho, c, basis)
        dt = 0.003
        for method in ("lsrk", "ader"):
            U = whole.to_device(U0)
            states = pt.to_device(U0)
            if method == "lsrk":
                whole.step_lsrk(U, dt, 3)
                pt.step_lsrk(dt, 3)
            else:
                whole.step_ader(U, dt, 3, 2)
                pt.step_ader(dt, 3, 2)
            torch.cuda.synchronize()
            got = pt.gather(states)
            ref = U.double().cpu().numpy()
            assert np.array_equal(got, ref), (k, method, float(np.abs(got - ref).max()))
            info = pt.info()                       # to_device binds a fresh part object
            assert info["parts"] == P and info["ghosts"] > 0
            assert info["exchanges"] == (3 * 5 if method == "lsrk" else 3)   # 5 per LSRK step, 1 per ADER step
        pt.close()
        whole.close()


def test_part_arguments_rejected():
    _cuda()
    mesh, rho, c, U0 = _curved(2, 2, 3, True)
    parts = partition.split(mesh, 2, rho, c)
    s = dgw.Solver(parts[0]["mesh"], 2, dgw.DG_FP64, 1.0, parts[0]["rho"], parts[0]["c"])
    with pytest.raises(dgw.DGError):
        s.set_owned(0)
    with pytest.raises(dgw.DGError):
        s.set_owned(parts[0]["mesh"]["n_elem"] + 1)
    pt = partition.Partitioned(mesh, 2, 2, dgw.DG_FP64, 1.0, rho, c)
    pt.parts[1]["src_part"] = np.full_like(pt.parts[1]["src_part"], 1)   # a ghost of itself
    with pytest.raises(dgw.DGError):
        pt.to_device(U0)
