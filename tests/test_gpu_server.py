"""Served form: a request's result is the same alone and in a mix of
concurrently admitted solves (bitwise, and equal to the single-solve path);
admission respects the HBM budget; oversize requests are rejected."""
import time

import numpy as np
import pytest

import synth
import paper_1805_03981_gb300 as dgw

pytestmark = pytest.mark.gpu


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _req(seed, N, k, nsteps, method=1):
    c = synth.configs.random_instance(seed, N=N, k=k, nsteps=nsteps, curved=False)
    c["method"] = method
    return c


def _submit(srv, c, prec):
    dt = np.float64 if prec == dgw.DG_FP64 else np.float32
    return srv.submit(c["mesh"], c["k"], c["rho"], c["c"], c["U0"].astype(dt), c["dt"], c["nsteps"],
                      method=c["method"], reduce_every=2)


def _wait(srv, ticket, limit_s=120):
    t0 = time.time()
    while True:
        r = srv.poll(ticket, timeout_ms=200)
        if r is not None:
            return r
        assert time.time() - t0 < limit_s, "request did not finish"


@pytest.mark.parametrize("prec", [dgw.DG_FP32, dgw.DG_FP64])
def test_alone_equals_mix_equals_solver(prec):
    torch = _cuda()
    target = _req(11, 4, 3, 21)
    others = [_req(20 + i, N, k, s, m) for i, (N, k, s, m) in
              enumerate([(3, 5, 3000, 1), (5, 2, 3000, 1), (2, 7, 13, 1), (4, 4, 17, 0), (3, 3, 25, 0)])]
    srv = dgw.Server(8 << 30, prec=prec, chunk_steps=5)
    alone = _wait(srv, _submit(srv, target, prec))
    assert alone["status"] == 0
    # the mix: two long solves first; the target once they run; the rest after it
    t = [_submit(srv, o, prec) for o in others[:2]]
    t0 = time.time()
    while srv.stats()["active"] < 2:
        assert time.time() - t0 < 60
        time.sleep(0.001)
    tt = _submit(srv, target, prec)
    t += [_submit(srv, o, prec) for o in others[2:]]
    mixed = _wait(srv, tt)
    rest = [_wait(srv, x) for x in t]
    assert all(r["status"] == 0 for r in rest)
    assert np.array_equal(alone["out"], mixed["out"])
    # the target's solve overlapped with the long ones
    assert mixed["t_admit"] < min(r["t_done"] for r in rest[:2])
    st = srv.stats()
    assert st["completed"] == 1 + 1 + len(others) and st["peak_active"] >= 3
    srv.close()
    s = dgw.Solver(target["mesh"], target["k"], prec, 1.0, target["rho"], target["c"])
    s.set_basis(dgw.BASIS_G)            # the server keeps admitted states at the Gauss points
    U = s.to_device(target["U0"])
    s.step_ader(U, target["dt"], target["nsteps"], 2)
    torch.cuda.synchronize()
    assert np.array_equal(U.cpu().numpy(), mixed["out"])


def test_budget_admission_and_rejection():
    _cuda()
    reqs = [_req(40 + i, 3, 3, 12) for i in range(6)]
    probe = dgw.Server(1 << 30, prec=dgw.DG_FP32)
    est = probe.request_bytes(27, 3, 1)           # what one of these solves reserves
    probe.close()
    assert est > 0
    # a budget for two of these solves at a time
    srv = dgw.Server(int(2.5 * est), prec=dgw.DG_FP32, chunk_steps=4)
    tickets = [_submit(srv, r, dgw.DG_FP32) for r in reqs]
    res = [_wait(srv, t) for t in tickets]
    assert all(r["status"] == 0 for r in res)
    st = srv.stats()
    assert st["hbm_peak"] <= int(2.5 * est)
    assert st["peak_active"] <= 2
    big = _req(50, 6, 5, 5)
    with pytest.raises(dgw.DGError):
        _submit(srv, big, dgw.DG_FP32)
    srv.close()
