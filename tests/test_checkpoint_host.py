"""Checkpoint files (paper_1805_03981_gb300.checkpoint) on the host: the
archive round trip, the problem fingerprint and the checks a restart makes.
The device copies behind save/restore are covered by the GPU tests."""
import os

import numpy as np
import pytest

import synth
from paper_1805_03981_gb300 import checkpoint as ck


def _mesh():
    return synth.cube_mesh(2, q=1, periodic=True,
                           frames=synth.mesh.random_frames(8, np.random.default_rng(3)))


def _fp(mesh, k=3, coef=None, alpha=1.0, dim=3):
    return ck.fingerprint(dim, k, mesh["nodes"], mesh["nbr"], mesh["nbr_face"], mesh["orient"], coef, alpha)


def test_round_trip(tmp_path):
    rng = np.random.default_rng(0)
    state = rng.standard_normal((8, 4, 64))
    path = str(tmp_path / "a.ckpt")
    meta = {"dim": 3, "k": 3, "n_elem": 8, "prec": 1, "t": 0.125, "step": 13, "fingerprint": "x",
            "extra": {"dt": 0.01, "method": "ader"}}
    ck.write(path, state, meta)
    back, m = ck.read(path)
    assert back.dtype == np.float64 and np.array_equal(back, state)
    assert m["t"] == 0.125 and m["step"] == 13 and m["extra"]["method"] == "ader"
    assert m["format"] == ck.FORMAT
    assert os.listdir(tmp_path) == ["a.ckpt"]  # no temporary file left behind


def test_overwrite_keeps_latest(tmp_path):
    path = str(tmp_path / "b.ckpt")
    meta = {"dim": 2, "k": 1, "n_elem": 2, "prec": 0, "t": 0.0, "step": 0, "fingerprint": "x"}
    ck.write(path, np.zeros((2, 3, 4)), meta)
    ck.write(path, np.ones((2, 3, 4)), dict(meta, step=5))
    s, m = ck.read(path)
    assert m["step"] == 5 and np.all(s == 1.0)


def test_fingerprint_sees_every_input():
    mesh = _mesh()
    base = _fp(mesh)
    assert base == _fp(mesh)
    assert _fp(mesh, k=4) != base
    assert _fp(mesh, dim=2) != base
    assert _fp(mesh, alpha=0.0) != base
    n = mesh["nodes"].copy()
    n[3, 2, 1] += 1e-15
    assert _fp(dict(mesh, nodes=n)) != base
    for key in ("nbr", "nbr_face", "orient"):
        a = mesh[key].copy()
        a[0, 0] ^= 1
        assert _fp(dict(mesh, **{key: a})) != base, key
    rho = np.ones(8 * 64)
    c = np.ones(8 * 64)
    with_coef = _fp(mesh, coef=(rho, c))
    assert with_coef != base
    c2 = c.copy()
    c2[100] = 1.0 + 2.0 ** -52
    assert _fp(mesh, coef=(rho, c2)) != with_coef


def test_read_rejects_bad_files(tmp_path):
    bad = tmp_path / "junk.ckpt"
    bad.write_bytes(b"not an archive")
    with pytest.raises(ValueError):
        ck.read(str(bad))
    path = str(tmp_path / "shape.ckpt")
    meta = {"dim": 3, "k": 3, "n_elem": 8, "prec": 0, "t": 0.0, "step": 0, "fingerprint": "x"}
    ck.write(path, np.zeros((8, 4, 27)), meta)  # (k+1)^3 = 64 nodes expected
    with pytest.raises(ValueError):
        ck.read(path)
    full = open(path, "rb").read()
    trunc = tmp_path / "trunc.ckpt"
    trunc.write_bytes(full[: len(full) // 2])
    with pytest.raises(ValueError):
        ck.read(str(trunc))


class _FakeSolver:
    """Stands in for a Solver on the host: the same attributes the
    checkpoint module reads, and host get/set_state."""
    _DIM = 3

    def __init__(self, mesh, k, alpha=1.0):
        self.k, self.E, self.prec, self.alpha = k, mesh["n_elem"], 0, alpha
        self._nodes, self._nbr, self._nbf, self._ori = mesh["nodes"], mesh["nbr"], mesh["nbr_face"], mesh["orient"]
        self.dev = None

    def get_state(self, U):
        return np.array(U, np.float64)

    def set_state(self, host, U=None):
        self.dev = np.array(host)
        return self.dev


def test_save_restore_checks_problem(tmp_path):
    mesh = _mesh()
    s = _FakeSolver(mesh, 2)
    U = np.random.default_rng(1).standard_normal((8, 4, 27))
    path = str(tmp_path / "c.ckpt")
    ck.save(path, s, U, t=0.5, step=7, extra={"dt": 0.01})
    V, t, step, meta = ck.restore(path, s)
    assert np.array_equal(V, U) and t == 0.5 and step == 7 and meta["extra"]["dt"] == 0.01
    other = _FakeSolver(mesh, 2, alpha=0.0)  # same shapes, another flux
    with pytest.raises(ValueError):
        ck.restore(path, other)
    V, *_ = ck.restore(path, other, check=False)
    assert np.array_equal(V, U)
    with pytest.raises(ValueError):
        ck.restore(path, _FakeSolver(mesh, 3))
