"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/dg.h declares, and rejects bad meshes and arguments
before touching a device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import synth
import paper_1805_03981_gb300 as dgw
from paper_1805_03981_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(dgw.library_path()):
        import __graft_entry__
        __graft_entry__.build()
    return dgw.load_library()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    assert sorted(names) == sorted(_lib.EXPORTED_SYMBOLS)
    for n in names:
        assert hasattr(lib, n), n


def test_strerror(lib):
    assert lib.dg_strerror(0) == b"ok"
    assert lib.dg_strerror(-7) == b"invalid mesh"


def _desc(mesh):
    keep = [np.ascontiguousarray(mesh["nodes"], np.float64), np.ascontiguousarray(mesh["nbr"], np.int32),
            np.ascontiguousarray(mesh["nbr_face"], np.int8), np.ascontiguousarray(mesh["orient"], np.int8)]
    d = _lib.MeshDesc(mesh["n_elem"], mesh["geom_degree"],
                      keep[0].ctypes.data_as(C.POINTER(C.c_double)),
                      keep[1].ctypes.data_as(C.POINTER(C.c_int32)),
                      keep[2].ctypes.data_as(C.POINTER(C.c_int8)),
                      keep[3].ctypes.data_as(C.POINTER(C.c_int8)))
    return d, keep


@pytest.mark.parametrize("corrupt", ["range", "reciprocity", "orient", "face"])
def test_mesh_validation_rejects(lib, corrupt):
    mesh = synth.cube_mesh(2, q=1, periodic=True,
                           frames=synth.mesh.random_frames(8, np.random.default_rng(1)))
    if corrupt == "range":
        mesh["nbr"][3, 2] = 99
    elif corrupt == "reciprocity":
        mesh["nbr"][0, 1] = 0 if mesh["nbr"][0, 1] != 0 else 1
    elif corrupt == "orient":
        e, f = 0, 0
        mesh["orient"][e, f] = (mesh["orient"][e, f] + 1) % 8
    else:
        mesh["nbr_face"][0, 0] = 7
    d, keep = _desc(mesh)
    ctx = C.c_void_p()
    rc = lib.dg_mesh_setup(C.byref(d), 2, 0, 1.0, 0, C.byref(ctx))
    assert rc == -7, rc
    assert not ctx.value
    assert lib.dg_last_error(None)


def test_argument_validation(lib):
    mesh = synth.cube_mesh(2, q=1, periodic=True)
    d, keep = _desc(mesh)
    ctx = C.c_void_p()
    assert lib.dg_mesh_setup(C.byref(d), 9, 0, 1.0, 0, C.byref(ctx)) == -4     # degree
    assert lib.dg_mesh_setup(C.byref(d), 2, 5, 1.0, 0, C.byref(ctx)) == -1     # precision
    assert lib.dg_mesh_setup(C.byref(d), 2, 0, 1.5, 0, C.byref(ctx)) == -1     # alpha
    assert lib.dg_mesh_setup(None, 2, 0, 1.0, 0, C.byref(ctx)) == -1
    assert lib.dg_apply_operator(None, None, None, 0) == -1
    assert lib.dg_get_state(None, None, None, 0) == -1
    assert lib.dg_set_state(None, None, None, 0) == -1
    lib.dg_destroy(None)  # NULL-safe
