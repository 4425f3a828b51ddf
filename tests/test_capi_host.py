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


def _setup_rc(lib, mesh, dim=3):
    """dg_mesh_setup's (or dg_mesh_setup_2d's) status for a mesh; a context
    it returns (a valid mesh on a machine with a GPU) is destroyed."""
    keep = [np.ascontiguousarray(mesh["nodes"], np.float64), np.ascontiguousarray(mesh["nbr"], np.int32),
            np.ascontiguousarray(mesh["nbr_face"], np.int8), np.ascontiguousarray(mesh["orient"], np.int8)]
    ptrs = (keep[0].ctypes.data_as(C.POINTER(C.c_double)), keep[1].ctypes.data_as(C.POINTER(C.c_int32)),
            keep[2].ctypes.data_as(C.POINTER(C.c_int8)), keep[3].ctypes.data_as(C.POINTER(C.c_int8)))
    ctx = C.c_void_p()
    if dim == 3:
        d = _lib.MeshDesc(mesh["n_elem"], mesh["geom_degree"], *ptrs)
        rc = lib.dg_mesh_setup(C.byref(d), 2, 0, 1.0, 0, C.byref(ctx))
    else:
        d = _lib.MeshDesc2D(mesh["n_elem"], mesh["geom_degree"], *ptrs)
        rc = lib.dg_mesh_setup_2d(C.byref(d), 2, 0, 1.0, None, None, 0, C.byref(ctx))
    if rc == 0:
        lib.dg_destroy(ctx)
    else:
        assert not ctx.value
    return rc


@pytest.mark.parametrize("dim", [3, 2])
def test_mesh_validation_fuzz(lib, dim):
    """Seeded random corruptions of a periodic mesh with rotated element
    frames: out-of-range neighbours, faces and orientation codes, broken
    reciprocity, swapped entries.  Set-up must reject each one cleanly
    (DG_EMESH, with a message) or, where a corruption happens to leave a
    consistent mesh, accept it (on a machine without a GPU: DG_ECUDA); it
    never crashes and never returns a context on error."""
    rng = np.random.default_rng(11 + dim)
    if dim == 3:
        base = synth.cube_mesh(3, q=1, periodic=True, frames=synth.mesh.random_frames(27, rng))
        nf, no = 6, 8
    else:
        from synth import mesh2d
        base = mesh2d.square_mesh(4, q=1, periodic=True, frames=mesh2d.random_frames_2d(16, rng))
        nf, no = 4, 2
    E = base["n_elem"]
    assert _setup_rc(lib, base, dim) in (0, -3)          # the uncorrupted mesh is consistent
    seen = set()
    for trial in range(300):
        m = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in base.items()}
        e, f = int(rng.integers(E)), int(rng.integers(nf))
        kind = trial % 5
        if kind == 0:
            m["nbr"][e, f] = int(rng.integers(-3, E + 3))
        elif kind == 1:
            m["nbr_face"][e, f] = int(rng.integers(-2, nf + 3))
        elif kind == 2:
            m["orient"][e, f] = int(rng.integers(-2, no + 3))
        elif kind == 3:
            e2, f2 = int(rng.integers(E)), int(rng.integers(nf))
            m["nbr"][e, f], m["nbr"][e2, f2] = m["nbr"][e2, f2], m["nbr"][e, f]
        else:
            m["nbr"][e, f] = -1                          # a wall on one side only
        rc = _setup_rc(lib, m, dim)
        assert rc in (-7, 0, -3), (trial, kind, rc)
        if rc == -7:
            assert lib.dg_last_error(None)
        seen.add(rc)
    assert -7 in seen


def test_header_and_library_from_plain_c(lib, tmp_path):
    """include/dg.h compiles as C99 and libdg.so links into a C program,
    whose GPU-free calls behave as documented (tests/c/abi_check.c)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(dgw.library_path())
    exe = str(tmp_path / "abi_check")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c", "abi_check.c"), "-L", libdir, "-ldg",
                        "-Wl,-rpath," + libdir, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c abi ok" in r.stdout
