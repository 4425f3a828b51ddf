"""Checkpoint files of a solve, for restart.

Both time integrators of the paper are one-step methods (Sec. 2.2: the LSRK
stages start from U_n alone; Sec. 2.3: the ADER step is built from U_n
alone), so the state between two step calls, with its time and step
count, is everything a solve carries forward.  A restart that loads it into
a context of the same mesh, degree, coefficients and flux gives, bit for
bit, what the same step calls give without the checkpoint, since
FP32 -> FP64 -> FP32 is exact (dg_get_state in include/dg.h).

File format (a NumPy ``.npz`` archive):
  ``state``  float64 [E][fields][npts], the GL-basis state (dg_get_state)
  ``meta``   a JSON string: ``format``, ``dim``, ``k``, ``n_elem``, ``prec``
             (the precision the state was taken in), ``t``, ``step``,
             ``fingerprint`` (SHA-256 over the mesh arrays, the degree and
             the coefficients) and the caller's ``extra`` dictionary.
Files are written to a temporary name beside the target and renamed over
it, so a crash mid-write leaves the previous checkpoint intact.

The device copies are made by the library; this module only hashes,
archives and checks.
"""
import hashlib
import io
import json
import os
import zipfile

import numpy as np

FORMAT = 1


def fingerprint(dim, k, nodes, nbr, nbr_face, orient, coef=None, alpha=None):
    """SHA-256 (hex) identifying the discrete problem a state belongs to."""
    h = hashlib.sha256()
    h.update(("dg-ckpt dim=%d k=%d" % (int(dim), int(k))).encode())
    for name, a, dt in (("nodes", nodes, np.float64), ("nbr", nbr, np.int32),
                        ("nbr_face", nbr_face, np.int8), ("orient", orient, np.int8)):
        a = np.ascontiguousarray(a, dt)
        h.update(("%s%s" % (name, a.shape)).encode())
        h.update(a.tobytes())
    if coef is not None:
        for name, a in zip(("rho", "c"), coef):
            a = np.ascontiguousarray(a, np.float64).reshape(-1)
            h.update(("%s%d" % (name, a.size)).encode())
            h.update(a.tobytes())
    if alpha is not None:
        h.update(np.float64(alpha).tobytes())
    return h.hexdigest()


def solver_fingerprint(solver):
    """fingerprint() of a Solver or Solver2D (its mesh, degree, coefficients
    as last set, and flux parameter)."""
    return fingerprint(solver._DIM, solver.k, solver._nodes, solver._nbr, solver._nbf, solver._ori,
                       getattr(solver, "_coef", None), getattr(solver, "alpha", None))


def write(path, state, meta):
    """Archive a host state and its metadata at ``path`` (atomically)."""
    state = np.ascontiguousarray(state, np.float64)
    meta = dict(meta, format=FORMAT)
    buf = io.BytesIO()
    np.savez(buf, state=state, meta=np.array(json.dumps(meta, sort_keys=True)))
    tmp = "%s.tmp%d" % (path, os.getpid())
    with open(tmp, "wb") as f:
        f.write(buf.getvalue())
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def read(path):
    """(state, meta) from a checkpoint file; ValueError if it is not one."""
    try:
        with np.load(path, allow_pickle=False) as z:
            state = np.array(z["state"])
            meta = json.loads(str(z["meta"]))
    except (OSError, KeyError, ValueError, EOFError, zipfile.BadZipFile) as e:
        raise ValueError("%s is not a readable checkpoint: %s" % (path, e)) from e
    if meta.get("format") != FORMAT:
        raise ValueError("%s: checkpoint format %r, expected %d" % (path, meta.get("format"), FORMAT))
    want = (int(meta["n_elem"]), int(meta["dim"]) + 1, (int(meta["k"]) + 1) ** int(meta["dim"]))
    if state.dtype != np.float64 or state.shape != want:
        raise ValueError("%s: state %s %s, expected float64 %s" % (path, state.dtype, state.shape, want))
    return state, meta


def save(path, solver, U, t, step, extra=None):
    """Write the device state U of ``solver`` at time t after ``step``
    steps.  Returns the metadata written."""
    meta = {"dim": solver._DIM, "k": solver.k, "n_elem": solver.E, "prec": solver.prec,
            "t": float(t), "step": int(step), "fingerprint": solver_fingerprint(solver),
            "extra": dict(extra or {})}
    write(path, solver.get_state(U), meta)
    return meta


def restore(path, solver, U=None, check=True):
    """Load a checkpoint into the device state U of ``solver`` (a new state
    when None).  With ``check`` the file must belong to the same problem
    (ValueError otherwise).  Returns (U, t, step, meta)."""
    state, meta = read(path)
    if (meta["dim"], meta["k"], meta["n_elem"]) != (solver._DIM, solver.k, solver.E):
        raise ValueError("%s: checkpoint of a dim %d, k %d, %d-element mesh; solver is dim %d, k %d, %d elements"
                         % (path, meta["dim"], meta["k"], meta["n_elem"], solver._DIM, solver.k, solver.E))
    if check and meta["fingerprint"] != solver_fingerprint(solver):
        raise ValueError("%s: checkpoint of a different mesh, coefficients or flux" % path)
    U = solver.set_state(state, U)
    return U, meta["t"], meta["step"], meta
