"""Partitioned solve: one mesh split into parts with ghost elements.

A part holds its owned elements followed by ghosts: copies of the elements
that neighbour an owned element across a face and belong to another part.
The operator of an owned element reads its neighbours' states across every
face (Sec. 2.4), so before each operator application the ghosts of its input
are refreshed from their owners; the ADER predictor is element-local, so an
ADER step needs one such exchange and an LSRK step five (Sec. 4.1, 4.8).

``split`` is host logic only (numpy): the parts' local meshes and the
exchange plan.  ``Partitioned`` runs all parts on this device through the
C ABI (dg_set_owned, dg_part_*): the exchange is one gather kernel.  The same
plan drives a multi-process exchange (one rank per part), see ``send_lists``.
"""
import ctypes as C

import numpy as np

from . import _lib


def split(mesh, P, rho=None, c=None):
    """Split a mesh into P parts of contiguous element ranges.

    Returns a list of dicts, one per part:
      mesh      local mesh (owned elements first, then ghosts, sorted by
                global index within each group); ghosts keep their faces
                towards elements present in the part, walls elsewhere
      owned     global indices of the owned elements
      ghost     global indices of the ghosts
      src_part, src_elem   owning part of each ghost and its owned index there
      rho, c    the local coefficients (if given)
    """
    E = int(mesh["n_elem"])
    if not 1 <= P <= E:
        raise ValueError("need 1 <= P <= number of elements")
    nbr = np.asarray(mesh["nbr"], np.int64)
    bounds = [E * p // P for p in range(P + 1)]
    part_of = np.empty(E, np.int64)
    for p in range(P):
        part_of[bounds[p]:bounds[p + 1]] = p
    parts = []
    for p in range(P):
        lo, hi = bounds[p], bounds[p + 1]
        owned = np.arange(lo, hi)
        nb = nbr[owned].ravel()
        nb = nb[nb >= 0]
        ghost = np.unique(nb[(nb < lo) | (nb >= hi)])
        elems = np.concatenate([owned, ghost])
        local = np.full(E, -1, np.int64)
        local[elems] = np.arange(elems.size)
        gl = nbr[elems]
        lnbr = np.where(gl >= 0, local[np.maximum(gl, 0)], -1)
        present = lnbr >= 0
        lmesh = {
            "n_elem": int(elems.size),
            "geom_degree": int(mesh["geom_degree"]),
            "nodes": np.ascontiguousarray(np.asarray(mesh["nodes"])[elems]),
            "nbr": np.ascontiguousarray(lnbr.astype(np.int32)),
            "nbr_face": np.ascontiguousarray(np.where(present, np.asarray(mesh["nbr_face"])[elems], -1).astype(np.int8)),
            "orient": np.ascontiguousarray(np.where(present, np.asarray(mesh["orient"])[elems], 0).astype(np.int8)),
        }
        part = {"mesh": lmesh, "owned": owned, "ghost": ghost,
                "src_part": part_of[ghost], "src_elem": ghost - np.asarray(bounds)[part_of[ghost]]}
        if rho is not None:
            part["rho"] = np.ascontiguousarray(np.asarray(rho)[elems])
            part["c"] = np.ascontiguousarray(np.asarray(c)[elems])
        parts.append(part)
    return parts


def send_lists(parts):
    """For a one-rank-per-part exchange: sends[p][q] = owned indices of part p
    whose tiles part q needs, in q's ghost order (empty where q needs none)."""
    P = len(parts)
    sends = [[np.zeros(0, np.int64) for _ in range(P)] for _ in range(P)]
    for q, part in enumerate(parts):
        for p in range(P):
            sel = part["src_part"] == p
            sends[p][q] = part["src_elem"][sel]
    return sends


def recv_slots(parts):
    """recv[q][p] = ghost slots of part q (0-based within its ghosts) filled
    from part p, in the order send_lists sends them."""
    P = len(parts)
    return [[np.nonzero(parts[q]["src_part"] == p)[0] for p in range(P)] for q in range(P)]


class Partitioned:
    """One solve split into P parts on the current device (include/dg.h,
    dg_part_*).  State tensors are per part: owned elements then ghosts."""

    def __init__(self, mesh, k, P, prec=_lib.DG_FP64, alpha=1.0, rho=None, c=None, basis=_lib.BASIS_GL):
        self.parts = split(mesh, P, rho, c)
        self.E = int(mesh["n_elem"])
        self.solvers = []
        for part in self.parts:
            s = _lib.Solver(part["mesh"], k, prec, alpha, part.get("rho"), part.get("c"))
            s.set_owned(part["owned"].size)
            s.set_basis(basis)
            self.solvers.append(s)
        self.lib = self.solvers[0].lib
        self.t = None

    def to_device(self, U_global):
        """Per-part device states from a global [E][4][n^3] host array; the
        parts are then bound to these states."""
        U_global = np.asarray(U_global)
        states = []
        for part, s in zip(self.parts, self.solvers):
            states.append(s.to_device(np.concatenate([U_global[part["owned"]], U_global[part["ghost"]]])))
        self.bind(states)
        return states

    def bind(self, states):
        if self.t is not None:
            self.lib.dg_part_destroy(self.t)
            self.t = None
        self.states = list(states)
        P = len(self.parts)
        ctxs = (C.c_void_p * P)(*[s.ctx.value for s in self.solvers])
        ptrs = (C.c_void_p * P)(*[s._state(u).value for s, u in zip(self.solvers, self.states)])
        ng = (C.c_int32 * P)(*[int(p["ghost"].size) for p in self.parts])
        sp = np.ascontiguousarray(np.concatenate([p["src_part"] for p in self.parts]).astype(np.int32))
        se = np.ascontiguousarray(np.concatenate([p["src_elem"] for p in self.parts]).astype(np.int32))
        t = C.c_void_p()
        rc = self.lib.dg_part_create(ctxs, ptrs, P, ng, sp.ctypes.data_as(C.POINTER(C.c_int32)),
                                     se.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(t))
        if rc != 0:
            raise _lib.DGError(rc, self.lib.dg_last_error(None).decode())
        self.t = t

    def _check(self, rc):
        if rc != 0:
            raise _lib.DGError(rc, self.lib.dg_part_last_error(self.t).decode())

    def step_lsrk(self, dt, nsteps, stream=None):
        self._check(self.lib.dg_part_step_lsrk(self.t, float(dt), int(nsteps), _lib._stream(stream)))

    def step_ader(self, dt, nsteps, reduce_every=2, stream=None):
        self._check(self.lib.dg_part_step_ader(self.t, float(dt), int(nsteps), int(reduce_every),
                                               _lib._stream(stream)))

    def step_hdg_ader(self, dt, nsteps, reduce_every=2, stream=None):
        self._check(self.lib.dg_part_step_hdg_ader(self.t, float(dt), int(nsteps), int(reduce_every),
                                                   _lib._stream(stream)))

    def exchange(self, stream=None):
        self._check(self.lib.dg_part_exchange(self.t, _lib._stream(stream)))

    def info(self):
        n, g, x = C.c_int32(), C.c_int32(), C.c_uint64()
        self._check(self.lib.dg_part_info(self.t, C.byref(n), C.byref(g), C.byref(x)))
        return {"parts": n.value, "ghosts": g.value, "exchanges": x.value}

    def gather(self, states=None):
        """The global state [E][4][n^3] (host, float64) from the parts' owned elements."""
        states = self.states if states is None else states
        out = None
        for part, u in zip(self.parts, states):
            a = u[: part["owned"].size].double().cpu().numpy()
            if out is None:
                out = np.empty((self.E,) + a.shape[1:])
            out[part["owned"]] = a
        return out

    def close(self):
        if self.t is not None:
            self.lib.dg_part_destroy(self.t)
            self.t = None
        for s in self.solvers:
            s.close()
