"""ctypes binding of libdg.so (include/dg.h): argument marshalling only."""
import ctypes as C
import os

import numpy as np

DG_FP64, DG_FP32 = 0, 1
_HERE = os.path.dirname(os.path.abspath(__file__))

# every symbol include/dg.h declares
EXPORTED_SYMBOLS = [
    "dg_mesh_setup", "dg_set_coefficients", "dg_apply_operator", "dg_step_lsrk",
    "dg_step_ader", "dg_tck", "dg_energy", "dg_norms", "dg_solve_host", "dg_info",
    "dg_device_bytes", "dg_launch_count", "dg_destroy", "dg_strerror", "dg_last_error",
    "dg_profile_enable", "dg_profile_read", "dg_energy_noalloc",
    "dg_set_tiling", "dg_get_tiling", "dg_tune", "dg_batch_create", "dg_batch_step_ader",
    "dg_batch_step_lsrk", "dg_batch_info", "dg_batch_last_error", "dg_batch_destroy",
    "dg_server_create", "dg_submit", "dg_poll", "dg_server_stats", "dg_server_destroy",
    "dg_request_bytes", "dg_mesh_setup_coef", "dg_set_basis", "dg_get_basis", "dg_check_device",
    "dg_is_affine", "dg_change_basis", "dg_batch_set_basis", "dg_batch_convert",
    "dg_set_owned", "dg_part_create", "dg_part_step_lsrk", "dg_part_step_ader", "dg_part_exchange",
    "dg_part_info", "dg_part_last_error", "dg_part_destroy", "dg_step_hdg_ader", "dg_part_step_hdg_ader",
    "dg_mesh_setup_2d", "dg_get_state", "dg_set_state",
    "dg_set_predictor_kernel", "dg_get_predictor_kernel", "dg_test_expire_waits",
    "dg_set_lsrk_scheme", "dg_get_lsrk_scheme", "dg_probe_fma_peak",
]
LSRK_CK54, LSRK45, LSRK59 = 0, 1, 2
BASIS_GL, BASIS_G = 0, 1
PRED_AUTO, PRED_LINES, PRED_COLUMNS, PRED_GL_PROJECTION, PRED_INTERLEAVED = 0, 1, 2, 3, 4
KIND_LSRK, KIND_ADER, KIND_TCK = 1, 2, 3
KINDS = ["operator", "lsrk_stage", "ader_update", "tck", "other"]


class DGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"dg status {status}: {msg}")
        self.status = status


class MeshDesc(C.Structure):
    _fields_ = [("n_elem", C.c_int32), ("geom_degree", C.c_int32),
                ("nodes", C.POINTER(C.c_double)), ("nbr", C.POINTER(C.c_int32)),
                ("nbr_face", C.POINTER(C.c_int8)), ("orient", C.POINTER(C.c_int8))]


class MeshDesc2D(C.Structure):
    _fields_ = [("n_elem", C.c_int32), ("geom_degree", C.c_int32),
                ("nodes", C.POINTER(C.c_double)), ("nbr", C.POINTER(C.c_int32)),
                ("nbr_face", C.POINTER(C.c_int8)), ("orient", C.POINTER(C.c_int8))]


class ServerOpts(C.Structure):
    _fields_ = [("device", C.c_int32), ("prec", C.c_int32), ("max_active", C.c_int32),
                ("chunk_steps", C.c_int32), ("max_active_dof", C.c_double)]


class Request(C.Structure):
    _fields_ = [("mesh", MeshDesc), ("k", C.c_int32), ("flux_alpha", C.c_double),
                ("rho", C.POINTER(C.c_double)), ("c", C.POINTER(C.c_double)), ("U0", C.c_void_p),
                ("U_out", C.c_void_p), ("dt", C.c_double), ("nsteps", C.c_int32), ("method", C.c_int32),
                ("reduce_every", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("status", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int32), ("active", C.c_int32), ("peak_active", C.c_int32),
                ("completed", C.c_uint64), ("rounds", C.c_uint64), ("batches_built", C.c_uint64),
                ("hbm_used", C.c_size_t), ("hbm_peak", C.c_size_t), ("dof_steps", C.c_double),
                ("busy_s", C.c_double)]


_lib = None


def library_path():
    return os.path.join(_HERE, "libdg.so")


def load_library():
    """Load libdg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with paper_1805_03981_gb300/build.py")
    lib = C.CDLL(path)
    vp, u = C.c_void_p, C.c_size_t
    st = C.c_size_t  # uintptr_t stream
    sig = {
        "dg_mesh_setup": (C.c_int, [C.POINTER(MeshDesc), C.c_int, C.c_int, C.c_double, st, C.POINTER(vp)]),
        "dg_mesh_setup_coef": (C.c_int, [C.POINTER(MeshDesc), C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double),
                                         C.POINTER(C.c_double), st, C.POINTER(vp)]),
        "dg_set_coefficients": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), st]),
        "dg_apply_operator": (C.c_int, [vp, vp, vp, st]),
        "dg_step_lsrk": (C.c_int, [vp, vp, C.c_double, C.c_int32, st]),
        "dg_step_ader": (C.c_int, [vp, vp, C.c_double, C.c_int32, C.c_int32, st]),
        "dg_tck": (C.c_int, [vp, vp, vp, C.c_double, C.c_int32, st]),
        "dg_energy": (C.c_int, [vp, vp, C.POINTER(C.c_double), st]),
        "dg_norms": (C.c_int, [vp, vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_double), st]),
        "dg_solve_host": (C.c_int, [vp, C.c_int, vp, vp, C.c_double, C.c_int32, C.c_int32, st]),
        "dg_info": (C.c_int, [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                              C.POINTER(u)]),
        "dg_device_bytes": (u, [vp]),
        "dg_launch_count": (C.c_uint64, [vp]),
        "dg_destroy": (None, [vp]),
        "dg_strerror": (C.c_char_p, [C.c_int]),
        "dg_profile_enable": (C.c_int, [vp, C.c_int]),
        "dg_energy_noalloc": (C.c_int, [vp, vp, vp, st]),
        "dg_set_tiling": (C.c_int, [vp, C.c_int32, C.c_int32]),
        "dg_get_tiling": (C.c_int, [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "dg_tune": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int32), C.c_int32, C.c_int32,
                              C.POINTER(C.c_double), st]),
        "dg_batch_create": (C.c_int, [C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_double), C.c_int32, st,
                                      C.POINTER(vp)]),
        "dg_batch_step_ader": (C.c_int, [vp, C.c_int32, C.c_int32, st]),
        "dg_batch_step_lsrk": (C.c_int, [vp, C.c_int32, st]),
        "dg_batch_info": (C.c_int, [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int32), C.POINTER(C.c_uint64)]),
        "dg_batch_last_error": (C.c_char_p, [vp]),
        "dg_batch_destroy": (None, [vp]),
        "dg_server_create": (C.c_int, [C.c_size_t, C.POINTER(ServerOpts), C.POINTER(vp)]),
        "dg_submit": (C.c_int, [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
        "dg_poll": (C.c_int, [vp, C.c_uint64, C.POINTER(Result), C.c_int32]),
        "dg_server_stats": (C.c_int, [vp, C.POINTER(ServerStats)]),
        "dg_server_destroy": (None, [vp]),
        "dg_request_bytes": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
        "dg_set_basis": (C.c_int, [vp, C.c_int]),
        "dg_check_device": (C.c_int, [vp, st]),
        "dg_test_expire_waits": (C.c_int, [vp, C.c_int32]),
        "dg_set_lsrk_scheme": (C.c_int, [vp, C.c_int32]),
        "dg_get_lsrk_scheme": (C.c_int, [vp]),
        "dg_probe_fma_peak": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_double), st]),
        "dg_is_affine": (C.c_int, [vp]),
        "dg_change_basis": (C.c_int, [vp, vp, C.c_int, st]),
        "dg_batch_set_basis": (C.c_int, [vp, C.c_int, C.c_int]),
        "dg_batch_convert": (C.c_int, [vp, C.c_int, st]),
        "dg_get_basis": (C.c_int, [vp]),
        "dg_profile_read": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int]),
        "dg_last_error": (C.c_char_p, [vp]),
        "dg_set_owned": (C.c_int, [vp, C.c_int32]),
        "dg_mesh_setup_2d": (C.c_int, [C.POINTER(MeshDesc2D), C.c_int, C.c_int, C.c_double,
                                       C.POINTER(C.c_double), C.POINTER(C.c_double), st, C.POINTER(vp)]),
        "dg_step_hdg_ader": (C.c_int, [vp, vp, C.c_double, C.c_int32, C.c_int32, st]),
        "dg_part_step_hdg_ader": (C.c_int, [vp, C.c_double, C.c_int32, C.c_int32, st]),
        "dg_part_create": (C.c_int, [C.POINTER(vp), C.POINTER(vp), C.c_int32, C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(vp)]),
        "dg_part_step_lsrk": (C.c_int, [vp, C.c_double, C.c_int32, st]),
        "dg_part_step_ader": (C.c_int, [vp, C.c_double, C.c_int32, C.c_int32, st]),
        "dg_part_exchange": (C.c_int, [vp, st]),
        "dg_part_info": (C.c_int, [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_uint64)]),
        "dg_part_last_error": (C.c_char_p, [vp]),
        "dg_part_destroy": (None, [vp]),
        "dg_get_state": (C.c_int, [vp, vp, C.POINTER(C.c_double), st]),
        "dg_set_state": (C.c_int, [vp, C.POINTER(C.c_double), vp, st]),
        "dg_set_predictor_kernel": (C.c_int, [vp, C.c_int]),
        "dg_get_predictor_kernel": (C.c_int, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x):
    return C.c_void_p(x.data_ptr())


def probe_fma_peak(prec, iters=4096, stream=None):
    """Measured FMA-pipe peak (TFLOP/s) of the current device (dg_probe_fma_peak)."""
    lib = load_library()
    v = C.c_double()
    rc = lib.dg_probe_fma_peak(int(prec), int(iters), C.byref(v), _stream(stream))
    if rc != 0:
        raise DGError(rc, "dg_probe_fma_peak failed")
    return v.value


class Solver:
    """One mesh, degree and precision on the current CUDA device.

    mesh: dict with ``n_elem``, ``geom_degree``, ``nodes`` [E,(q+1)^3,3],
    ``nbr``, ``nbr_face``, ``orient`` [E,6] (see include/dg.h).
    States are torch CUDA tensors [E, 4, (k+1)^3] of the solver's dtype.
    """

    def __init__(self, mesh, k, prec=DG_FP64, alpha=1.0, rho=None, c=None, stream=None):
        import torch
        self.lib = load_library()
        self.k, self.n, self.prec = int(k), int(k) + 1, int(prec)
        self.alpha = float(alpha)
        self.E = int(mesh["n_elem"])
        self.dtype = torch.float64 if self.prec == DG_FP64 else torch.float32
        self.device = torch.cuda.current_device()
        self._nodes = np.ascontiguousarray(mesh["nodes"], np.float64)
        self._nbr = np.ascontiguousarray(mesh["nbr"], np.int32)
        self._nbf = np.ascontiguousarray(mesh["nbr_face"], np.int8)
        self._ori = np.ascontiguousarray(mesh["orient"], np.int8)
        desc = MeshDesc(self.E, int(mesh["geom_degree"]),
                        self._nodes.ctypes.data_as(C.POINTER(C.c_double)),
                        self._nbr.ctypes.data_as(C.POINTER(C.c_int32)),
                        self._nbf.ctypes.data_as(C.POINTER(C.c_int8)),
                        self._ori.ctypes.data_as(C.POINTER(C.c_int8)))
        ctx = C.c_void_p()
        rc = self.lib.dg_mesh_setup(C.byref(desc), self.k, self.prec, float(alpha),
                                    _stream(stream), C.byref(ctx))
        if rc != 0:
            raise DGError(rc, self.lib.dg_last_error(None).decode())
        self.ctx = ctx
        if rho is not None or c is not None:
            self.set_coefficients(rho, c, stream)

    def _check(self, rc):
        if rc != 0:
            raise DGError(rc, self.lib.dg_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.dg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- state helpers -------------------------------------------------
    _FIELDS, _DIM = 4, 3

    def _state_shape(self):
        return (self.E, self._FIELDS, self.n ** self._DIM)

    def empty_state(self):
        import torch
        return torch.empty(self._state_shape(), dtype=self.dtype, device="cuda")

    def to_device(self, U):
        import torch
        return torch.as_tensor(np.ascontiguousarray(U)).to(device="cuda", dtype=self.dtype).contiguous()

    def _state(self, U):
        import torch
        if not (isinstance(U, torch.Tensor) and U.is_cuda and U.dtype == self.dtype and U.is_contiguous()
                and U.numel() == int(np.prod(self._state_shape()))):
            raise DGError(-1, "state must be a contiguous CUDA tensor %s of the solver dtype"
                          % (list(self._state_shape()),))
        return _ptr(U)

    # --- C ABI calls ------------------------------------------------------
    def set_coefficients(self, rho, c, stream=None):
        rho = np.ascontiguousarray(rho, np.float64).reshape(-1)
        c = np.ascontiguousarray(c, np.float64).reshape(-1)
        self._coef = (rho.copy(), c.copy())
        self._check(self.lib.dg_set_coefficients(
            self.ctx, rho.ctypes.data_as(C.POINTER(C.c_double)),
            c.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)))

    def apply(self, U, R=None, stream=None):
        R = self.empty_state() if R is None else R
        self._check(self.lib.dg_apply_operator(self.ctx, self._state(U), self._state(R), _stream(stream)))
        return R

    def step_lsrk(self, U, dt, nsteps, stream=None):
        self._check(self.lib.dg_step_lsrk(self.ctx, self._state(U), float(dt), int(nsteps), _stream(stream)))
        return U

    def step_ader(self, U, dt, nsteps, reduce_every=2, stream=None):
        self._check(self.lib.dg_step_ader(self.ctx, self._state(U), float(dt), int(nsteps),
                                          int(reduce_every), _stream(stream)))
        return U

    def step_hdg_ader(self, U, dt, nsteps, reduce_every=2, stream=None):
        """HDG-ADER steps (Eq. hdg-ader), U updated in place."""
        self._check(self.lib.dg_step_hdg_ader(self.ctx, self._state(U), float(dt), int(nsteps),
                                              int(reduce_every), _stream(stream)))
        return U

    def tck(self, U, dt, reduce_every=2, out=None, stream=None):
        out = self.empty_state() if out is None else out
        self._check(self.lib.dg_tck(self.ctx, self._state(U), self._state(out), float(dt),
                                    int(reduce_every), _stream(stream)))
        return out

    def energy(self, U, stream=None):
        v = C.c_double()
        self._check(self.lib.dg_energy(self.ctx, self._state(U), C.byref(v), _stream(stream)))
        return v.value

    def energy_noalloc(self, U, out, stream=None):
        """Energy into the device double ``out`` (a float64 CUDA tensor on
        this solver's device) without any allocation by the library; see
        include/dg.h."""
        import torch
        if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64
                and out.numel() >= 1 and out.device.index == self.device):
            raise DGError(-1, "out must be a float64 CUDA tensor on device %d" % self.device)
        self._check(self.lib.dg_energy_noalloc(self.ctx, self._state(U), _ptr(out), _stream(stream)))
        return out

    def energy_noalloc_raw(self, U, out_ptr, stream=None):
        """dg_energy_noalloc with an unchecked address (tests of the C
        library's own argument checks)."""
        return int(self.lib.dg_energy_noalloc(self.ctx, self._state(U), C.c_void_p(out_ptr), _stream(stream)))

    def norms(self, A, B=None, stream=None):
        aa, dd = C.c_double(), C.c_double()
        self._check(self.lib.dg_norms(self.ctx, self._state(A), None if B is None else self._state(B),
                                      C.byref(aa), C.byref(dd), _stream(stream)))
        return aa.value, dd.value

    def solve_host(self, method, U_host, U_out_host, dt, nsteps, reduce_every=2, stream=None):
        """method 0 = LSRK, 1 = ADER; host buffers (torch CPU tensors, ideally pinned)."""
        self._check(self.lib.dg_solve_host(self.ctx, int(method), _ptr(U_host), _ptr(U_out_host),
                                           float(dt), int(nsteps), int(reduce_every), _stream(stream)))
        return U_out_host

    def get_state(self, U, stream=None):
        """The device state U as a new FP64 host array (dg_get_state)."""
        out = np.empty(self._state_shape(), np.float64)
        self._check(self.lib.dg_get_state(self.ctx, self._state(U), out.ctypes.data_as(C.POINTER(C.c_double)),
                                          _stream(stream)))
        return out

    def set_state(self, host, U=None, stream=None):
        """Copy an FP64 host array into the device state U (a new one when
        None) with dg_set_state; returns U."""
        host = np.ascontiguousarray(host, np.float64)
        if host.size != int(np.prod(self._state_shape())):
            raise DGError(-1, "host state must have %d entries" % int(np.prod(self._state_shape())))
        U = self.empty_state() if U is None else U
        self._check(self.lib.dg_set_state(self.ctx, host.ctypes.data_as(C.POINTER(C.c_double)),
                                          self._state(U), _stream(stream)))
        return U

    def info(self):
        E, k, p, b = C.c_int32(), C.c_int32(), C.c_int32(), C.c_size_t()
        self._check(self.lib.dg_info(self.ctx, C.byref(E), C.byref(k), C.byref(p), C.byref(b)))
        return {"n_elem": E.value, "k": k.value, "prec": p.value, "state_bytes": b.value}

    def profile(self, enable=True):
        self._check(self.lib.dg_profile_enable(self.ctx, int(bool(enable))))

    def profile_read(self, reset=True):
        """{kind: (total_ms, launches)} since the last reset."""
        ms = (C.c_double * len(KINDS))()
        cnt = (C.c_int64 * len(KINDS))()
        self._check(self.lib.dg_profile_read(self.ctx, ms, cnt, int(bool(reset))))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KINDS)}

    def check_device(self, stream=None):
        """Raise DGError(DG_ETIMEOUT) if a bounded device wait gave up."""
        self._check(self.lib.dg_check_device(self.ctx, _stream(stream)))

    def set_lsrk_scheme(self, scheme):
        """LSRK_CK54 (default), LSRK45 or LSRK59 for step_lsrk (dg_set_lsrk_scheme)."""
        self._check(self.lib.dg_set_lsrk_scheme(self.ctx, int(scheme)))

    def lsrk_scheme(self):
        return int(self.lib.dg_get_lsrk_scheme(self.ctx))

    def test_expire_waits(self, on=True):
        """Testing only: the first bounded wait of the staged FP32 operators
        gives up at once (dg_test_expire_waits)."""
        self._check(self.lib.dg_test_expire_waits(self.ctx, int(bool(on))))

    def change_basis(self, U, to_g, stream=None):
        self._check(self.lib.dg_change_basis(self.ctx, self._state(U), int(bool(to_g)), _stream(stream)))
        return U

    def is_affine(self):
        return bool(self.lib.dg_is_affine(self.ctx))

    def set_owned(self, n_owned):
        """Step only the first n_owned elements (the rest are ghosts of a part)."""
        self._check(self.lib.dg_set_owned(self.ctx, int(n_owned)))

    def set_basis(self, basis):
        """BASIS_GL (paper's storage, default) or BASIS_G (Gauss values inside the steppers)."""
        self._check(self.lib.dg_set_basis(self.ctx, int(basis)))

    def set_predictor_kernel(self, kind):
        """PRED_AUTO, PRED_LINES, PRED_COLUMNS or PRED_GL_PROJECTION (include/dg.h)."""
        self._check(self.lib.dg_set_predictor_kernel(self.ctx, int(kind)))

    def predictor_kernel(self):
        return int(self.lib.dg_get_predictor_kernel(self.ctx))

    def basis(self):
        return int(self.lib.dg_get_basis(self.ctx))

    def set_tiling(self, epb_op=0, epb_tck=0):
        self._check(self.lib.dg_set_tiling(self.ctx, int(epb_op), int(epb_tck)))

    def tiling(self):
        a, b = C.c_int32(), C.c_int32()
        self._check(self.lib.dg_get_tiling(self.ctx, C.byref(a), C.byref(b)))
        return a.value, b.value

    def tune(self, kind, candidates, reps=3, stream=None):
        """Per-candidate ms per launch of one kernel kind; leaves the best set."""
        cand = (C.c_int32 * len(candidates))(*candidates)
        ms = (C.c_double * len(candidates))()
        self._check(self.lib.dg_tune(self.ctx, int(kind), cand, len(candidates), int(reps), ms,
                                     _stream(stream)))
        return list(ms)

    def device_bytes(self):
        return int(self.lib.dg_device_bytes(self.ctx))

    def launch_count(self):
        return int(self.lib.dg_launch_count(self.ctx))


class Solver2D(Solver):
    """A 2D mesh of quadrilaterals (include/dg.h, dg_mesh_setup_2d).

    mesh: dict with ``n_elem``, ``geom_degree``, ``nodes`` [E,(q+1)^2,2],
    ``nbr``, ``nbr_face``, ``orient`` [E,4] (see ``synth.mesh2d``).  States
    are torch CUDA tensors [E, 3, (k+1)^2]; the steppers work in the Gauss
    basis (the only basis a 2D context takes)."""

    _FIELDS, _DIM = 3, 2

    def __init__(self, mesh, k, prec=DG_FP64, alpha=1.0, rho=None, c=None, stream=None):
        import torch
        self.lib = load_library()
        self.k, self.n, self.prec = int(k), int(k) + 1, int(prec)
        self.alpha = float(alpha)
        self.E = int(mesh["n_elem"])
        self.dtype = torch.float64 if self.prec == DG_FP64 else torch.float32
        self.device = torch.cuda.current_device()
        self._nodes = np.ascontiguousarray(mesh["nodes"], np.float64)
        self._nbr = np.ascontiguousarray(mesh["nbr"], np.int32)
        self._nbf = np.ascontiguousarray(mesh["nbr_face"], np.int8)
        self._ori = np.ascontiguousarray(mesh["orient"], np.int8)
        desc = MeshDesc2D(self.E, int(mesh["geom_degree"]),
                          self._nodes.ctypes.data_as(C.POINTER(C.c_double)),
                          self._nbr.ctypes.data_as(C.POINTER(C.c_int32)),
                          self._nbf.ctypes.data_as(C.POINTER(C.c_int8)),
                          self._ori.ctypes.data_as(C.POINTER(C.c_int8)))
        rho_p = c_p = None
        if rho is not None:
            self._rho = np.ascontiguousarray(rho, np.float64).reshape(-1)
            self._c = np.ascontiguousarray(c, np.float64).reshape(-1)
            self._coef = (self._rho.copy(), self._c.copy())
            rho_p = self._rho.ctypes.data_as(C.POINTER(C.c_double))
            c_p = self._c.ctypes.data_as(C.POINTER(C.c_double))
        ctx = C.c_void_p()
        rc = self.lib.dg_mesh_setup_2d(C.byref(desc), self.k, self.prec, float(alpha), rho_p, c_p,
                                       _stream(stream), C.byref(ctx))
        if rc != 0:
            raise DGError(rc, self.lib.dg_last_error(None).decode())
        self.ctx = ctx


class Batch:
    """Independent solves advanced together (include/dg.h, dg_batch_*).

    solvers: list of Solver (one precision); states: matching CUDA tensors
    (kept alive by the batch); dts: time steps."""

    def __init__(self, solvers, states, dts, stream=None):
        self.lib = load_library()
        self.solvers, self.states = list(solvers), list(states)
        n = len(self.solvers)
        ctxs = (C.c_void_p * n)(*[s.ctx.value for s in self.solvers])
        ptrs = (C.c_void_p * n)(*[s._state(u).value for s, u in zip(self.solvers, self.states)])
        dt = (C.c_double * n)(*[float(x) for x in dts])
        b = C.c_void_p()
        rc = self.lib.dg_batch_create(ctxs, ptrs, dt, n, _stream(stream), C.byref(b))
        if rc != 0:
            raise DGError(rc, self.lib.dg_last_error(None).decode())
        self.b = b

    def _check(self, rc):
        if rc != 0:
            raise DGError(rc, self.lib.dg_batch_last_error(self.b).decode())

    def set_basis(self, basis, convert_each_call=True):
        self._check(self.lib.dg_batch_set_basis(self.b, int(basis), int(bool(convert_each_call))))

    def convert(self, to_g, stream=None):
        self._check(self.lib.dg_batch_convert(self.b, int(bool(to_g)), _stream(stream)))

    def step_ader(self, nsteps, reduce_every=2, stream=None):
        self._check(self.lib.dg_batch_step_ader(self.b, int(nsteps), int(reduce_every), _stream(stream)))

    def step_lsrk(self, nsteps, stream=None):
        self._check(self.lib.dg_batch_step_lsrk(self.b, int(nsteps), _stream(stream)))

    def info(self):
        vals = [C.c_int32() for _ in range(4)] + [C.c_uint64()]
        self._check(self.lib.dg_batch_info(self.b, *[C.byref(v) for v in vals]))
        return dict(zip(["instances", "items", "block", "grid", "launches"], [v.value for v in vals]))

    def close(self):
        if getattr(self, "b", None):
            self.lib.dg_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (include/dg.h, dg_server_*).

    submit() copies the request's inputs and returns a ticket; poll() returns
    None until the solve is done, then a dict with times and status; the
    final state is in the host array given as ``out`` at submit."""

    def __init__(self, hbm_budget, prec=DG_FP32, device=0, max_active=0, chunk_steps=0, max_active_dof=0.0):
        self.lib = load_library()
        self.prec = prec
        self.np_dtype = np.float64 if prec == DG_FP64 else np.float32
        o = ServerOpts(int(device), int(prec), int(max_active), int(chunk_steps), float(max_active_dof))
        s = C.c_void_p()
        rc = self.lib.dg_server_create(C.c_size_t(int(hbm_budget)), C.byref(o), C.byref(s))
        if rc != 0:
            raise DGError(rc, "dg_server_create failed")
        self.s = s
        self._outs = {}

    def submit(self, mesh, k, rho, c, U0, dt, nsteps, method=1, reduce_every=2, alpha=1.0, out=None):
        nodes = np.ascontiguousarray(mesh["nodes"], np.float64)
        nbr = np.ascontiguousarray(mesh["nbr"], np.int32)
        nbf = np.ascontiguousarray(mesh["nbr_face"], np.int8)
        ori = np.ascontiguousarray(mesh["orient"], np.int8)
        rho = np.ascontiguousarray(rho, np.float64)
        c = np.ascontiguousarray(c, np.float64)
        U0 = np.ascontiguousarray(U0, self.np_dtype)
        if out is None:
            out = np.empty_like(U0)
        desc = MeshDesc(int(mesh["n_elem"]), int(mesh["geom_degree"]),
                        nodes.ctypes.data_as(C.POINTER(C.c_double)), nbr.ctypes.data_as(C.POINTER(C.c_int32)),
                        nbf.ctypes.data_as(C.POINTER(C.c_int8)), ori.ctypes.data_as(C.POINTER(C.c_int8)))
        req = Request(desc, int(k), float(alpha), rho.ctypes.data_as(C.POINTER(C.c_double)),
                      c.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(U0.ctypes.data),
                      C.c_void_p(out.ctypes.data), float(dt), int(nsteps), int(method), int(reduce_every))
        t = C.c_uint64()
        rc = self.lib.dg_submit(self.s, C.byref(req), C.byref(t))
        if rc != 0:
            raise DGError(rc, "dg_submit rejected the request")
        self._outs[t.value] = out
        return t.value

    def poll(self, ticket, timeout_ms=0):
        r = Result()
        rc = self.lib.dg_poll(self.s, C.c_uint64(ticket), C.byref(r), int(timeout_ms))
        if rc == -5:
            return None
        if rc != 0:
            raise DGError(rc, "dg_poll failed")
        return {"t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done, "status": r.status,
                "out": self._outs.pop(ticket)}

    def request_bytes(self, n_elem, k, geom_degree=1):
        return int(self.lib.dg_request_bytes(int(n_elem), int(k), int(geom_degree), int(self.prec)))

    def stats(self):
        st = ServerStats()
        rc = self.lib.dg_server_stats(self.s, C.byref(st))
        if rc != 0:
            raise DGError(rc, "dg_server_stats failed")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "s", None):
            self.lib.dg_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
