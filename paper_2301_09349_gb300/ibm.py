"""Python binding of the C ABI in include/ibm.h (ctypes).

Every function named ibm_* below calls the C entry point of the same name and
only marshals arguments; all computation runs in the CUDA kernels of
libibm_gb300.so.  There is no fallback: if the library is missing or cannot
be loaded, importing the binding's functions raises.

`Grid` is a convenience owner of the device memory (a torch uint8 workspace
and state tensors) around one handle.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import cases
from .build import LIB

IBM_OK = 0
_STATUS = {1: "IBM_ERR_ARG", 2: "IBM_ERR_CUDA", 3: "IBM_ERR_NONFINITE", 4: "IBM_ERR_NOCONV",
           5: "IBM_ERR_WORKSPACE", 6: "IBM_ERR_TIMEOUT", 7: "IBM_ERR_STATE",
           8: "IBM_ERR_UNSUPPORTED", 9: "IBM_ERR_BOUNDS"}


class IbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s (%d): %s" % (_STATUS.get(status, "?"), status, message))
        self.status = status
        self.message = message


class GridDescC(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
        ("h", ctypes.c_double), ("fp_bytes", ctypes.c_int), ("gamma", ctypes.c_double),
        ("Pr", ctypes.c_double), ("Re", ctypes.c_double), ("Mach", ctypes.c_double),
        ("sutherland_S", ctypes.c_double), ("cfl", ctypes.c_double), ("bc", ctypes.c_int * 6),
        ("tile", ctypes.c_int * 3), ("D", ctypes.c_double), ("energy_reading", ctypes.c_int),
        ("forcing_per_stage", ctypes.c_int),
    ]


class MotionC(ctypes.Structure):
    _fields_ = [("amp", ctypes.c_double), ("freq", ctypes.c_double), ("axis", ctypes.c_int)]


class BatchTuningC(ctypes.Structure):
    _fields_ = [("tile_shape", ctypes.c_int), ("markers_per_block", ctypes.c_int),
                ("use_graph", ctypes.c_int)]


_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_up = ctypes.POINTER(ctypes.c_uint)
_lib = None

# (name, restype, argtypes) of every entry point declared in include/ibm.h
SIGNATURES = [
    ("ibm_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(GridDescC), ctypes.c_int]),
    ("ibm_create_grid", ctypes.c_int, [ctypes.POINTER(GridDescC), ctypes.c_int, _vp,
                                       ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
    ("ibm_destroy", ctypes.c_int, [_vp]),
    ("ibm_set_state", ctypes.c_int, [_vp, _vp]),
    ("ibm_get_state", ctypes.c_int, [_vp, _vp]),
    ("ibm_set_state_host", ctypes.c_int, [_vp, _vp]),
    ("ibm_get_state_host", ctypes.c_int, [_vp, _vp]),
    ("ibm_set_markers", ctypes.c_int, [_vp, ctypes.c_int, _dp, _dp, _dp, ctypes.POINTER(MotionC),
                                       ctypes.c_int, _ip]),
    ("ibm_set_wall_temperature", ctypes.c_int, [_vp, _dp]),
    ("ibm_set_quadrature", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int]),
    ("ibm_step", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double]),
    ("ibm_step_graphs", ctypes.c_int, [_vp, ctypes.c_int]),
    ("ibm_forces_and_nusselt", ctypes.c_int, [_vp, _dp, _dp, _dp, _dp, _dp]),
    ("ibm_backward", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, _dp, _dp]),
    ("ibm_sync", ctypes.c_int, [_vp]),
    ("ibm_last_error", ctypes.c_char_p, [_vp]),
    ("ibm_get_markers", ctypes.c_int, [_vp, _dp, _dp, _ip]),
    ("ibm_get_marker_forcing", ctypes.c_int, [_vp, _dp, _dp, _dp]),
    ("ibm_get_bins", ctypes.c_int, [_vp, _ip, _ip, _up, _ip]),
    ("ibm_get_time", ctypes.c_int, [_vp, _dp, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    ("ibm_rhs", ctypes.c_int, [_vp, _vp, _vp]),
    ("ibm_interpolate", ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    ("ibm_spread", ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    ("ibm_profile", ctypes.c_int, [_vp, ctypes.c_int]),
    ("ibm_profile_read", ctypes.c_int, [_vp, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    ("ibm_rhs_dt_noalloc", ctypes.c_int, [ctypes.POINTER(GridDescC), _vp, _vp, _vp, _vp]),
    ("ibm_adjoint_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(GridDescC), ctypes.c_int,
                                                      ctypes.c_int, ctypes.c_int]),
    ("ibm_record", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t]),
    ("ibm_rhs_vjp", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("ibm_surface_pressure", ctypes.c_int, [_vp, _dp]),
    ("ibm_batch_workspace_bytes", ctypes.c_size_t, [ctypes.c_int, ctypes.POINTER(GridDescC), _ip]),
    ("ibm_create_batch", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(GridDescC), _ip, _vp,
                                        ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
    ("ibm_batch_destroy", ctypes.c_int, [_vp]),
    ("ibm_batch_case", _vp, [_vp, ctypes.c_int]),
    ("ibm_batch_step", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double]),
    ("ibm_batch_sync", ctypes.c_int, [_vp, _ip]),
    ("ibm_batch_set_wall_temperature", ctypes.c_int, [_vp, _dp]),
    ("ibm_batch_forces", ctypes.c_int, [_vp, _dp]),
    ("ibm_batch_get_tuning", ctypes.c_int, [_vp, ctypes.POINTER(BatchTuningC)]),
    ("ibm_batch_set_tuning", ctypes.c_int, [_vp, ctypes.POINTER(BatchTuningC)]),
    ("ibm_batch_autotune", ctypes.c_int, [_vp, ctypes.c_int, _dp, _dp]),
    ("ibm_batch_profile", ctypes.c_int, [_vp, ctypes.c_int]),
    ("ibm_batch_profile_read", ctypes.c_int, [_vp, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    ("ibm_batch_last_error", ctypes.c_char_p, [_vp]),
]

BATCH_TILE_SHAPES = [(16, 16), (32, 8), (64, 4), (8, 32)]
BATCH_WARPS = [1, 2, 4, 8, 16]
BATCH_FORCE_FIELDS = ["Fx", "Fy", "heat_rate", "Cd", "Cl", "Nu", "dt", "t"]

PROF_GROUPS = ["stage1", "stage2", "markers", "interp_force", "spread_apply", "finish"]


def lib_path() -> str:
    return os.environ.get("IBM_GB300_LIB", LIB)


def lib():
    """Load libibm_gb300.so; raises when it is missing (no CPU fallback)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("libibm_gb300.so is not built (%s); run "
                               "paper_2301_09349_gb300.build.build() first" % path)
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st: int, handle=None):
    if st != IBM_OK:
        msg = lib().ibm_last_error(handle)
        raise IbmError(st, msg.decode() if msg else "")


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


def make_desc(g: cases.GridDesc, energy_reading: int = 0) -> GridDescC:
    d = GridDescC()
    d.dim = g.dim
    for i in range(3):
        d.n[i] = int(g.n[i]) if i < g.dim else 1
        d.lo[i] = float(g.lo[i]) if i < len(g.lo) else 0.0
        d.tile[i] = int(g.tile[i]) if i < g.dim else 1
    d.h = g.h
    d.fp_bytes = g.fp_bytes
    d.gamma, d.Pr, d.Re, d.Mach = g.gamma, g.Pr, g.Re, g.Mach
    d.sutherland_S, d.cfl = g.sutherland_S, g.cfl
    for i in range(6):
        d.bc[i] = int(g.bc[i])
    d.D = g.D
    d.energy_reading = energy_reading
    d.forcing_per_stage = int(getattr(g, "forcing_per_stage", 0))
    return d


# ---------------------------------------------------------------------------
# thin entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def ibm_workspace_bytes(desc: GridDescC, max_markers: int) -> int:
    return int(lib().ibm_workspace_bytes(ctypes.byref(desc), int(max_markers)))


def ibm_create_grid(desc: GridDescC, max_markers: int, workspace_ptr: int, nbytes: int,
                    stream_ptr: int):
    h = _vp()
    st = lib().ibm_create_grid(ctypes.byref(desc), int(max_markers), _vp(workspace_ptr),
                               ctypes.c_size_t(nbytes), _vp(stream_ptr), ctypes.byref(h))
    _check(st, None)
    return h


def ibm_destroy(h):
    _check(lib().ibm_destroy(h), None)


def ibm_set_state(h, U_ptr: int):
    _check(lib().ibm_set_state(h, _vp(U_ptr)), h)


def ibm_get_state(h, U_ptr: int):
    _check(lib().ibm_get_state(h, _vp(U_ptr)), h)


def ibm_set_state_host(h, U_host_ptr: int):
    _check(lib().ibm_set_state_host(h, _vp(U_host_ptr)), h)


def ibm_get_state_host(h, U_host_ptr: int):
    _check(lib().ibm_get_state_host(h, _vp(U_host_ptr)), h)


def ibm_set_markers(h, X, Tw, Ub=None, motion: Optional[cases.Motion] = None,
                    dedup: bool = True) -> int:
    X = _f64(X)
    Tw = _f64(Tw)
    Ub = None if Ub is None else _f64(Ub)
    mc = None
    if motion is not None:
        mc = MotionC(motion.amp, motion.freq, motion.axis)
    nk = ctypes.c_int(0)
    n = 0 if X.size == 0 else X.shape[0]
    st = lib().ibm_set_markers(h, n, _ptr(X), _ptr(Ub), _ptr(Tw),
                               ctypes.byref(mc) if mc is not None else None, int(bool(dedup)),
                               ctypes.byref(nk))
    _check(st, h)
    return nk.value


def ibm_set_wall_temperature(h, Tw):
    Tw = _f64(Tw)
    _check(lib().ibm_set_wall_temperature(h, _ptr(Tw)), h)


def ibm_set_quadrature(h, tol: float, maxit: int):
    _check(lib().ibm_set_quadrature(h, ctypes.c_double(tol), int(maxit)), h)


def ibm_step(h, nsteps: int, dt_fixed: float = 0.0):
    _check(lib().ibm_step(h, int(nsteps), ctypes.c_double(dt_fixed)), h)


def ibm_step_graphs(h, steps_per_graph: int):
    _check(lib().ibm_step_graphs(h, int(steps_per_graph)), h)


def ibm_forces_and_nusselt(h) -> dict:
    f = (ctypes.c_double * 3)()
    q, cd, cl, nu = (ctypes.c_double() for _ in range(4))
    _check(lib().ibm_forces_and_nusselt(h, f, ctypes.byref(q), ctypes.byref(cd), ctypes.byref(cl),
                                        ctypes.byref(nu)), h)
    return {"force": np.array(f[:]), "heat_rate": q.value, "Cd": cd.value, "Cl": cl.value,
            "Nu": nu.value}


def ibm_backward(h, dJ_dCd: float, dJ_dNu: float, n_kept: int, dim: int):
    dX = np.zeros(max(n_kept * dim, 1))
    dT = np.zeros(max(n_kept, 1))
    _check(lib().ibm_backward(h, dJ_dCd, dJ_dNu, _ptr(dX), _ptr(dT)), h)
    return dX[: n_kept * dim].reshape(n_kept, dim), dT[:n_kept]


def ibm_adjoint_workspace_bytes(desc: GridDescC, max_markers: int, max_steps: int,
                                every: int) -> int:
    return int(lib().ibm_adjoint_workspace_bytes(ctypes.byref(desc), int(max_markers),
                                                 int(max_steps), int(every)))


def ibm_record(h, max_steps: int, every: int, workspace_ptr: int, nbytes: int):
    _check(lib().ibm_record(h, int(max_steps), int(every), _vp(workspace_ptr),
                            ctypes.c_size_t(nbytes)), h)


def ibm_rhs_vjp(h, U_ptr: int, V_ptr: int, out_ptr: int):
    _check(lib().ibm_rhs_vjp(h, _vp(U_ptr), _vp(V_ptr), _vp(out_ptr)), h)


def ibm_surface_pressure(h, n_kept: int) -> np.ndarray:
    cp = np.zeros(max(n_kept, 1))
    _check(lib().ibm_surface_pressure(h, _ptr(cp)), h)
    return cp[:n_kept]


def ibm_sync(h):
    _check(lib().ibm_sync(h), h)


def ibm_last_error(h) -> str:
    m = lib().ibm_last_error(h)
    return m.decode() if m else ""


def ibm_get_markers(h, n_kept: int, dim: int):
    X = np.zeros((max(n_kept, 1), dim))
    eps = np.zeros(max(n_kept, 1))
    idx = np.zeros(max(n_kept, 1), dtype=np.int32)
    _check(lib().ibm_get_markers(h, _ptr(X), _ptr(eps), _ptr(idx, _ip)), h)
    return X[:n_kept], eps[:n_kept], idx[:n_kept]


def ibm_get_marker_forcing(h, n_kept: int, dim: int):
    rho = np.zeros(max(n_kept, 1))
    F = np.zeros((max(n_kept, 1), dim))
    Q = np.zeros(max(n_kept, 1))
    _check(lib().ibm_get_marker_forcing(h, _ptr(rho), _ptr(F), _ptr(Q)), h)
    return rho[:n_kept], F[:n_kept], Q[:n_kept]


def ibm_get_bins(h, n_tiles: int, n_kept: int):
    tile_off = np.zeros(n_tiles + 1, dtype=np.int32)
    perm = np.zeros(max(n_kept, 1), dtype=np.int32)
    keys = np.zeros(max(n_kept, 1), dtype=np.uint32)
    nt = ctypes.c_int(0)
    _check(lib().ibm_get_bins(h, _ptr(tile_off, _ip), _ptr(perm, _ip), _ptr(keys, _up),
                              ctypes.byref(nt)), h)
    return tile_off, perm[:n_kept], keys[:n_kept]


def ibm_get_time(h):
    dt, t = ctypes.c_double(), ctypes.c_double()
    s = ctypes.c_longlong()
    _check(lib().ibm_get_time(h, ctypes.byref(dt), ctypes.byref(t), ctypes.byref(s)), h)
    return dt.value, t.value, s.value


def ibm_rhs(h, U_ptr: int, L_ptr: int):
    _check(lib().ibm_rhs(h, _vp(U_ptr), _vp(L_ptr)), h)


def ibm_interpolate(h, field_ptr: int, nc: int, out_ptr: int):
    _check(lib().ibm_interpolate(h, _vp(field_ptr), int(nc), _vp(out_ptr)), h)


def ibm_spread(h, R_ptr: int, nc: int, out_ptr: int):
    _check(lib().ibm_spread(h, _vp(R_ptr), int(nc), _vp(out_ptr)), h)


def ibm_profile(h, enable: bool):
    _check(lib().ibm_profile(h, int(bool(enable))), h)


def ibm_profile_read(h) -> dict:
    ms = (ctypes.c_double * len(PROF_GROUPS))()
    n = (ctypes.c_longlong * len(PROF_GROUPS))()
    _check(lib().ibm_profile_read(h, ms, n), h)
    return {name: (ms[i], n[i]) for i, name in enumerate(PROF_GROUPS)}


def ibm_rhs_dt_noalloc(desc: GridDescC, U_ptr: int, L_ptr: int, dt_ptr: int, stream_ptr: int):
    """Stage 1 without handle or workspace (scratch in a static device array;
    overlapping calls race)."""
    _check(lib().ibm_rhs_dt_noalloc(ctypes.byref(desc), _vp(U_ptr), _vp(L_ptr), _vp(dt_ptr),
                                    _vp(stream_ptr)), None)


def _bcheck(st: int, handle=None):
    if st != IBM_OK:
        msg = lib().ibm_batch_last_error(handle)
        raise IbmError(st, msg.decode() if msg else "")


def _desc_array(descs):
    arr = (GridDescC * len(descs))()
    for i, d in enumerate(descs):
        arr[i] = d
    return arr


def ibm_batch_workspace_bytes(descs, max_markers) -> int:
    mm = np.ascontiguousarray(max_markers, dtype=np.int32)
    return int(lib().ibm_batch_workspace_bytes(len(descs), _desc_array(descs), _ptr(mm, _ip)))


def ibm_create_batch(descs, max_markers, workspace_ptr: int, nbytes: int, stream_ptr: int):
    mm = np.ascontiguousarray(max_markers, dtype=np.int32)
    h = _vp()
    st = lib().ibm_create_batch(len(descs), _desc_array(descs), _ptr(mm, _ip), _vp(workspace_ptr),
                                ctypes.c_size_t(nbytes), _vp(stream_ptr), ctypes.byref(h))
    _bcheck(st, None)
    return h


def ibm_batch_destroy(h):
    _bcheck(lib().ibm_batch_destroy(h), None)


def ibm_batch_case(h, c: int):
    p = lib().ibm_batch_case(h, int(c))
    if not p:
        raise IbmError(1, "no case %d in this batch" % c)
    return _vp(p)


def ibm_batch_step(h, nsteps: int, dt_fixed: float = 0.0):
    _bcheck(lib().ibm_batch_step(h, int(nsteps), ctypes.c_double(dt_fixed)), h)


def ibm_batch_sync(h):
    bad = ctypes.c_int(-1)
    _bcheck(lib().ibm_batch_sync(h, ctypes.byref(bad)), h)


def ibm_batch_set_wall_temperature(h, Tw):
    """Tw: the kept markers' wall temperatures of all cases, case after case"""
    Tw = _f64(Tw)
    _bcheck(lib().ibm_batch_set_wall_temperature(h, _ptr(Tw)), h)


def ibm_batch_forces(h, ncases: int) -> np.ndarray:
    """(ncases, 8) array: Fx, Fy, heat rate, Cd, Cl, Nu, dt, t per case."""
    out = np.zeros((ncases, 8))
    _bcheck(lib().ibm_batch_forces(h, _ptr(out)), h)
    return out


def ibm_batch_get_tuning(h) -> dict:
    t = BatchTuningC()
    _bcheck(lib().ibm_batch_get_tuning(h, ctypes.byref(t)), h)
    return {"tile_shape": t.tile_shape, "markers_per_block": t.markers_per_block,
            "use_graph": t.use_graph}


def ibm_batch_set_tuning(h, tile_shape: int, markers_per_block: int, use_graph: int):
    t = BatchTuningC(int(tile_shape), int(markers_per_block), int(use_graph))
    _bcheck(lib().ibm_batch_set_tuning(h, ctypes.byref(t)), h)


def ibm_batch_profile(h, enable: bool):
    _bcheck(lib().ibm_batch_profile(h, int(bool(enable))), h)


def ibm_batch_profile_read(h) -> dict:
    ms = (ctypes.c_double * len(PROF_GROUPS))()
    n = (ctypes.c_longlong * len(PROF_GROUPS))()
    _bcheck(lib().ibm_batch_profile_read(h, ms, n), h)
    return {name: (ms[i], n[i]) for i, name in enumerate(PROF_GROUPS)}


def ibm_batch_autotune(h, reps: int = 5) -> dict:
    sms = np.zeros(len(BATCH_TILE_SHAPES))
    ims = np.zeros(len(BATCH_WARPS))
    _bcheck(lib().ibm_batch_autotune(h, int(reps), _ptr(sms), _ptr(ims)), h)
    return {"stage_ms": sms, "interp_ms": ims}


# ---------------------------------------------------------------------------
# convenience owner of device memory
# ---------------------------------------------------------------------------

class Grid:
    """One IBM grid on one GPU: a torch-allocated workspace plus the handle."""

    def __init__(self, g: cases.GridDesc, max_markers: int = 0, device="cuda", stream=None,
                 energy_reading: int = 0):
        import torch
        self.torch = torch
        self.g = g
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.dtype = torch.float32 if g.fp_bytes == 4 else torch.float64
        self.desc = make_desc(g, energy_reading)
        nbytes = ibm_workspace_bytes(self.desc, max_markers)
        if nbytes == 0:
            raise IbmError(1, "invalid grid description")
        # over-allocate by 256 bytes and align the base
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self.ws_ptr = (base + 255) // 256 * 256
        self.nbytes = nbytes
        self.h = ibm_create_grid(self.desc, max_markers, self.ws_ptr, nbytes,
                                 self.stream.cuda_stream)
        self.max_markers = max_markers
        self.n_kept = 0

    @classmethod
    def _borrowed(cls, h, g: cases.GridDesc, device, stream, energy_reading: int = 0):
        """A Grid view of a handle owned elsewhere (a batch case)."""
        import torch
        self = cls.__new__(cls)
        self.torch = torch
        self.g = g
        self.device = torch.device(device)
        self.stream = stream
        self.dtype = torch.float32 if g.fp_bytes == 4 else torch.float64
        self.desc = make_desc(g, energy_reading)
        self.ws = None
        self.h = h
        self.n_kept = 0
        self._owned = False
        return self

    def close(self):
        if getattr(self, "h", None) is not None:
            if getattr(self, "_owned", True):
                ibm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state -----------------------------------------------------------
    def empty_state(self):
        return self.torch.empty(self.g.shape(), dtype=self.dtype, device=self.device)

    def _order(self):
        """make the library's stream wait for work queued on torch's stream"""
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def set_state(self, U):
        t = self.torch
        if isinstance(U, np.ndarray):
            U = t.from_numpy(np.ascontiguousarray(U))
        U = U.to(self.device, self.dtype).contiguous()
        self._order()
        ibm_set_state(self.h, U.data_ptr())
        self.stream.synchronize()

    def get_state(self):
        out = self.empty_state()
        self._order()
        ibm_get_state(self.h, out.data_ptr())
        return out

    # -- markers ---------------------------------------------------------
    def set_markers(self, X, Tw, Ub=None, motion=None, dedup=True) -> int:
        self.n_kept = ibm_set_markers(self.h, X, Tw, Ub, motion, dedup)
        return self.n_kept

    def set_wall_temperature(self, Tw):
        ibm_set_wall_temperature(self.h, Tw)

    def set_quadrature(self, tol: float, maxit: int = 4000):
        """stopping rule of the A~ eps~ = 1 solve, from the next set_markers"""
        ibm_set_quadrature(self.h, tol, maxit)

    def step(self, nsteps: int = 1, dt_fixed: float = 0.0):
        ibm_step(self.h, nsteps, dt_fixed)

    def use_graphs(self, steps_per_graph: int):
        """replay chunks of steps_per_graph (even) steps from CUDA graphs"""
        ibm_step_graphs(self.h, steps_per_graph)

    def sync(self):
        ibm_sync(self.h)

    def forces(self) -> dict:
        return ibm_forces_and_nusselt(self.h)

    def markers(self):
        return ibm_get_markers(self.h, self.n_kept, self.g.dim)

    def surface_pressure(self):
        """C_p at the kept markers from the current state"""
        return ibm_surface_pressure(self.h, self.n_kept)

    def marker_forcing(self):
        return ibm_get_marker_forcing(self.h, self.n_kept, self.g.dim)

    def bins(self):
        nt = 1
        for d in range(self.g.dim):
            nt *= -(-self.g.n[d] // self.g.tile[d])
        return ibm_get_bins(self.h, nt, self.n_kept)

    def time(self):
        return ibm_get_time(self.h)

    # -- operators -------------------------------------------------------
    def rhs(self, U):
        U = U.to(self.device, self.dtype).contiguous()
        L = self.torch.empty_like(U)
        self._order()
        ibm_rhs(self.h, U.data_ptr(), L.data_ptr())
        self.stream.synchronize()
        return L

    def interpolate(self, field):
        field = field.to(self.device, self.dtype).contiguous()
        nc = field.shape[0]
        out = self.torch.empty((max(self.n_kept, 1), nc), dtype=self.torch.float64,
                               device=self.device)
        self._order()
        ibm_interpolate(self.h, field.data_ptr(), nc, out.data_ptr())
        self.stream.synchronize()
        return out[: self.n_kept]

    # -- discrete adjoint ------------------------------------------------
    def record(self, max_steps: int, every: int = 50):
        """allocate the adjoint workspace and start recording steps"""
        nb = ibm_adjoint_workspace_bytes(self.desc, self.max_markers, max_steps, every)
        if nb == 0:
            raise IbmError(1, "invalid adjoint workspace request")
        self.adj_ws = self.torch.empty(nb + 256, dtype=self.torch.uint8, device=self.device)
        ptr = (self.adj_ws.data_ptr() + 255) // 256 * 256
        ibm_record(self.h, max_steps, every, ptr, nb)

    def backward(self, dJ_dCd: float, dJ_dNu: float):
        """(dJ/dX (n_kept, dim), dJ/dT_w (n_kept)) over the recorded steps"""
        return ibm_backward(self.h, dJ_dCd, dJ_dNu, self.n_kept, self.g.dim)

    def rhs_vjp(self, U, V):
        U = U.to(self.device, self.dtype).contiguous()
        V = V.to(self.device, self.dtype).contiguous()
        out = self.torch.empty_like(U)
        self._order()
        ibm_rhs_vjp(self.h, U.data_ptr(), V.data_ptr(), out.data_ptr())
        self.stream.synchronize()
        return out

    def spread(self, R):
        R = R.to(self.device, self.torch.float64).contiguous()
        nc = R.shape[1]
        shape = (nc,) + tuple(reversed(self.g.n[: self.g.dim]))
        out = self.torch.empty(shape, dtype=self.dtype, device=self.device)
        self._order()
        ibm_spread(self.h, R.data_ptr(), nc, out.data_ptr())
        self.stream.synchronize()
        return out


class Batch:
    """Many independent 2D grids advanced together (one launch per stage).

    `cases[c]` is a Grid view of case c: set its state and markers and read
    its state, forces and time through it.  The batch owns the memory."""

    def __init__(self, gs, max_markers, device="cuda", stream=None, energy_reading: int = 0):
        import torch
        self.torch = torch
        self.gs = list(gs)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.descs = [make_desc(g, energy_reading) for g in self.gs]
        self.max_markers = [int(m) for m in max_markers]
        nbytes = ibm_batch_workspace_bytes(self.descs, self.max_markers)
        if nbytes == 0:
            # let the library say why (it checks the description first)
            ibm_create_batch(self.descs, self.max_markers, 0, 0, 0)
            raise IbmError(1, "invalid batch description")
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = (self.ws.data_ptr() + 255) // 256 * 256
        self.nbytes = nbytes
        self.h = ibm_create_batch(self.descs, self.max_markers, self.ws_ptr, nbytes,
                                  self.stream.cuda_stream)
        self.cases = [Grid._borrowed(ibm_batch_case(self.h, c), g, self.device, self.stream,
                                     energy_reading)
                      for c, g in enumerate(self.gs)]

    def __len__(self):
        return len(self.cases)

    def close(self):
        if getattr(self, "h", None) is not None:
            for c in self.cases:
                c.h = None
            ibm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps: int = 1, dt_fixed: float = 0.0):
        ibm_batch_step(self.h, nsteps, dt_fixed)

    def sync(self):
        ibm_batch_sync(self.h)

    def set_wall_temperature(self, Tw):
        """wall temperatures of every case's kept markers, concatenated in case order"""
        ibm_batch_set_wall_temperature(self.h, Tw)

    def forces(self) -> np.ndarray:
        return ibm_batch_forces(self.h, len(self.cases))

    def tuning(self) -> dict:
        return ibm_batch_get_tuning(self.h)

    def set_tuning(self, tile_shape=None, markers_per_block=None, use_graph=None):
        t = self.tuning()
        ibm_batch_set_tuning(self.h,
                             t["tile_shape"] if tile_shape is None else tile_shape,
                             t["markers_per_block"] if markers_per_block is None
                             else markers_per_block,
                             t["use_graph"] if use_graph is None else int(bool(use_graph)))

    def autotune(self, reps: int = 5) -> dict:
        return ibm_batch_autotune(self.h, reps)


def cd_nu_objective():
    """torch.autograd.Function computing J = a C_d + b Nu after `steps` IBM
    steps from the state U0, as a function of the marker positions X (n, dim)
    and wall temperatures Tw (n) (float64 CPU tensors, static markers).  The
    forward pass runs set_markers / set_state / record / step on `grid`; the
    backward pass is ibm_backward.  Markers dropped by the one-per-cell dedup
    get zero gradient."""
    import torch

    class CdNuObjective(torch.autograd.Function):
        @staticmethod
        def forward(ctx, X, Tw, grid, U0, steps, a, b, every):
            Xn = X.detach().cpu().numpy().astype(np.float64)
            Tn = Tw.detach().cpu().numpy().astype(np.float64)
            grid.set_markers(Xn, Tn)
            grid.set_state(U0)
            grid.record(int(steps), int(every))
            grid.step(int(steps))
            f = grid.forces()
            ctx.grid, ctx.a, ctx.b, ctx.n, ctx.dim = grid, float(a), float(b), len(Xn), Xn.shape[1]
            return torch.tensor(ctx.a * f["Cd"] + ctx.b * f["Nu"], dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            gXk, gTk = ctx.grid.backward(ctx.a, ctx.b)
            _, _, idx = ctx.grid.markers()
            gX = np.zeros((ctx.n, ctx.dim))
            gT = np.zeros(ctx.n)
            gX[idx] = gXk
            gT[idx] = gTk
            s = float(gJ)
            return (torch.from_numpy(gX * s), torch.from_numpy(gT * s),
                    None, None, None, None, None, None)

    return CdNuObjective
