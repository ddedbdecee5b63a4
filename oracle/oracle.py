"""Python face of the FP64 CPU oracle (oracle/ibm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by the benchmark's CPU-baseline leg.  The product path (the CUDA library and
its binding) never imports this module.  Arrays are numpy float64; the
conserved state is (ncomp, [nz,] ny, nx) as built by the seeded generators.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ibm_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_up = ctypes.POINTER(ctypes.c_uint)


class OrDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
        ("h", ctypes.c_double), ("gamma", ctypes.c_double), ("Pr", ctypes.c_double),
        ("Re", ctypes.c_double), ("Mach", ctypes.c_double), ("S", ctypes.c_double),
        ("cfl", ctypes.c_double), ("bc", ctypes.c_int * 6), ("tile", ctypes.c_int * 3),
        ("D", ctypes.c_double), ("energy_reading", ctypes.c_int),
        ("forcing_per_stage", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, OpenMP, no fast-math)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        L.or_phi.restype = ctypes.c_double
        L.or_phi.argtypes = [ctypes.c_double]
        L.or_dt.restype = ctypes.c_double
        L.or_fluid_predictor.restype = ctypes.c_double
        L.or_step.restype = ctypes.c_double
        L.or_num_tiles.restype = ctypes.c_long
        _lib = L
    return _lib


def _p(a, t=_dp):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def desc(g, energy_reading: int = 0) -> OrDesc:
    """Oracle descriptor from a cases.GridDesc."""
    d = OrDesc()
    d.dim = g.dim
    for i in range(3):
        d.n[i] = int(g.n[i]) if i < g.dim else 1
        d.lo[i] = float(g.lo[i]) if i < len(g.lo) else 0.0
        d.tile[i] = int(g.tile[i]) if i < g.dim else 1
    d.h = g.h
    d.gamma, d.Pr, d.Re, d.Mach, d.S, d.cfl = g.gamma, g.Pr, g.Re, g.Mach, g.sutherland_S, g.cfl
    for i in range(6):
        d.bc[i] = int(g.bc[i])
    d.D = g.D
    d.energy_reading = energy_reading
    d.forcing_per_stage = int(getattr(g, "forcing_per_stage", 0))
    return d


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return lib().or_get_threads()


def phi(r):
    r = _f64(np.atleast_1d(r))
    out = np.empty_like(r)
    lib().or_phi_many(_p(r), ctypes.c_long(r.size), _p(out))
    return out


def owner_cells(g, X):
    X = _f64(X)
    cell = np.zeros((len(X), g.dim), dtype=np.int32)
    rc = lib().or_owner_cells(ctypes.byref(desc(g)), len(X), _p(X), _p(cell, _ip))
    return rc, cell


def dedup(g, X):
    X = _f64(X)
    keep = np.zeros(max(len(X), 1), dtype=np.int32)
    nk = ctypes.c_int(0)
    rc = lib().or_dedup(ctypes.byref(desc(g)), len(X), _p(X), _p(keep, _ip), ctypes.byref(nk))
    return rc, keep[: nk.value].copy()


def num_tiles(g) -> int:
    return int(lib().or_num_tiles(ctypes.byref(desc(g))))


def bin_markers(g, X):
    X = _f64(X)
    nt = num_tiles(g)
    tile_off = np.zeros(nt + 1, dtype=np.int32)
    perm = np.zeros(max(len(X), 1), dtype=np.int32)
    keys = np.zeros(max(len(X), 1), dtype=np.uint32)
    rc = lib().or_bin(ctypes.byref(desc(g)), len(X), _p(X), _p(tile_off, _ip), _p(perm, _ip),
                      _p(keys, _up))
    return rc, tile_off, perm[: len(X)].copy(), keys[: len(X)].copy()


def _field2d(g, f):
    f = _f64(f)
    return f.reshape(-1, g.ncells)


def interp(g, X, field, dense: bool = False):
    """I[field] at the markers; field is (nc, cells...) -> (ns, nc)."""
    X = _f64(X)
    f = _field2d(g, field)
    nc = f.shape[0]
    out = np.zeros((len(X), nc))
    fn = lib().or_interp_dense if dense else lib().or_interp
    fn(ctypes.byref(desc(g)), len(X), _p(X), _p(f), nc, _p(out))
    return out


def spread(g, X, eps_t, R, dense: bool = False):
    """S[R] on the grid; R is (ns, nc) -> (nc, N)."""
    X, eps_t, R = _f64(X), _f64(eps_t), _f64(R)
    nc = R.shape[1]
    out = np.zeros((nc, g.ncells))
    fn = lib().or_spread_dense if dense else lib().or_spread
    fn(ctypes.byref(desc(g)), len(X), _p(X), _p(eps_t), _p(R), nc, _p(out))
    return out


def assemble_A_dense(g, X):
    X = _f64(X)
    A = np.zeros((len(X), len(X)))
    lib().or_assemble_A_dense(ctypes.byref(desc(g)), len(X), _p(X), _p(A))
    return A


def quadrature(g, X, tol: float = 1e-12, maxit: int = 20000, eps0=None):
    X = _f64(X)
    eps = np.zeros(max(len(X), 1)) if eps0 is None else _f64(eps0).copy()
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    rc = lib().or_quadrature(ctypes.byref(desc(g)), len(X), _p(X), _p(eps), ctypes.c_double(tol),
                             int(maxit), int(eps0 is not None), ctypes.byref(it),
                             ctypes.byref(res))
    return rc, eps[: len(X)].copy(), it.value, res.value


def rhs(g, U):
    U = _f64(U)
    L = np.zeros_like(U)
    lib().or_rhs(ctypes.byref(desc(g)), _p(U), _p(L))
    return L


def dt(g, U) -> float:
    U = _f64(U)
    return float(lib().or_dt(ctypes.byref(desc(g)), _p(U)))


def fill_ghosts(g, U):
    U = _f64(U)
    P = [g.n[d] + 4 if d < g.dim else 1 for d in range(3)]
    out = np.zeros((g.ncomp, P[2], P[1], P[0]))
    lib().or_fill_ghosts(ctypes.byref(desc(g)), _p(U), _p(out))
    return out.reshape((g.ncomp,) + tuple(reversed(P[: g.dim])))


def predictor(g, U, dt_fixed: float = 0.0):
    U = _f64(U)
    out = np.zeros_like(U)
    d = lib().or_fluid_predictor(ctypes.byref(desc(g)), _p(U), _p(out), ctypes.c_double(dt_fixed))
    return float(d), out


def interp_force(g, X, Ub, Tw, Ustar):
    X, Tw, Us = _f64(X), _f64(Tw), _f64(Ustar)
    ns = len(X)
    rhoL = np.zeros(max(ns, 1))
    G = np.zeros((max(ns, 1), g.dim))
    H = np.zeros(max(ns, 1))
    ubp = _p(_f64(Ub)) if Ub is not None else None
    lib().or_interp_force(ctypes.byref(desc(g)), ns, _p(X), ubp, _p(Tw), _p(Us), _p(rhoL), _p(G),
                          _p(H))
    return rhoL[:ns], G[:ns], H[:ns]


def spread_apply(g, X, eps_t, G, H, U, energy_reading: int = 0):
    out = _f64(U).copy()
    X, eps_t, G, H = _f64(X), _f64(eps_t), _f64(G), _f64(H)
    lib().or_spread_apply(ctypes.byref(desc(g, energy_reading)), len(X), _p(X), _p(eps_t), _p(G),
                          _p(H), _p(out))
    return out


def band_mask(g, X):
    X = _f64(X)
    mask = np.zeros(g.ncells, dtype=np.uint8)
    cnt = lib().or_band_mask(ctypes.byref(desc(g)), len(X), _p(X), _p(mask, ctypes.POINTER(ctypes.c_ubyte)))
    return cnt, mask


def step(g, X, Ub, Tw, eps_t, U, dt_fixed: float = 0.0, energy_reading: int = 0):
    """One IBM step.  Returns (dt, Unew, G, H, rhoL) with G = dt F, H = dt Q."""
    X, Tw, eps_t, U = _f64(X), _f64(Tw), _f64(eps_t), _f64(U)
    ns = len(X)
    out = np.zeros_like(U)
    G = np.zeros((max(ns, 1), g.dim))
    H = np.zeros(max(ns, 1))
    rhoL = np.zeros(max(ns, 1))
    ubp = _p(_f64(Ub)) if Ub is not None else None
    d = lib().or_step(ctypes.byref(desc(g, energy_reading)), ns, _p(X), ubp, _p(Tw), _p(eps_t),
                      _p(U), _p(out), ctypes.c_double(dt_fixed), _p(G), _p(H), _p(rhoL))
    return float(d), out, G[:ns], H[:ns], rhoL[:ns]


def forces(g, eps_t, G, H, Tw, dt):
    eps_t, G, H, Tw = _f64(eps_t), _f64(G), _f64(H), _f64(Tw)
    f = np.zeros(3)
    heat, Cd, Cl, Nu = (ctypes.c_double() for _ in range(4))
    lib().or_forces(ctypes.byref(desc(g)), len(eps_t), _p(eps_t), _p(G), _p(H), _p(Tw),
                    ctypes.c_double(dt), _p(f), ctypes.byref(heat), ctypes.byref(Cd),
                    ctypes.byref(Cl), ctypes.byref(Nu))
    return f, heat.value, Cd.value, Cl.value, Nu.value


def surface_pressure(g, X, U):
    """C_p,k = (I[p]_k - p_inf) / (1/2): the pressure p = (gamma - 1)(rho E -
    |rho u|^2/(2 rho)) of every cell, interpolated to the markers (Eq. interp)."""
    U = _f64(U).reshape(g.ncomp, -1)
    rho = U[0]
    msq = (U[1: g.dim + 1] ** 2).sum(axis=0)
    p = (g.gamma - 1.0) * (U[g.dim + 1] - 0.5 * msq / rho)
    p_inf = 1.0 / (g.gamma * g.Mach * g.Mach)
    return 2.0 * (interp(g, X, p.reshape((1,) + U.shape[1:]))[:, 0] - p_inf)


def motion(X0, amp, freq, axis, t):
    X0 = _f64(X0)
    ns, dim = X0.shape
    X = np.zeros_like(X0)
    Ub = np.zeros_like(X0)
    lib().or_motion(ns, dim, _p(X0), ctypes.c_double(amp), ctypes.c_double(freq), int(axis),
                    ctypes.c_double(t), _p(X), _p(Ub))
    return X, Ub


class Run:
    """A multi-step oracle run of one case (static or moving markers),
    mirroring the step order of the GPU library: dt from U^n, markers moved
    to t^{n+1}, quadrature, predictor, forcing."""

    def __init__(self, g, X_in, Tw_in, Ub_in=None, motion=None, dedup_markers: bool = True,
                 energy_reading: int = 0, tol: float = 1e-12):
        self.g = g
        X_in = _f64(X_in)
        if dedup_markers:
            rc, keep = dedup(g, X_in)
            if rc != 0:
                raise ValueError("marker outside the admissible region")
        else:
            keep = np.arange(len(X_in))
        self.keep = keep
        self.X0 = X_in[keep].copy()
        self.Tw = _f64(Tw_in)[keep].copy()
        self.Ub0 = None if Ub_in is None else _f64(Ub_in)[keep].copy()
        self.motion = motion
        self.energy_reading = energy_reading
        self.tol = tol
        self.t = 0.0
        self.X = self.X0.copy()
        self.Ub = self.Ub0
        rc, self.eps, self.cg_iters, self.cg_res = quadrature(g, self.X, tol=tol)
        if rc != 0:
            raise RuntimeError("oracle quadrature did not converge (res %g)" % self.cg_res)
        self.G = self.H = self.rhoL = None
        self.dt = None

    def step(self, U, dt_fixed: float = 0.0):
        g = self.g
        dtv = dt_fixed if dt_fixed > 0 else dt(g, U)
        if self.motion is not None:
            m = self.motion
            self.X, ub = motion(self.X0, m.amp, m.freq, m.axis, self.t + dtv)
            self.Ub = ub if self.Ub0 is None else ub + self.Ub0
            rc, self.eps, self.cg_iters, self.cg_res = quadrature(g, self.X, tol=self.tol,
                                                                  eps0=self.eps)
            if rc != 0:
                raise RuntimeError("oracle quadrature did not converge")
        d, Unew, self.G, self.H, self.rhoL = step(g, self.X, self.Ub, self.Tw, self.eps, U,
                                                  dt_fixed=dtv, energy_reading=self.energy_reading)
        self.t += dtv
        self.dt = dtv
        return Unew

    def forces(self):
        return forces(self.g, self.eps, self.G, self.H, self.Tw, self.dt)
