"""Studies run on the CUDA path (host drivers only; every step runs in the
library's kernels).

self_convergence(): C_d of the heated cylinder (Re 40, Ma 0.1, T_w 1.1) at a
fixed time T on grids h = D/8, D/16, ... (App. C reports the L_inf error
against grid refinement with an order close to 2); each grid takes the
largest step size that keeps the CFL bound and reaches T in a whole number of
steps, so every grid stops at the same time.  The observed order between
three successive grids is log2(|C(h) - C(h/2)| / |C(h/2) - C(h/4)|).

fixed_cylinder_strouhal(): the natural shedding Strouhal number of the fixed
cylinder at the parameters of the paper's oscillating-cylinder study (Sec. 5:
Ma 0.3, Re 100, temperature ratio 1), from the lift history (diagnostics).
"""
from __future__ import annotations

import math

import numpy as np

from . import cases as C
from . import diagnostics, ibm


def _cylinder(div: int, Re: float, Mach: float, Tw: float, lo, extent, fp_bytes: int):
    h = 1.0 / div
    n = (int(round(extent[0] / h)), int(round(extent[1] / h)), 1)
    g = C.GridDesc(dim=2, n=n, lo=(lo[0], lo[1], 0.0), h=h, fp_bytes=fp_bytes, Re=Re,
                   Mach=Mach, bc=C._bc_for(2, Mach), tile=(16, 16, 1))
    X = C.circle_markers(int(math.ceil(math.pi / h)))
    return g, X, np.full(len(X), Tw)


def self_convergence(divs=(8, 16, 32, 64), T: float = 2.0, fp_bytes: int = 4, seed: int = 1):
    """[(D/h, steps, C_d(T), Nu(T))] and the observed orders"""
    rows = []
    for div in divs:
        g, X, Tw = _cylinder(div, 40.0, 0.1, 1.1, (-4.0, -4.0), (16.0, 8.0), fp_bytes)
        grid = ibm.Grid(g, max_markers=len(X))
        grid.set_markers(X, Tw)
        U0 = C.initial_state(g, seed, noise=0.0)
        grid.set_state(U0.astype(np.float32 if fp_bytes == 4 else np.float64))
        grid.step(1)
        dt0 = grid.time()[0]
        grid.set_state(U0.astype(np.float32 if fp_bytes == 4 else np.float64))
        nsteps = int(math.ceil(T / (0.8 * dt0)))
        grid.step(nsteps, dt_fixed=T / nsteps)
        f = grid.forces()
        rows.append((div, nsteps, f["Cd"], f["Nu"]))
        grid.close()
    cd = [r[2] for r in rows]
    orders = []
    for i in range(len(cd) - 2):
        a, b = abs(cd[i] - cd[i + 1]), abs(cd[i + 1] - cd[i + 2])
        orders.append(math.log2(a / b) if a > 0 and b > 0 else float("nan"))
    return rows, orders


def fixed_cylinder_strouhal(div: int = 16, t_end: float = 250.0, t_min: float = 120.0,
                            every: int = 10, seed: int = 6):
    """(St, t, C_l) of the fixed cylinder at Ma 0.3, Re 100, T_w = T_inf"""
    g, X, Tw = _cylinder(div, 100.0, 0.3, 1.0, (-8.0, -8.0), (32.0, 16.0), 4)
    grid = ibm.Grid(g, max_markers=len(X))
    grid.set_markers(X, Tw)
    grid.set_state(C.initial_state(g, seed).astype(np.float32))
    ts, cls = [], []
    t = 0.0
    while t < t_end:
        grid.step(every)
        _, t, _ = grid.time()
        ts.append(t)
        cls.append(grid.forces()["Cl"])
    grid.close()
    return diagnostics.strouhal(ts, cls, t_min=t_min), np.array(ts), np.array(cls)
