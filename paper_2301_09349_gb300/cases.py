"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds input *construction* only: grid descriptions, marker clouds,
the seeded density noise and the initial conserved state built from them.  It
contains none of the method's arithmetic (no delta kernel, no fluxes, no
forcing); both implementations receive the arrays produced here.

Workloads are shaped after the paper's test cases (heated cylinder of Sec. 3,
heated sphere of Sec. 4, oscillating cylinder of Sec. 5) on uniform Cartesian
grids.  Non-dimensionalisation: rho_inf = U_inf = T_inf = D = 1, so the gas
constant is r = 1/(gamma Ma^2), p_inf = 1/(gamma Ma^2) (perfect gas, Sec. 2.1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

# Boundary-condition codes, one per domain face (x-, x+, y-, y+, z-, z+).
BC_FREESTREAM = 0
BC_ZEROGRAD = 1
BC_SLIP = 2
BC_PERIODIC = 3

# Sutherland constant S = 110.4 K / 288.15 K in units of T_inf (Sec. 2.1 names
# Sutherland's law without constants).
SUTHERLAND_S = 110.4 / 288.15


@dataclasses.dataclass
class GridDesc:
    """Uniform Cartesian grid plus gas and scheme parameters."""
    dim: int
    n: tuple
    lo: tuple
    h: float
    fp_bytes: int = 4
    gamma: float = 1.4
    Pr: float = 0.72
    Re: float = 100.0          # Re <= 0 means inviscid (mu = 0)
    Mach: float = 0.3
    sutherland_S: float = SUTHERLAND_S
    cfl: float = 0.4
    bc: tuple = (BC_FREESTREAM, BC_ZEROGRAD, BC_SLIP, BC_SLIP, BC_SLIP, BC_SLIP)
    tile: tuple = (8, 8, 8)
    D: float = 1.0             # reference length (body diameter)
    forcing_per_stage: int = 0  # 1: force after each SSP-RK2 stage, not once per step

    @property
    def ncomp(self) -> int:
        return self.dim + 2

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n[: self.dim]))

    @property
    def hi(self) -> tuple:
        return tuple(self.lo[d] + self.n[d] * self.h for d in range(self.dim))

    def shape(self) -> tuple:
        """Storage shape of one conserved-state array: (ncomp, [nz,] ny, nx)."""
        return (self.ncomp,) + tuple(reversed(self.n[: self.dim]))


@dataclasses.dataclass
class Motion:
    """Prescribed marker motion X(t) = X(0) + amp sin(2 pi freq t) e_axis."""
    amp: float
    freq: float
    axis: int


@dataclasses.dataclass
class Case:
    name: str
    grid: GridDesc
    X: np.ndarray              # (n_markers, dim) float64 marker positions
    Tw: np.ndarray             # (n_markers,) float64 wall temperature / T_inf
    Ub: Optional[np.ndarray]   # (n_markers, dim) body velocity or None (= 0)
    motion: Optional[Motion]
    steps: int
    seed: int
    noise: float = 1e-3


# ---------------------------------------------------------------------------
# marker clouds
# ---------------------------------------------------------------------------

def circle_markers(n: int, radius: float = 0.5, center=(0.0, 0.0)) -> np.ndarray:
    """n markers equally spaced on a circle, theta_k = 2 pi k / n."""
    k = np.arange(n, dtype=np.float64)
    th = 2.0 * math.pi * k / n
    return np.stack([center[0] + radius * np.cos(th), center[1] + radius * np.sin(th)], axis=1)


def fibonacci_sphere_markers(n: int, radius: float = 0.5, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Fibonacci lattice: z_i = 1 - 2(i+1/2)/n, azimuth pi (1 + sqrt 5) i."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - 2.0 * (i + 0.5) / n
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    az = math.pi * (1.0 + math.sqrt(5.0)) * i
    pts = np.stack([rxy * np.cos(az), rxy * np.sin(az), z], axis=1)
    return pts * radius + np.asarray(center, dtype=np.float64)[None, :]


# ---------------------------------------------------------------------------
# initial state
# ---------------------------------------------------------------------------

def freestream_primitive(g: GridDesc):
    """(rho, velocity vector, pressure) of the free stream in the units above."""
    p_inf = 1.0 / (g.gamma * g.Mach * g.Mach)
    u = np.zeros(g.dim)
    u[0] = 1.0
    return 1.0, u, p_inf


def initial_state(g: GridDesc, seed: int, noise: float = 1e-3, dtype=None) -> np.ndarray:
    """Uniform free stream plus seeded Gaussian density noise.

    rho_j = 1 + noise * N(0,1) drawn by numpy PCG64(seed) in cell-linear order
    (x fastest); velocity and pressure are uniform, so temperature carries the
    perturbation.  Returned as the conserved state (rho, rho u, [rho v, rho w],
    rho E) with rho E = p/(gamma-1) + rho |u|^2 / 2, shape g.shape().
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    N = g.ncells
    rho = 1.0 + noise * rng.standard_normal(N)
    _, u, p = freestream_primitive(g)
    U = np.empty((g.ncomp, N), dtype=np.float64)
    U[0] = rho
    for d in range(g.dim):
        U[1 + d] = rho * u[d]
    U[g.dim + 1] = p / (g.gamma - 1.0) + 0.5 * rho * float(np.dot(u, u))
    U = U.reshape(g.shape())
    if dtype is not None:
        U = U.astype(dtype)
    return U


def random_state(g: GridDesc, seed: int, amp: float = 0.05) -> np.ndarray:
    """A smooth-ish random positive state (for operator tests): free stream with
    seeded perturbations of every primitive variable."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = g.ncells
    rho0, u0, p0 = freestream_primitive(g)
    rho = rho0 * (1.0 + amp * rng.standard_normal(N))
    u = [u0[d] + amp * rng.standard_normal(N) for d in range(g.dim)]
    p = p0 * (1.0 + amp * rng.standard_normal(N))
    U = np.empty((g.ncomp, N))
    U[0] = rho
    ke = np.zeros(N)
    for d in range(g.dim):
        U[1 + d] = rho * u[d]
        ke += u[d] * u[d]
    U[g.dim + 1] = p / (g.gamma - 1.0) + 0.5 * rho * ke
    return U.reshape(g.shape())


# ---------------------------------------------------------------------------
# the workloads (uniform-grid stand-ins for the paper's cases)
# ---------------------------------------------------------------------------

def _bc_for(dim: int, mach: float) -> tuple:
    side = BC_SLIP if mach < 1.0 else BC_ZEROGRAD
    bc = [BC_FREESTREAM, BC_ZEROGRAD, side, side, side, side]
    return tuple(bc)


def heated_cylinder(scale: int = 1, seed: int = 1) -> Case:
    """2D heated cylinder at rest: 128x64 over [-4,12]x[-4,4], 100 markers on
    r = 0.5, Ma 0.1, Re 40, T_w = 1.1, FP64 (Sec. 3 stand-in).  `scale`
    multiplies the resolution (tests use 1)."""
    n = (128 * scale, 64 * scale, 1)
    g = GridDesc(dim=2, n=n, lo=(-4.0, -4.0, 0.0), h=0.125 / scale, fp_bytes=8,
                 Re=40.0, Mach=0.1, bc=_bc_for(2, 0.1), tile=(16, 16, 1))
    X = circle_markers(100)
    return Case("heated_cylinder_128x64", g, X, np.full(len(X), 1.1), None, None, 200, seed)


def markers_at_cell_spacing(h: float, D: float = 1.0) -> int:
    """Fibonacci marker count whose mean spacing on a sphere of diameter D is
    one cell: surface area / h^2 (the paper's sphere has 12119 markers for
    pi D^2 / h^2 = 12868 at h = D/64, Sec. 4.1)."""
    return int(round(math.pi * D * D / (h * h)))


def heated_sphere(n: int = 256, mach: float = 0.3, Tw: float = 1.5,
                  n_markers: Optional[int] = None, seed: int = 2) -> Case:
    """3D heated sphere: n^3 over [-3,5]x[-4,4]^2, Fibonacci markers on r = 0.5
    at a spacing of about one cell (3217 at n = 256), Re 300, FP32 (Sec. 4
    stand-in).  n = 256 is the full workload."""
    h = 8.0 / n
    if n_markers is None:
        n_markers = markers_at_cell_spacing(h)
    g = GridDesc(dim=3, n=(n, n, n), lo=(-3.0, -4.0, -4.0), h=h, fp_bytes=4,
                 Re=300.0, Mach=mach, bc=_bc_for(3, mach), tile=(8, 8, 8))
    X = fibonacci_sphere_markers(n_markers)
    return Case(f"heated_sphere_{n}^3_Ma{mach}_Tw{Tw}", g, X, np.full(len(X), Tw), None, None,
                1000, seed)


def markers_at_arc_spacing(h: float, D: float = 1.0) -> int:
    """Markers on a circle of diameter D one cell apart along the arc:
    round(pi D / h) (101 at h = D/32).  A moving body keeps the marker set
    it starts with; at this spacing the set stays close to one marker per
    cell as it moves, where a denser set thinned to one per cell at t = 0
    ends up with up to 35 cells holding two markers, a near-singular A~ and
    a run that goes non-finite (measured on the transverse case)."""
    return int(round(math.pi * D / h))


def oscillating_cylinder(scale_div: int = 1, seed: int = 3) -> Case:
    """2D cylinder in transverse motion y(t) = 0.2 sin(2 pi 0.2 t): 1024x512 over
    [-8,24]x[-8,8], markers one cell apart on the circle (101), Ma 0.2,
    Re 100, T_w 1.2, FP32 (Sec. 5 stand-in).  `scale_div` divides the
    resolution for reduced-size tests."""
    n = (1024 // scale_div, 512 // scale_div, 1)
    h = (1.0 / 32.0) * scale_div
    g = GridDesc(dim=2, n=n, lo=(-8.0, -8.0, 0.0), h=h, fp_bytes=4,
                 Re=100.0, Mach=0.2, bc=_bc_for(2, 0.2), tile=(16, 16, 1))
    X = circle_markers(markers_at_arc_spacing(h))
    return Case(f"oscillating_cylinder_{n[0]}x{n[1]}", g, X, np.full(len(X), 1.2), None,
                Motion(amp=0.2, freq=0.2, axis=1), 5000, seed)


# Natural shedding Strouhal number f_0 D / U_inf of the fixed cylinder at Re
# 100, Ma 0.3: as in the paper (Sec. 5) it comes from a preliminary run of the
# fixed cylinder on the same kind of grid, here studies.fixed_cylinder_strouhal
# at h = D/16 (0.1801); it sets the streamwise forcing frequency f_c = 2 f_0.
ST0_RE100 = 0.180


def streamwise_oscillating_cylinder(scale_div: int = 1, f0: float = ST0_RE100,
                                    seed: int = 6) -> Case:
    """2D cylinder oscillating in the streamwise direction (Sec. 5):
    x(t) = x(0) + A sin(2 pi f_c t), A = 0.14 D, f_c = 2 f_0; Ma 0.3, Re 100,
    T_w = T_inf (temperature ratio 1); 1024x512 over [-8,24]x[-8,8], FP32.
    `scale_div` divides the resolution for reduced-size tests."""
    n = (1024 // scale_div, 512 // scale_div, 1)
    h = (1.0 / 32.0) * scale_div
    g = GridDesc(dim=2, n=n, lo=(-8.0, -8.0, 0.0), h=h, fp_bytes=4, Re=100.0, Mach=0.3,
                 bc=_bc_for(2, 0.3), tile=(16, 16, 1))
    X = circle_markers(markers_at_arc_spacing(h))
    return Case(f"streamwise_oscillating_cylinder_{n[0]}x{n[1]}", g, X, np.full(len(X), 1.0),
                None, Motion(amp=0.14, freq=2.0 * f0, axis=0), 5000, seed)


def adjoint_sphere(seed: int = 5) -> Case:
    """3D sphere 128^3 over [-3,5]x[-4,4]^2, Fibonacci markers at one-cell
    spacing (804), Ma 0.5, Re 100."""
    g = GridDesc(dim=3, n=(128, 128, 128), lo=(-3.0, -4.0, -4.0), h=1.0 / 16.0, fp_bytes=4,
                 Re=100.0, Mach=0.5, bc=_bc_for(3, 0.5), tile=(8, 8, 8))
    X = fibonacci_sphere_markers(markers_at_cell_spacing(g.h))
    return Case("adjoint_sphere_128^3", g, X, np.full(len(X), 1.5), None, None, 500, seed)


def sphere_variants(n: int = 256) -> list:
    """The four sphere runs: Mach in {0.3, 2.0} x T_w in {0.5, 1.5}."""
    out = []
    for i, (ma, tw) in enumerate([(0.3, 1.5), (0.3, 0.5), (2.0, 1.5), (2.0, 0.5)]):
        out.append(heated_sphere(n=n, mach=ma, Tw=tw, seed=2 + 10 * i))
    return out


def batched_cylinders(ncases: int = 64, sizes: Sequence[int] = (128, 256, 384, 512),
                      seed: int = 4, fp_bytes: int = 4) -> list:
    """A batch of independent 2D heated-cylinder cases of uneven size (a
    design-space sweep): case i draws, from PCG64(1000 * seed + i), a grid of
    n^2 cells with n from `sizes` over [-4,12]x[-8,8] (h = 16/n), 1 to 8
    cylinders of diameter 1 with centres uniform in [-2,6]x[-6,6] and every
    two centres at least 1.5 + 4h apart (a gap of at least half a diameter
    plus four cells), ceil(pi/h) markers per cylinder, T_w ~ U[0.5, 2],
    Ma ~ U[0.1, 0.5], Re ~ U[40, 200].  The initial state's noise seed is the
    case seed."""
    out = []
    for i in range(ncases):
        cs = 1000 * seed + i
        rng = np.random.Generator(np.random.PCG64(cs))
        n = int(sizes[int(rng.integers(len(sizes)))])
        h = 16.0 / n
        ncyl = int(rng.integers(1, 9))
        gap = 1.5 + 4.0 * h
        centres = []
        for _ in range(10000):
            if len(centres) == ncyl:
                break
            c = (float(rng.uniform(-2.0, 6.0)), float(rng.uniform(-6.0, 6.0)))
            if all(math.hypot(c[0] - q[0], c[1] - q[1]) >= gap for q in centres):
                centres.append(c)
        Tw = float(rng.uniform(0.5, 2.0))
        mach = float(rng.uniform(0.1, 0.5))
        Re = float(rng.uniform(40.0, 200.0))
        g = GridDesc(dim=2, n=(n, n, 1), lo=(-4.0, -8.0, 0.0), h=h, fp_bytes=fp_bytes, Re=Re,
                     Mach=mach, bc=_bc_for(2, mach), tile=(16, 16, 1))
        nm = int(math.ceil(math.pi / h))
        X = np.concatenate([circle_markers(nm, 0.5, c) for c in centres], axis=0)
        out.append(Case(f"batch{seed}_case{i}_{n}^2_{len(centres)}cyl", g, X, np.full(len(X), Tw),
                        None, None, 1000, cs))
    return out


def small_grid(dim: int, n: Sequence[int], h: float = 0.125, lo=None, fp_bytes: int = 8,
               bc=None, Re: float = 100.0, Mach: float = 0.3, tile=None) -> GridDesc:
    """A small grid for operator tests."""
    if lo is None:
        lo = tuple(-0.5 * n[d] * h for d in range(dim)) + (0.0,) * (3 - dim)
    n3 = tuple(n) + (1,) * (3 - len(n))
    if bc is None:
        bc = _bc_for(dim, Mach)
    if tile is None:
        tile = (8, 8, 8) if dim == 3 else (16, 16, 1)
    return GridDesc(dim=dim, n=n3, lo=tuple(lo) + (0.0,) * (3 - len(lo)), h=h, fp_bytes=fp_bytes,
                    Re=Re, Mach=Mach, bc=tuple(bc), tile=tuple(tile))


def random_markers(g: GridDesc, n: int, seed: int, margin_cells: float = 2.5) -> np.ndarray:
    """n markers uniform in the grid minus a margin of `margin_cells` cells."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.array(g.lo[: g.dim]) + margin_cells * g.h
    hi = np.array(g.hi[: g.dim]) - margin_cells * g.h
    return lo + (hi - lo) * rng.random((n, g.dim))
