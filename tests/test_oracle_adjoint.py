"""Pins of the oracle's discrete adjoint (oracle/adjoint.py) to things other
than itself: its forward map equals the C oracle's step to round-off, its
flux transpose-Jacobian product equals central differences of the C oracle's
L(U), and its gradient of J = a C_d + b Nu equals central finite differences
of the C oracle's J with respect to marker positions and wall temperatures.
Perturbations are small enough (1e-6) that no marker crosses a cell face."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint as A
from paper_2301_09349_gb300 import cases as C


def cyl_case(n=(40, 32), h=0.1, fp=8, seed=3, Tw=1.4, mach=0.3, bc=None):
    g = C.small_grid(2, n, h=h, fp_bytes=fp, Re=100.0, Mach=mach, bc=bc)
    X = C.circle_markers(int(np.ceil(np.pi / h)), 0.5, (0.05, -0.03))
    return g, X, np.full(len(X), Tw), seed


def kept(oracle, g, X):
    rc, keep = oracle.dedup(g, X)
    assert rc == 0
    return X[keep]


@pytest.mark.parametrize("bc", ["default", "periodic"])
def test_torch_forward_equals_c_oracle(oracle, bc):
    bcs = None if bc == "default" else (C.BC_PERIODIC,) * 6
    g, X, Tw, seed = cyl_case(bc=bcs)
    X = kept(oracle, g, X)
    Tw = Tw[: len(X)]
    U0 = C.initial_state(g, seed)
    dt = oracle.dt(g, U0)
    U, G, H, eps = A.run(g, torch.tensor(X), torch.tensor(Tw), U0, [dt, dt])
    eps_c = np.linalg.solve(oracle.assemble_A_dense(g, X), np.ones(len(X)))
    assert np.max(np.abs(eps.numpy() - eps_c) / eps_c) < 1e-12
    Uc = U0
    for _ in range(2):
        _, Uc, Gc, Hc, _ = oracle.step(g, X, None, Tw, eps_c, Uc, dt_fixed=dt)
    Ut = U.detach().numpy().reshape(Uc.shape)
    assert np.linalg.norm(Ut - Uc) / np.linalg.norm(Uc) < 1e-13
    assert np.max(np.abs(G.detach().numpy() - Gc)) < 1e-12 * max(1.0, np.abs(Gc).max())
    assert np.max(np.abs(H.detach().numpy() - Hc)) < 1e-11 * max(1.0, np.abs(Hc).max())


def test_torch_forward_3d_equals_c_oracle(oracle):
    g = C.small_grid(3, (16, 14, 12), h=0.125, fp_bytes=8, Re=80.0, Mach=0.4)
    X = kept(oracle, g, C.fibonacci_sphere_markers(150, 0.45))
    Tw = np.full(len(X), 0.7)
    U0 = C.initial_state(g, 5)
    dt = oracle.dt(g, U0)
    U, _, _, eps = A.run(g, torch.tensor(X), torch.tensor(Tw), U0, [dt])
    _, Uc, _, _, _ = oracle.step(g, X, None, Tw, eps.detach().numpy(), U0, dt_fixed=dt)
    Ut = U.detach().numpy().reshape(Uc.shape)
    assert np.linalg.norm(Ut - Uc) / np.linalg.norm(Uc) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_rhs_vjp_matches_central_differences(oracle, dim):
    if dim == 2:
        g = C.small_grid(2, (13, 11), h=0.1, fp_bytes=8, Re=60.0, Mach=0.4)
    else:
        g = C.small_grid(3, (7, 6, 5), h=0.1, fp_bytes=8, Re=60.0, Mach=0.4,
                         bc=(C.BC_FREESTREAM, C.BC_ZEROGRAD, C.BC_SLIP, C.BC_SLIP,
                             C.BC_PERIODIC, C.BC_PERIODIC))
    U = C.random_state(g, seed=17, amp=0.05)
    rng = np.random.default_rng(2)
    v = rng.standard_normal(U.shape)
    vjp = A.rhs_vjp(g, U, v)
    for trial in range(3):
        w = rng.standard_normal(U.shape) * np.abs(U).mean(axis=tuple(range(1, U.ndim)),
                                                         keepdims=True)
        d = 1e-6
        fd = np.sum(v * (oracle.rhs(g, U + d * w) - oracle.rhs(g, U - d * w))) / (2 * d)
        ad = np.sum(vjp * w)
        assert abs(ad - fd) <= 1e-6 * abs(fd), (trial, ad, fd)


def _fd_check(oracle, g, X, Tw, U0, dts, a, b, n_checks, seed):
    J, gX, gT = A.gradient(g, X, Tw, U0, dts, a, b)
    Jc = A.objective_c(g, X, Tw, U0, dts, a, b)
    assert abs(J - Jc) <= 1e-12 * abs(Jc)
    rng = np.random.default_rng(seed)
    d = 1e-6
    scale = np.abs(gX).max()
    for _ in range(n_checks):
        k = int(rng.integers(len(X)))
        ax = int(rng.integers(g.dim))
        Xp, Xm = X.copy(), X.copy()
        Xp[k, ax] += d
        Xm[k, ax] -= d
        fd = (A.objective_c(g, Xp, Tw, U0, dts, a, b) -
              A.objective_c(g, Xm, Tw, U0, dts, a, b)) / (2 * d)
        assert abs(gX[k, ax] - fd) <= 1e-7 * scale + 1e-6 * abs(fd), (k, ax, gX[k, ax], fd)
    scale = np.abs(gT).max()
    for _ in range(n_checks // 2):
        k = int(rng.integers(len(X)))
        Tp, Tm = Tw.copy(), Tw.copy()
        Tp[k] += d
        Tm[k] -= d
        fd = (A.objective_c(g, X, Tp, U0, dts, a, b) -
              A.objective_c(g, X, Tm, U0, dts, a, b)) / (2 * d)
        assert abs(gT[k] - fd) <= 1e-7 * scale + 1e-6 * abs(fd), (k, gT[k], fd)
    return gX, gT


def test_gradient_matches_central_differences_2d(oracle):
    g, X, Tw, seed = cyl_case()
    X = kept(oracle, g, X)
    Tw = np.linspace(1.2, 1.6, len(X))
    U0 = C.initial_state(g, seed)
    dt = oracle.dt(g, U0)
    _fd_check(oracle, g, X, Tw, U0, [dt, 0.9 * dt, dt], 1.0, 0.3, 12, 1)


def test_gradient_matches_central_differences_3d(oracle):
    g = C.small_grid(3, (12, 12, 12), h=0.125, fp_bytes=8, Re=80.0, Mach=0.4)
    X = kept(oracle, g, C.fibonacci_sphere_markers(120, 0.4))
    Tw = np.full(len(X), 1.5)
    U0 = C.initial_state(g, 9)
    dt = oracle.dt(g, U0)
    _fd_check(oracle, g, X, Tw, U0, [dt, dt], 0.5, 1.0, 6, 4)


def _capped_cells(oracle, g, X, Tw, U0):
    """cells whose heat source the cap limits in the first step"""
    run = oracle.Run(g, X, Tw, dedup_markers=False)
    _, Us = oracle.predictor(g, U0)
    Un = run.step(U0)
    nc = g.ncomp

    def internal(U):
        U = U.reshape(nc, -1)
        return U[-1] - 0.5 * (U[1:nc - 1] ** 2).sum(0) / U[0]
    return int(np.sum(np.isclose(internal(Un) / internal(Us), 0.1, rtol=1e-12)))


@pytest.mark.parametrize("energy_reading", [0, 1])
def test_forward_and_gradient_with_the_heat_source_cap(oracle, energy_reading):
    """A cold wall (T_w 0.25-0.35 at Mach 0.3) whose cooling the heat-source
    cap limits in a dozen forced cells: the torch restatement equals the C
    oracle's states, and its gradient equals central differences of the C
    oracle's J (the cap is a max, differentiated on its branch)."""
    g, X, _, seed = cyl_case()
    X = kept(oracle, g, X)
    Tw = np.linspace(0.25, 0.35, len(X))
    U0 = C.initial_state(g, seed)
    assert _capped_cells(oracle, g, X, Tw, U0) >= 10
    dt = oracle.dt(g, U0)
    U, G, H, eps = A.run(g, torch.tensor(X), torch.tensor(Tw), U0, [dt, dt],
                         energy_reading=energy_reading)
    Uc = U0
    for _ in range(2):
        _, Uc, _, _, _ = oracle.step(g, X, None, Tw, eps.detach().numpy(), Uc, dt_fixed=dt,
                                     energy_reading=energy_reading)
    Ut = U.detach().numpy().reshape(Uc.shape)
    assert np.linalg.norm(Ut - Uc) / np.linalg.norm(Uc) < 1e-13
    if energy_reading == 0:
        _fd_check(oracle, g, X, Tw, U0, [dt, dt], 1.0, 0.3, 8, 7)
