"""GPU: the discrete adjoint (ibm_record / ibm_backward / ibm_rhs_vjp)
against the oracle's adjoint (oracle/adjoint.py: the oracle's step restated
in PyTorch FP64 and differentiated by reverse mode, itself pinned to the C
oracle and to finite differences in tests/test_oracle_adjoint.py).

Tolerances.  FP64 grids: the CUDA reverse sweep and the oracle's autograd
evaluate the same derivative with different rounding order, and the GPU's
weights come from CG to 1e-12 rather than a dense solve, so gradients agree
to ~1e-9 of their largest entry (gate 1e-7).  FP32 grids: the forward
trajectory itself carries FP32 rounding (~1e-7 relative per step, amplified
by the flux cancellation), the reverse sweep runs in FP32 with FP64
accumulators; gate 2e-3 of the largest entry.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2301_09349_gb300 import cases as C
from paper_2301_09349_gb300 import ibm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup(oracle):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2301_09349_gb300 import build
    build.build()
    oracle.set_threads(os.cpu_count() or 1)


def adj():
    from oracle import adjoint
    return adjoint


MIXED = (C.BC_FREESTREAM, C.BC_ZEROGRAD, C.BC_SLIP, C.BC_SLIP, C.BC_PERIODIC, C.BC_PERIODIC)


@pytest.mark.parametrize("dim,fp,tol", [(2, 8, 1e-11), (3, 8, 1e-11), (2, 4, 2e-4), (3, 4, 2e-4)])
@pytest.mark.parametrize("bc", ["mixed", "periodic", "default"])
def test_rhs_vjp_matches_oracle(dim, fp, tol, bc):
    n = (13, 11) if dim == 2 else (9, 7, 6)
    bcs = {"mixed": MIXED, "periodic": (C.BC_PERIODIC,) * 6, "default": None}[bc]
    g = C.small_grid(dim, n, h=0.1, fp_bytes=fp, Re=60.0, Mach=0.4, bc=bcs)
    U = C.random_state(g, seed=23, amp=0.05)
    rng = np.random.default_rng(5)
    V = rng.standard_normal(U.shape)
    dt_ = np.float32 if fp == 4 else np.float64
    U = U.astype(dt_)
    V = V.astype(dt_)
    grid = ibm.Grid(g)
    grid.record(1, 1)
    out = grid.rhs_vjp(torch.from_numpy(U), torch.from_numpy(V)).cpu().numpy()
    ref = adj().rhs_vjp(g, U.astype(np.float64), V.astype(np.float64))
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert err < tol, err


@pytest.mark.parametrize("dim,fp,tol", [(2, 8, 1e-11), (3, 8, 1e-11), (2, 4, 2e-4)])
def test_rhs_vjp_inviscid_matches_oracle(dim, fp, tol):
    n = (13, 11) if dim == 2 else (9, 7, 6)
    g = C.small_grid(dim, n, h=0.1, fp_bytes=fp, Re=0.0, Mach=0.6, bc=MIXED)
    U = C.random_state(g, seed=29, amp=0.05)
    V = np.random.default_rng(6).standard_normal(U.shape)
    dt_ = np.float32 if fp == 4 else np.float64
    grid = ibm.Grid(g)
    grid.record(1, 1)
    out = grid.rhs_vjp(torch.from_numpy(U.astype(dt_)), torch.from_numpy(V.astype(dt_))).cpu().numpy()
    ref = adj().rhs_vjp(g, U.astype(dt_).astype(np.float64), V.astype(dt_).astype(np.float64))
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < tol


def cylinder(fp, n=(40, 32), h=0.1):
    g = C.small_grid(2, n, h=h, fp_bytes=fp, Re=100.0, Mach=0.3)
    X = C.circle_markers(int(np.ceil(np.pi / h)), 0.5, (0.05, -0.03))
    return g, X, np.linspace(1.2, 1.6, len(X)), 3


def gpu_gradient(g, X, Tw, seed, steps, every, a, b, energy_reading=0):
    grid = ibm.Grid(g, max_markers=len(X), energy_reading=energy_reading)
    grid.set_markers(X, Tw)
    U0 = C.initial_state(g, seed)
    U0 = U0.astype(np.float32 if g.fp_bytes == 4 else np.float64)
    grid.set_state(U0)
    grid.record(steps, every)
    dts = []
    for _ in range(steps):
        grid.step(1)
        dts.append(grid.time()[0])
    f = grid.forces()
    J = a * f["Cd"] + b * f["Nu"]
    Xk, _, idx = grid.markers()
    U_end = grid.get_state().cpu().numpy()
    gX, gT = grid.backward(a, b)
    # the handle's state and forcing are left as they were
    assert np.array_equal(grid.get_state().cpu().numpy(), U_end)
    f2 = grid.forces()
    assert f2["Cd"] == f["Cd"] and f2["heat_rate"] == f["heat_rate"]
    return J, gX, gT, Xk, np.asarray(Tw)[idx], U0.astype(np.float64), dts


def compare(g, X, Tw, seed, steps, every, a, b, tol, energy_reading=0):
    J, gX, gT, Xk, Twk, U0, dts = gpu_gradient(g, X, Tw, seed, steps, every, a, b,
                                               energy_reading)
    Jo, oX, oT = adj().gradient(g, Xk, Twk, U0, dts, a, b, energy_reading=energy_reading)
    assert abs(J - Jo) <= max(tol, 1e-9) * abs(Jo)
    ex = np.abs(gX - oX).max() / np.abs(oX).max()
    et = np.abs(gT - oT).max() / np.abs(oT).max()
    assert ex < tol and et < tol, (ex, et)
    return ex, et


def test_backward_fp64_2d_matches_oracle():
    g, X, Tw, seed = cylinder(8)
    compare(g, X, Tw, seed, steps=3, every=2, a=1.0, b=0.3, tol=1e-7)


def test_backward_fp64_2d_energy_reading_total():
    g, X, Tw, seed = cylinder(8)
    compare(g, X, Tw, seed, steps=2, every=1, a=0.5, b=1.0, tol=1e-7, energy_reading=1)


def test_backward_fp64_2d_many_steps_with_checkpoints():
    g, X, Tw, seed = cylinder(8, n=(36, 28), h=0.125)
    compare(g, X, Tw, seed, steps=12, every=5, a=1.0, b=0.2, tol=1e-7)


@pytest.mark.parametrize("energy_reading", [0, 1])
def test_backward_fp64_2d_with_the_heat_source_cap(energy_reading):
    """A cold wall (T_w 0.25-0.35 at Mach 0.3) whose cooling the heat-source
    cap limits in a dozen forced cells (counted in the oracle's pins): the
    reverse of the capped update against the oracle's autograd."""
    g, X, _, seed = cylinder(8)
    Tw = np.linspace(0.25, 0.35, len(X))
    compare(g, X, Tw, seed, steps=3, every=2, a=1.0, b=0.3, tol=1e-7,
            energy_reading=energy_reading)


def test_backward_fp64_3d_matches_oracle(oracle):
    g = C.small_grid(3, (12, 12, 12), h=0.125, fp_bytes=8, Re=80.0, Mach=0.4)
    X = C.fibonacci_sphere_markers(120, 0.4)
    compare(g, X, np.full(len(X), 1.5), 9, steps=2, every=1, a=0.5, b=1.0, tol=1e-7)


def test_backward_at_the_configured_cadence():
    """A checkpoint every 50 of 100 recorded steps (the benchmark's cadence:
    two replayed segments) on a 12^3 box in FP64 against the oracle's
    autograd over the same 100 steps."""
    g = C.small_grid(3, (12, 12, 12), h=0.125, fp_bytes=8, Re=80.0, Mach=0.4)
    X = C.fibonacci_sphere_markers(120, 0.4)
    compare(g, X, np.full(len(X), 1.5), 9, steps=100, every=50, a=0.5, b=1.0, tol=1e-7)


@pytest.mark.parametrize("fp", [4, 8])
def test_backward_is_bitwise_reproducible(fp):
    """The flux transpose sums every cell's stencil contributions in a fixed
    order (no float atomics), so two reverse sweeps of one recording, and the
    sweep of a second handle that recorded the same run, agree bit for bit."""
    g = C.small_grid(3, (20, 18, 16), h=0.1, fp_bytes=fp, Re=80.0, Mach=0.4)
    X = C.fibonacci_sphere_markers(200, 0.5)
    dt_ = np.float32 if fp == 4 else np.float64
    outs = []
    for _ in range(2):
        grid = ibm.Grid(g, max_markers=len(X))
        grid.set_markers(X, np.full(len(X), 1.4))
        grid.set_state(C.initial_state(g, 13).astype(dt_))
        grid.record(6, 3)
        grid.step(6)
        first = grid.backward(1.0, 0.5)
        second = grid.backward(1.0, 0.5)
        for a_, b_ in zip(first, second):
            np.testing.assert_array_equal(a_, b_)
        outs.append(first)
        grid.close()
    for a_, b_ in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a_, b_)


def test_backward_fp32_2d_matches_oracle():
    g, X, Tw, seed = cylinder(4)
    compare(g, X, Tw, seed, steps=3, every=2, a=1.0, b=0.3, tol=2e-3)


def test_backward_fp32_3d_matches_oracle():
    g = C.small_grid(3, (16, 16, 12), h=0.125, fp_bytes=4, Re=80.0, Mach=0.4)
    X = C.fibonacci_sphere_markers(150, 0.45)
    compare(g, X, np.full(len(X), 0.7), 11, steps=2, every=2, a=1.0, b=0.5, tol=2e-3)


def test_backward_matches_gpu_finite_differences():
    """Central differences (h = 1e-6) of the GPU's own J in FP64 with the
    recorded step sizes held fixed, on 32 seeded (marker, axis) draws whose
    shift keeps the marker in its owner cell (so the bins do not change) and
    16 wall temperatures.  The 32 markers are few enough for the direct
    (Cholesky) quadrature solve, so eps~ moves smoothly with X and the
    differences are clean: gate 1e-4 relative, with an absolute floor of 1e-6
    of the largest entry for entries near zero."""
    g, X, Tw, seed = cylinder(8)
    a, b = 1.0, 0.3
    _, gX, gT, Xk, Twk, U0, dts = gpu_gradient(g, X, Tw, seed, 3, 2, a, b)

    def J_of(Xp, Twp):
        gr = ibm.Grid(g, max_markers=len(Xp))
        gr.set_markers(Xp, Twp, dedup=False)
        gr.set_state(U0)
        for dt in dts:
            gr.step(1, dt_fixed=dt)
        f = gr.forces()
        gr.close()
        return a * f["Cd"] + b * f["Nu"]

    lo = np.array(g.lo[:2])
    rng = np.random.default_rng(7)
    d = 1e-6
    done = 0
    while done < 32:
        k, ax = int(rng.integers(len(Xk))), int(rng.integers(2))
        cell = np.floor((Xk[k, ax] - lo[ax]) / g.h)
        if (np.floor((Xk[k, ax] + d - lo[ax]) / g.h) != cell or
                np.floor((Xk[k, ax] - d - lo[ax]) / g.h) != cell):
            continue
        Xp, Xm = Xk.copy(), Xk.copy()
        Xp[k, ax] += d
        Xm[k, ax] -= d
        fd = (J_of(Xp, Twk) - J_of(Xm, Twk)) / (2 * d)
        assert abs(gX[k, ax] - fd) <= 1e-4 * abs(fd) + 1e-6 * np.abs(gX).max(), \
            (k, ax, gX[k, ax], fd)
        done += 1
    for _ in range(16):
        k = int(rng.integers(len(Xk)))
        Tp, Tm = Twk.copy(), Twk.copy()
        Tp[k] += d
        Tm[k] -= d
        fd = (J_of(Xk, Tp) - J_of(Xk, Tm)) / (2 * d)
        assert abs(gT[k] - fd) <= 1e-4 * abs(fd) + 1e-6 * np.abs(gT).max(), (k, gT[k], fd)


def test_backward_at_the_benchmark_size_matches_central_differences():
    """The 128^3 adjoint sphere (804 markers, 698 kept) in FP64, 20 recorded
    steps with a checkpoint every 10 (two replayed segments): central
    differences of the GPU's own J with the recorded step sizes held fixed,
    on 32 seeded (marker, axis) draws that keep the marker in its owner cell
    and 16 wall temperatures; gate 1e-4 relative with a floor of 1e-6 of the
    largest entry.  J is only piecewise smooth here: 20 steps after the
    impulsive start, limiter and Rusanov-max switches sit within 1e-6 of some
    draws, so the step is h = 1e-7, where the central differences resolve
    the local branch and the FP64 rounding of J (~1e-13) stays below 1e-5 of
    the entries.  Where a switch sits exactly at the point (a tie such as a
    slope that is exactly zero), J has a kink there: its one-sided slopes
    differ at every h, the central difference is their mean, and the adjoint
    is one of them (a one-sided derivative of the discrete scheme).  Such a
    draw is accepted when the one-sided slopes at h = 1e-6 differ well above
    their rounding and the adjoint matches one of them; at most a few per
    kind.  The weights are solved to a residual of 1e-14
    (ibm_set_quadrature) to keep the solver's own noise out too."""
    import dataclasses
    c = C.adjoint_sphere()
    g = dataclasses.replace(c.grid, fp_bytes=8)
    a, b = 1.0, 0.5
    tol = 1e-14
    U0 = C.initial_state(g, c.seed)
    grid = ibm.Grid(g, max_markers=len(c.X))
    grid.set_quadrature(tol, 20000)
    grid.set_markers(c.X, c.Tw)
    grid.set_state(U0)
    grid.record(20, 10)
    dts = []
    for _ in range(20):
        grid.step(1)
        dts.append(grid.time()[0])
    Xk, _, idx = grid.markers()
    Twk = np.asarray(c.Tw)[idx]
    gX, gT = grid.backward(a, b)
    grid.close()

    def J_of(Xp, Twp):
        gr = ibm.Grid(g, max_markers=len(Xp))
        gr.set_quadrature(tol, 20000)
        gr.set_markers(Xp, Twp, dedup=False)
        gr.set_state(U0)
        for dt in dts:
            gr.step(1, dt_fixed=dt)
        f = gr.forces()
        gr.close()
        return a * f["Cd"] + b * f["Nu"]

    lo = np.array(g.lo[:3])
    rng = np.random.default_rng(11)
    d, d1 = 1e-7, 1e-6
    J0 = []

    def check(adj, pm, scale, what):
        """the adjoint entry against the central difference, or against a
        one-sided slope where J has a kink at the point; True for a kink"""
        jp, jm = pm(d)
        fd = (jp - jm) / (2 * d)
        gate = lambda ref: 1e-4 * abs(ref) + 1e-6 * scale
        if abs(adj - fd) <= gate(fd):
            return False
        if not J0:
            J0.append(J_of(Xk, Twk))
        jp, jm = pm(d1)
        fwd, bwd = (jp - J0[0]) / d1, (J0[0] - jm) / d1
        assert abs(fwd - bwd) > 5 * gate(fd), (what, adj, fd, fwd, bwd)
        assert min(abs(adj - fwd), abs(adj - bwd)) <= gate(fd), (what, adj, fd, fwd, bwd)
        return True

    def x_pm(k, ax):
        def f(h):
            Xp, Xm = Xk.copy(), Xk.copy()
            Xp[k, ax] += h
            Xm[k, ax] -= h
            return J_of(Xp, Twk), J_of(Xm, Twk)
        return f

    def tw_pm(k):
        def f(h):
            Tp, Tm = Twk.copy(), Twk.copy()
            Tp[k] += h
            Tm[k] -= h
            return J_of(Xk, Tp), J_of(Xk, Tm)
        return f

    done = kinks = 0
    while done < 32:
        k, ax = int(rng.integers(len(Xk))), int(rng.integers(3))
        cell = np.floor((Xk[k, ax] - lo[ax]) / g.h)
        if (np.floor((Xk[k, ax] + d1 - lo[ax]) / g.h) != cell or
                np.floor((Xk[k, ax] - d1 - lo[ax]) / g.h) != cell):
            continue
        kinks += check(gX[k, ax], x_pm(k, ax), np.abs(gX).max(), (k, ax))
        done += 1
    assert kinks <= 4, kinks
    kinks = 0
    for k in rng.choice(len(Xk), 16, replace=False):
        kinks += check(gT[k], tw_pm(int(k)), np.abs(gT).max(), int(k))
    assert kinks <= 2, kinks


def test_autograd_function_returns_the_adjoint_gradient():
    g, X, Tw, seed = cylinder(8)
    U0 = C.initial_state(g, seed)
    grid = ibm.Grid(g, max_markers=len(X))
    Xt = torch.tensor(X, requires_grad=True)
    Tt = torch.tensor(Tw, requires_grad=True)
    J = ibm.cd_nu_objective().apply(Xt, Tt, grid, U0, 3, 1.0, 0.3, 2)
    (2.0 * J).backward()
    ref = ibm.Grid(g, max_markers=len(X))
    ref.set_markers(X, Tw)
    ref.set_state(U0)
    ref.record(3, 2)
    ref.step(3)
    f = ref.forces()
    assert float(J) == 1.0 * f["Cd"] + 0.3 * f["Nu"]
    gX, gT = ref.backward(1.0, 0.3)
    _, _, idx = ref.markers()
    # the reverse sweep is bitwise reproducible: the autograd wrapper returns
    # exactly twice the direct call's gradient
    np.testing.assert_array_equal(Xt.grad.numpy()[idx], 2.0 * gX)
    np.testing.assert_array_equal(Tt.grad.numpy()[idx], 2.0 * gT)
    dropped = np.setdiff1d(np.arange(len(X)), idx)
    assert np.all(Xt.grad.numpy()[dropped] == 0.0)


def test_adjoint_errors():
    g, X, Tw, seed = cylinder(8)
    grid = ibm.Grid(g, max_markers=len(X))
    grid.set_markers(X, Tw)
    grid.set_state(C.initial_state(g, seed))
    with pytest.raises(ibm.IbmError) as e:
        grid.backward(1.0, 0.0)
    assert e.value.status == 7
    nb = ibm.ibm_adjoint_workspace_bytes(grid.desc, len(X), 4, 2)
    assert nb > 0 and ibm.ibm_adjoint_workspace_bytes(grid.desc, len(X), 0, 2) == 0
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    ptr = (ws.data_ptr() + 255) // 256 * 256
    with pytest.raises(ibm.IbmError) as e:
        ibm.ibm_record(grid.h, 4, 2, ptr, nb - 1024)
    assert e.value.status == 5
    ibm.ibm_record(grid.h, 4, 2, ptr, nb)
    with pytest.raises(ibm.IbmError) as e:
        grid.step(5)
    assert e.value.status == 5
    grid.step(2)
    gX, gT = grid.backward(1.0, 0.0)
    assert np.all(np.isfinite(gX)) and np.all(np.isfinite(gT))
    # Nu is undefined on an inviscid grid: weighting it is an argument error
    gi = C.small_grid(2, (40, 32), h=0.1, fp_bytes=8, Re=0.0, Mach=0.3)
    inv = ibm.Grid(gi, max_markers=len(X))
    inv.set_markers(X, Tw)
    inv.set_state(C.initial_state(gi, seed))
    inv.record(2, 1)
    inv.step(1)
    with pytest.raises(ibm.IbmError) as e:
        inv.backward(0.0, 1.0)
    assert e.value.status == 1
    gX, gT = inv.backward(1.0, 0.0)          # drag alone is fine
    assert np.all(np.isfinite(gX))
    mov = ibm.Grid(g, max_markers=len(X))
    mov.set_markers(X, Tw, motion=C.Motion(0.05, 1.0, 1))
    mov.set_state(C.initial_state(g, seed))
    with pytest.raises(ibm.IbmError) as e:
        mov.record(4, 2)
    assert e.value.status == 8


def test_backward_at_the_benchmark_size_fp32_equals_fp64():
    """The 128^3 adjoint workload (804 markers, 698 kept), 4 recorded steps
    over two checkpoint segments, in FP32 (the benchmark) and in FP64 (the
    path pinned to the oracle at small sizes): the gradients agree to 1e-4
    of their largest entries.  (Central differences are no check at this
    size: after the impulsive start, any finite change of T_w crosses
    limiter and Rusanov-max switches, and the differences drift with the
    step - 0.054 at +-0.05, 0.046 at +-0.01 for a gradient entry of 0.0446 -
    in FP32 and FP64 alike.)"""
    import dataclasses
    c = C.adjoint_sphere()
    out = {}
    for fp in (4, 8):
        g = dataclasses.replace(c.grid, fp_bytes=fp)
        _, gX, gT, Xk, _, _, _ = gpu_gradient(g, c.X, c.Tw, c.seed, 4, 2, 1.0, 0.5)
        out[fp] = (gX, gT, Xk)
    assert np.array_equal(out[4][2], out[8][2])
    for i in (0, 1):
        a32, a64 = out[4][i], out[8][i]
        assert np.abs(a32 - a64).max() <= 1e-4 * np.abs(a64).max(), (i, np.abs(a32 - a64).max())
