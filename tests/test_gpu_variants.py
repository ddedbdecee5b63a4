"""GPU: the method variants and diagnostics - surface pressure coefficient,
the streamwise-oscillating cylinder of Sec. 5, the self-convergence of C_d
(App. C) and the fixed cylinder's shedding Strouhal number."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2301_09349_gb300 import cases as C
from paper_2301_09349_gb300 import ibm, studies

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup(oracle):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2301_09349_gb300 import build
    build.build()
    oracle.set_threads(os.cpu_count() or 1)


@pytest.mark.parametrize("fp,tol", [(8, 1e-12), (4, 1e-6)])
def test_surface_pressure_matches_oracle(oracle, fp, tol):
    c = C.heated_cylinder()
    g = c.grid
    if fp == 4:
        import dataclasses
        g = dataclasses.replace(g, fp_bytes=4)
    grid = ibm.Grid(g, max_markers=len(c.X))
    grid.set_markers(c.X, c.Tw)
    grid.set_state(C.initial_state(g, c.seed).astype(np.float32 if fp == 4 else np.float64))
    grid.step(3)
    cp = grid.surface_pressure()
    Xk, _, _ = grid.markers()
    ref = oracle.surface_pressure(g, Xk, grid.get_state().cpu().numpy().astype(np.float64))
    p_inf = 1.0 / (g.gamma * g.Mach ** 2)
    assert np.max(np.abs(cp - ref)) <= tol * 2.0 * p_inf


def test_streamwise_oscillating_cylinder_matches_oracle(oracle):
    c = C.streamwise_oscillating_cylinder(scale_div=4)
    g = c.grid
    U0 = C.initial_state(g, c.seed).astype(np.float32)
    grid = ibm.Grid(g, max_markers=len(c.X))
    nk = grid.set_markers(c.X, c.Tw, motion=c.motion)
    grid.set_state(U0)
    run = oracle.Run(g, c.X, c.Tw, motion=c.motion)
    assert nk == len(run.X)
    U = U0.astype(np.float64)
    for s in range(5):
        grid.step(1)
        dtg = grid.time()[0]
        Ug = grid.get_state().cpu().numpy()
        U = run.step(U, dt_fixed=dtg)
        for gr in ([0], [1, 2], [3]):
            e = np.linalg.norm(Ug[gr] - U[gr]) / np.linalg.norm(U[gr])
            assert e < 1e-5, (s, gr, e)
    Xg, _, _ = grid.markers()
    assert np.max(np.abs(Xg - run.X)) < 1e-12       # markers moved along x only
    assert np.max(np.abs(Xg[:, 1] - run.X0[:, 1])) == 0.0
    fo = run.forces()
    fg = grid.forces()
    assert abs(fg["Cd"] - fo[2]) <= 2e-3 * abs(fo[2])


def test_self_convergence_of_drag():
    rows, orders = studies.self_convergence(divs=(8, 16, 32, 64), T=2.0)
    cds = [r[2] for r in rows]
    assert all(np.isfinite(cds)) and all(0.5 < cd < 20.0 for cd in cds)
    # successive differences shrink under refinement (the observed orders are
    # recorded in the design notes)
    d = np.abs(np.diff(cds))
    assert d[-1] < d[0], (rows, orders)
    # measured 1.39 and 1.50 on a GB300: between first and second order, rising
    assert all(o > 1.2 for o in orders), orders
    print("self-convergence", rows, orders)


def test_fixed_cylinder_sheds_at_a_plausible_strouhal_number():
    St, t, cl = studies.fixed_cylinder_strouhal()
    assert np.max(np.abs(cl[t > 150.0])) > 0.05       # shedding has developed
    assert 0.15 < St < 0.21, St                       # measured 0.180 at D/16
    print("Strouhal", St)


def _run_pair(oracle, g, case, steps, tol, share_eps):
    U0 = C.initial_state(g, case.seed).astype(np.float32 if g.fp_bytes == 4 else np.float64)
    grid = ibm.Grid(g, max_markers=len(case.X))
    nk = grid.set_markers(case.X, case.Tw, motion=case.motion)
    grid.set_state(U0)
    run = oracle.Run(g, case.X, case.Tw, motion=case.motion)
    assert nk == len(run.X)
    if share_eps:
        run.eps = grid.markers()[1].copy()
    U = U0.astype(np.float64)
    for s in range(steps):
        grid.step(1)
        dtg = grid.time()[0]
        U = run.step(U, dt_fixed=dtg if g.fp_bytes == 4 else 0.0)
        Ug = grid.get_state().cpu().numpy()
        for gr in ([0], list(range(1, g.dim + 1)), [g.dim + 1]):
            e = np.linalg.norm(Ug[gr] - U[gr]) / np.linalg.norm(U[gr])
            assert e < tol, (s, gr, e)
    fo = run.forces()
    fg = grid.forces()
    return fg, fo


def test_forcing_per_stage_fp64_matches_oracle(oracle):
    import dataclasses
    c = C.heated_cylinder()
    g = dataclasses.replace(c.grid, forcing_per_stage=1)
    fg, fo = _run_pair(oracle, g, c, 10, 1e-11, share_eps=True)
    assert abs(fg["Cd"] - fo[2]) <= 1e-9 * abs(fo[2])
    assert abs(fg["heat_rate"] - fo[1]) <= 1e-9 * abs(fo[1])
    # a different step from the default placement of the forcing
    g0 = dataclasses.replace(g, forcing_per_stage=0)
    a = ibm.Grid(g0, max_markers=len(c.X))
    a.set_markers(c.X, c.Tw)
    a.set_state(C.initial_state(g0, c.seed))
    a.step(10)
    assert abs(a.forces()["Cd"] - fg["Cd"]) > 1e-6 * abs(fg["Cd"])


def test_forcing_per_stage_fp32_moving_cylinder(oracle):
    import dataclasses
    c = C.oscillating_cylinder(scale_div=4)
    g = dataclasses.replace(c.grid, forcing_per_stage=1)
    fg, fo = _run_pair(oracle, g, c, 4, 1e-5, share_eps=False)
    assert abs(fg["Cd"] - fo[2]) <= 2e-3 * abs(fo[2])


def test_forcing_per_stage_is_refused_by_batch_and_adjoint():
    import dataclasses
    g = dataclasses.replace(C.small_grid(2, (32, 32), h=0.1, fp_bytes=8), forcing_per_stage=1)
    with pytest.raises(ibm.IbmError) as e:
        ibm.Batch([g], [0])
    assert e.value.status == 8
    grid = ibm.Grid(g, max_markers=4)
    with pytest.raises(ibm.IbmError) as e:
        grid.record(4, 2)
    assert e.value.status == 8


@pytest.mark.parametrize("moving", [False, True])
def test_step_graphs_are_bitwise_direct_launches(moving):
    c = C.oscillating_cylinder(scale_div=4) if moving else C.heated_cylinder()
    g = c.grid
    U0 = C.initial_state(g, c.seed).astype(np.float32 if g.fp_bytes == 4 else np.float64)
    grids = []
    for k in (0, 4):
        gr = ibm.Grid(g, max_markers=len(c.X))
        gr.set_markers(c.X, c.Tw, motion=c.motion)
        gr.set_state(U0)
        gr.use_graphs(k)
        grids.append(gr)
    for n in (9, 4, 3):          # chunks of 4 plus direct remainders, both parities
        for gr in grids:
            gr.step(n)
        a, b = (gr.get_state().cpu().numpy() for gr in grids)
        assert np.array_equal(a, b)
        assert grids[0].time() == grids[1].time()
        assert grids[0].forces()["Cd"] == grids[1].forces()["Cd"]
    # new markers: the graphs are recaptured
    X2 = c.X + np.array([0.02, -0.01])
    for gr in grids:
        gr.set_markers(X2, c.Tw, motion=c.motion)
        gr.step(8, dt_fixed=1e-3)
    a, b = (gr.get_state().cpu().numpy() for gr in grids)
    assert np.array_equal(a, b)
    with pytest.raises(ibm.IbmError):
        grids[1].use_graphs(3)
