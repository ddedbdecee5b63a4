"""GPU: batches of independent 2D grids.

A batch step runs each stage as one persistent launch over (case, tile) work
items.  Every case's arithmetic is the single-grid kernels' own device code
(the per-tile flux function, the interpolation terms, the spreading of one
marker tile, the finish of one grid), and maxima do not depend on the order
they are taken in, so the batch must reproduce the plain per-case loop of
ibm_step BIT FOR BIT - states, step sizes, times, marker forcing and force
sums - whatever the tile shape, markers per block or graph setting.  Cases
are also checked against the FP64 oracle directly.
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


def cast(U, g):
    return U.astype(np.float32 if g.fp_bytes == 4 else np.float64)


def rel_l2(a, b):
    """relative L2 error per conserved quantity: density, momentum vector,
    total energy"""
    a = np.asarray(a, dtype=np.float64).reshape(a.shape[0], -1)
    b = np.asarray(b, dtype=np.float64).reshape(b.shape[0], -1)
    nc = a.shape[0]
    groups = [[0], list(range(1, nc - 1)), [nc - 1]]
    return np.array([np.linalg.norm(a[gr] - b[gr]) / max(np.linalg.norm(b[gr]), 1e-300)
                     for gr in groups])


def small_batch(fp, n=5, sizes=(40, 56, 64), seed=7):
    """uneven small grids: 40 and 56 leave ragged tiles for every shape"""
    return C.batched_cylinders(ncases=n, sizes=sizes, seed=seed, fp_bytes=fp)


def make_batch(cs):
    b = ibm.Batch([c.grid for c in cs], [len(c.X) for c in cs])
    for cg, c in zip(b.cases, cs):
        cg.set_markers(c.X, c.Tw)
        cg.set_state(cast(C.initial_state(c.grid, c.seed), c.grid))
    return b


def make_loop(cs):
    out = []
    for c in cs:
        gr = ibm.Grid(c.grid, max_markers=len(c.X))
        gr.set_markers(c.X, c.Tw)
        gr.set_state(cast(C.initial_state(c.grid, c.seed), c.grid))
        out.append(gr)
    return out


def same(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return a.shape == b.shape and np.array_equal(a, b, equal_nan=True)


def assert_bitwise(b, loop):
    F = b.forces()
    for i, (cg, gr) in enumerate(zip(b.cases, loop)):
        assert torch.equal(cg.get_state(), gr.get_state()), i
        assert cg.time() == gr.time(), i
        for x, y in zip(cg.marker_forcing(), gr.marker_forcing()):
            assert same(x, y), i
        f = gr.forces()
        dt, t, _ = gr.time()
        ref = [f["force"][0], f["force"][1], f["heat_rate"], f["Cd"], f["Cl"], f["Nu"], dt, t]
        assert same(F[i], ref), (i, F[i], ref)


@pytest.mark.parametrize("fp", [4, 8])
@pytest.mark.parametrize("shape,warps,graph", [
    (0, 4, 1), (1, 1, 0), (2, 16, 1), (3, 8, 0), (1, 2, 1),
])
def test_batch_bitwise_equals_per_case_loop(fp, shape, warps, graph):
    cs = small_batch(fp)
    b = make_batch(cs)
    b.set_tuning(shape, warps, graph)
    assert b.tuning() == {"tile_shape": shape, "markers_per_block": warps, "use_graph": graph}
    loop = make_loop(cs)
    b.step(3)
    for gr in loop:
        gr.step(3)
    assert_bitwise(b, loop)
    # odd and even parities, graphs replayed more than once
    b.step(4)
    for gr in loop:
        gr.step(4)
    assert_bitwise(b, loop)


def test_batch_energy_reading_total_equals_loop():
    cs = small_batch(4, n=3, seed=17)
    b = ibm.Batch([c.grid for c in cs], [len(c.X) for c in cs], energy_reading=1)
    loop = []
    for cg, c in zip(b.cases, cs):
        cg.set_markers(c.X, c.Tw)
        cg.set_state(cast(C.initial_state(c.grid, c.seed), c.grid))
        gr = ibm.Grid(c.grid, max_markers=len(c.X), energy_reading=1)
        gr.set_markers(c.X, c.Tw)
        gr.set_state(cast(C.initial_state(c.grid, c.seed), c.grid))
        loop.append(gr)
    b.step(3)
    for gr in loop:
        gr.step(3)
    assert_bitwise(b, loop)


def test_batch_fixed_dt_and_changes_between_steps():
    cs = small_batch(4, n=4, seed=9)
    b = make_batch(cs)
    loop = make_loop(cs)
    b.step(2, dt_fixed=2e-3)
    for gr in loop:
        gr.step(2, dt_fixed=2e-3)
    assert_bitwise(b, loop)
    # one case stepped on its own: the batch rebuilds its tables
    b.cases[1].step(1)
    loop[1].step(1)
    b.step(2)
    for gr in loop:
        gr.step(2)
    assert_bitwise(b, loop)
    # new markers (and a new tuning) on a case between batch steps
    c = cs[2]
    X2 = c.X + np.array([0.3, -0.2])
    b.cases[2].set_markers(X2, c.Tw)
    loop[2].set_markers(X2, c.Tw)
    b.set_tuning(tile_shape=2)
    b.step(3)
    for gr in loop:
        gr.step(3)
    assert_bitwise(b, loop)


def test_autotune_changes_speed_not_results():
    cs = small_batch(4, n=6, seed=11)
    b = make_batch(cs)
    loop = make_loop(cs)
    b.step(1)
    for gr in loop:
        gr.step(1)
    before = [cg.get_state().clone() for cg in b.cases]
    forcing = [cg.marker_forcing() for cg in b.cases]
    times = [cg.time() for cg in b.cases]
    r = b.autotune(reps=2)
    assert r["stage_ms"].shape == (4,) and np.all(r["stage_ms"] > 0)
    assert r["interp_ms"].shape == (5,) and np.all(r["interp_ms"] > 0)
    t = b.tuning()
    assert t["tile_shape"] == int(np.argmin(r["stage_ms"]))
    assert t["markers_per_block"] == ibm.BATCH_WARPS[int(np.argmin(r["interp_ms"]))]
    for cg, U, fr, tm in zip(b.cases, before, forcing, times):
        assert torch.equal(cg.get_state(), U)
        assert all(same(x, y) for x, y in zip(cg.marker_forcing(), fr))
        assert cg.time() == tm
    b.step(3)
    for gr in loop:
        gr.step(3)
    assert_bitwise(b, loop)


def test_batch_cases_match_the_oracle(oracle):
    """FP64 batch against the FP64 oracle case by case (each case's quadrature
    weights handed to the oracle, as in the single-grid FP64 test)."""
    cs = small_batch(8, n=3, sizes=(48, 64), seed=13)
    b = make_batch(cs)
    runs, Us = [], []
    for cg, c in zip(b.cases, cs):
        run = oracle.Run(c.grid, c.X, c.Tw)
        _, eps_g, _ = cg.markers()
        assert len(eps_g) == len(run.X)
        assert np.max(np.abs(eps_g - run.eps) / run.eps) < 1e-7
        run.eps = eps_g.copy()
        runs.append(run)
        Us.append(C.initial_state(c.grid, c.seed))
    for s in range(3):
        b.step(1)
        F = b.forces()
        for i, (cg, run) in enumerate(zip(b.cases, runs)):
            Uo = run.step(Us[i])
            Ug = cg.get_state().cpu().numpy()
            err = rel_l2(Ug, Uo)
            assert np.all(err < 1e-11), (s, i, err)
            assert abs(F[i, 6] - run.dt) <= 1e-9 * run.dt
            fo = run.forces()
            assert abs(F[i, 3] - fo[2]) <= 1e-9 * abs(fo[2]) + 1e-12
            assert abs(F[i, 2] - fo[1]) <= 1e-9 * abs(fo[1]) + 1e-12
            Us[i] = Uo


def test_full_size_batch_one_step_equals_loop():
    """The 64-case workload at full size: one batched step (autotuned, graph)
    against the per-case loop, bit for bit."""
    cs = C.batched_cylinders()
    b = make_batch(cs)
    b.autotune(reps=2)
    loop = make_loop(cs)
    b.step(2)
    for gr in loop:
        gr.step(2)
    assert_bitwise(b, loop)


def test_batch_errors():
    g2 = C.small_grid(2, (32, 32), h=0.1, fp_bytes=4)
    g3 = C.small_grid(3, (16, 16, 16), h=0.1, fp_bytes=4)
    g2d = C.small_grid(2, (32, 32), h=0.1, fp_bytes=8)
    with pytest.raises(ibm.IbmError) as e:
        ibm.Batch([g2, g3], [0, 0])
    assert e.value.status == 8
    with pytest.raises(ibm.IbmError) as e:
        ibm.Batch([g2, g2d], [0, 0])
    assert e.value.status == 8
    b = ibm.Batch([g2, g2], [4, 4])
    with pytest.raises(ibm.IbmError) as e:
        b.step(1)
    assert e.value.status == 7
    with pytest.raises(ibm.IbmError) as e:
        ibm.ibm_destroy(b.cases[0].h)
    assert e.value.status == 1
    with pytest.raises(ibm.IbmError) as e:
        b.set_tuning(tile_shape=4)
    assert e.value.status == 1
    U = C.random_state(g2, seed=3)
    b.cases[0].set_state(U)
    b.cases[1].set_state(U)
    b.cases[1].set_markers(np.array([[0.4, 0.0]]), np.ones(1), motion=C.Motion(0.1, 1.0, 1))
    with pytest.raises(ibm.IbmError) as e:
        b.step(1)
    assert e.value.status == 8
    # a non-positive state in one case is reported with that case's index
    b = ibm.Batch([g2, g2, g2], [0, 0, 0])
    U2 = U.copy()
    U2[0, 7, 9] = -1.0
    for i, Ui in enumerate([U, U2, U]):
        b.cases[i].set_state(Ui)
    b.step(1)
    with pytest.raises(ibm.IbmError) as e:
        b.sync()
    assert e.value.status == 3 and "case 1" in e.value.message


def test_batch_wall_temperature_setter_equals_per_case_setter():
    """ibm_batch_set_wall_temperature (one upload for all cases) leaves every
    case as ibm_set_wall_temperature on each case would, bit for bit; a bad
    value anywhere is rejected and changes nothing."""
    cs = small_batch(4, n=4, seed=11)
    b = make_batch(cs)
    loop = make_loop(cs)
    b.step(2)
    for gr in loop:
        gr.step(2)
    rng = np.random.default_rng(5)
    new = [rng.uniform(0.6, 1.9, cg.n_kept) for cg in b.cases]
    b.set_wall_temperature(np.concatenate(new))
    for gr, t in zip(loop, new):
        gr.set_wall_temperature(t)
    b.step(3)
    for gr in loop:
        gr.step(3)
    assert_bitwise(b, loop)
    bad = np.concatenate(new)
    bad[-1] = -1.0
    with pytest.raises(ibm.IbmError) as e:
        b.set_wall_temperature(bad)
    assert e.value.status == 1 and "finite and positive" in e.value.message
    b.step(1)
    for gr in loop:
        gr.step(1)
    assert_bitwise(b, loop)


def test_batch_forces_report_the_failing_case():
    """the error words travel with the gathered force sums: ibm_batch_forces
    reports a failing case as ibm_batch_sync does"""
    g2 = C.small_grid(2, (32, 32), h=0.1, fp_bytes=4)
    U = C.random_state(g2, seed=3)
    b = ibm.Batch([g2, g2, g2], [0, 0, 0])
    U2 = U.copy()
    U2[0, 7, 9] = -1.0
    for i, Ui in enumerate([U, U, U2]):
        b.cases[i].set_state(Ui)
    b.step(1)
    with pytest.raises(ibm.IbmError) as e:
        b.forces()
    assert e.value.status == 3 and "case 2" in e.value.message
