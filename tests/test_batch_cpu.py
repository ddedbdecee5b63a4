"""Batches of 2D grids without a GPU: the seeded batch generator and the
host-side checks of the batch entry points (no compute calls here)."""
import ctypes
import math

import numpy as np
import pytest

from paper_2301_09349_gb300 import build, cases, ibm


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ibm.lib()


def test_batched_cylinders_follow_their_recipe():
    bs = cases.batched_cylinders()
    assert len(bs) == 64
    assert {c.grid.n[0] for c in bs} <= {128, 256, 384, 512}
    assert len({c.grid.n[0] for c in bs}) == 4          # uneven sizes really occur
    for i, c in enumerate(bs):
        g = c.grid
        assert c.seed == 4000 + i
        assert g.dim == 2 and g.n[0] == g.n[1] and g.fp_bytes == 4
        assert g.h == pytest.approx(16.0 / g.n[0])
        assert g.lo[:2] == (-4.0, -8.0)
        assert 0.5 <= c.Tw[0] <= 2.0 and np.all(c.Tw == c.Tw[0])
        assert 0.1 <= g.Mach <= 0.5 and 40.0 <= g.Re <= 200.0
        nm = math.ceil(math.pi / g.h)
        ncyl = len(c.X) // nm
        assert len(c.X) == ncyl * nm and 1 <= ncyl <= 8
        centres = c.X.reshape(ncyl, nm, 2).mean(axis=1)
        assert np.all(centres[:, 0] >= -2.0 - 1e-12) and np.all(centres[:, 0] <= 6.0 + 1e-12)
        assert np.all(np.abs(centres[:, 1]) <= 6.0 + 1e-12)
        for a in range(ncyl):
            for b in range(a):
                assert np.hypot(*(centres[a] - centres[b])) >= 1.5 + 4 * g.h - 1e-9
        # every marker at least two cells inside the domain (support + halo)
        cell = np.floor((c.X - np.array(g.lo[:2])) / g.h)
        assert cell.min() >= 2 and cell.max() <= g.n[0] - 3


def test_batched_cylinders_are_deterministic():
    a = cases.batched_cylinders(ncases=5, sizes=(40, 56), seed=7)
    b = cases.batched_cylinders(ncases=5, sizes=(40, 56), seed=7)
    for x, y in zip(a, b):
        assert x.name == y.name and np.array_equal(x.X, y.X) and x.grid == y.grid
    c = cases.batched_cylinders(ncases=5, sizes=(40, 56), seed=8)
    assert any(not np.array_equal(x.X, y.X) for x, y in zip(a, c))


def test_batch_workspace_bytes(lib):
    bs = cases.batched_cylinders(ncases=6, sizes=(40, 56, 64), seed=7)
    descs = [ibm.make_desc(c.grid) for c in bs]
    mm = [len(c.X) for c in bs]
    total = ibm.ibm_batch_workspace_bytes(descs, mm)
    per_case = sum(ibm.ibm_workspace_bytes(d, m) for d, m in zip(descs, mm))
    assert per_case < total < per_case + (8 << 20)
    assert total % 256 == 0
    d3 = ibm.make_desc(cases.small_grid(3, (16, 16, 16), fp_bytes=4))
    assert ibm.ibm_batch_workspace_bytes([descs[0], d3], [0, 0]) == 0
    d64 = ibm.make_desc(cases.small_grid(2, (32, 32), fp_bytes=8))
    assert ibm.ibm_batch_workspace_bytes([descs[0], d64], [0, 0]) == 0
    assert ibm.ibm_batch_workspace_bytes(descs[:1], [-1]) == 0
    assert lib.ibm_batch_workspace_bytes(0, ibm._desc_array(descs), None) == 0


def test_create_batch_rejects_bad_arguments_before_touching_the_gpu(lib):
    bs = cases.batched_cylinders(ncases=2, sizes=(40,), seed=7)
    descs = ibm._desc_array([ibm.make_desc(c.grid) for c in bs])
    h = ctypes.c_void_p()
    st = lib.ibm_create_batch(2, descs, None, ctypes.c_void_p(256), 1 << 30, None, None)
    assert st == 1
    st = lib.ibm_create_batch(2, descs, None, None, 1 << 30, None, ctypes.byref(h))
    assert st == 1 and h.value is None
    st = lib.ibm_create_batch(2, descs, None, ctypes.c_void_p(256 + 8), 1 << 30, None,
                              ctypes.byref(h))
    assert st == 1 and b"aligned" in lib.ibm_batch_last_error(None)
    st = lib.ibm_create_batch(2, descs, None, ctypes.c_void_p(256), 4096, None, ctypes.byref(h))
    assert st == 5 and b"too small" in lib.ibm_batch_last_error(None)
    d3 = ibm._desc_array([ibm.make_desc(cases.small_grid(3, (16, 16, 16), fp_bytes=4))])
    st = lib.ibm_create_batch(1, d3, None, ctypes.c_void_p(256), 1 << 30, None, ctypes.byref(h))
    assert st == 8 and b"2D" in lib.ibm_batch_last_error(None)


def test_null_batch_is_an_argument_error(lib):
    assert lib.ibm_batch_step(None, 1, ctypes.c_double(0.0)) == 1
    assert lib.ibm_batch_sync(None, None) == 1
    assert lib.ibm_batch_destroy(None) == 1
    assert lib.ibm_batch_forces(None, None) == 1
    assert lib.ibm_batch_set_wall_temperature(None, None) == 1
    assert lib.ibm_batch_autotune(None, 1, None, None) == 1
    assert lib.ibm_batch_set_tuning(None, None) == 1
    assert lib.ibm_batch_get_tuning(None, None) == 1
    assert lib.ibm_batch_case(None, 0) is None


def test_batched_cases_are_dealt_to_ranks_exactly_once():
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    names = [c.name for c in cases.batched_cylinders()]
    for world in (1, 2, 3, 8):
        dealt = [c.name for r in range(world) for c in bench.batch_cases(r, world)]
        assert sorted(dealt) == sorted(names)
        sizes = [len(bench.batch_cases(r, world)) for r in range(world)]
        assert max(sizes) - min(sizes) <= 1
