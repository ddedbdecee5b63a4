"""GPU: the bounds-checked build (IBM_CHECKED), the stand-in for a memory
checker on this pool.  In that build every instrumented global index - the
state loads and stores of the fluid stages (z-march and tiled), the support
cells and marker indices of interpolation and spreading, the columns of the
quadrature rows - is checked; a violation is recorded in the device error
word (reported as IBM_ERR_BOUNDS) and the access skipped, so nothing traps.

A child process loads the checked library and runs the small cases of every
path - 2D FP64 and FP32, 3D FP32 through the z-march with and without bulk
copies (ragged extents), 3D FP64, moving markers, a batch, the adjoint - and
each must finish with a clean error word; one case is also compared with the
oracle to show the checked build computes the same step.
"""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import os, sys
sys.path.insert(0, os.environ["IBM_ROOT"])
import numpy as np
import torch
from paper_2301_09349_gb300 import cases as C, ibm
from oracle import oracle as O

assert ibm.lib_path().endswith("libibm_gb300_checked.so"), ibm.lib_path()
O.set_threads(os.cpu_count() or 1)

def run(g, X, Tw, steps, fp=None, motion=None):
    grid = ibm.Grid(g, max_markers=max(len(X), 1))
    if len(X):
        grid.set_markers(X, Tw, motion=motion)
    U0 = C.initial_state(g, 7)
    grid.set_state(U0.astype(np.float32 if g.fp_bytes == 4 else np.float64))
    grid.step(steps)
    grid.sync()                       # raises on any device error bit
    out = grid.get_state().cpu().numpy()
    grid.close()
    return out

# 2D FP64 heated cylinder, compared with the oracle
c = C.heated_cylinder()
Ug = run(c.grid, c.X, c.Tw, 3)
r = O.Run(c.grid, c.X, c.Tw)
U = C.initial_state(c.grid, 7)
for _ in range(3):
    U = r.step(U)
err = np.linalg.norm(Ug - U) / np.linalg.norm(U)
assert err < 1e-8, err

# 3D FP32 sphere (z-march with bulk copies), 3D FP32 ragged (no copies)
s = C.heated_sphere(n=48, n_markers=2000)
run(s.grid, s.X, s.Tw, 3)
g = C.small_grid(3, (45, 38, 29), h=0.1, fp_bytes=4, Re=150.0, Mach=0.4)
run(g, C.fibonacci_sphere_markers(300, 0.6), np.full(300, 1.3), 3)
# 3D FP64 and 2D FP32 tiled stages
g = C.small_grid(3, (21, 19, 13), h=0.1, fp_bytes=8, Re=80.0, Mach=0.4)
run(g, np.zeros((0, 3)), np.zeros(0), 2)
g = C.small_grid(2, (77, 53), h=0.1, fp_bytes=4, Re=80.0, Mach=0.4)
run(g, C.circle_markers(40, 1.0), np.full(40, 1.2), 3)
# moving markers (bins and weights rebuilt every step)
m = C.oscillating_cylinder(scale_div=4)
run(m.grid, m.X, m.Tw, 3, motion=m.motion)
# a batch of two cases
cs = C.batched_cylinders(ncases=2, sizes=(128,))
b = ibm.Batch([x.grid for x in cs], [len(x.X) for x in cs])
for cg, x in zip(b.cases, cs):
    cg.set_markers(x.X, x.Tw)
    cg.set_state(C.initial_state(x.grid, x.seed).astype(np.float32))
b.step(3)
b.sync()
for cg in b.cases:
    cg.sync()
b.close()
# the adjoint (record, replay and reverse)
g = C.small_grid(3, (12, 12, 12), h=0.125, fp_bytes=8, Re=80.0, Mach=0.4)
X = C.fibonacci_sphere_markers(120, 0.4)
grid = ibm.Grid(g, max_markers=len(X))
grid.set_markers(X, np.full(len(X), 1.5))
grid.set_state(C.initial_state(g, 9))
grid.record(4, 2)
grid.step(4)
gX, gT = grid.backward(1.0, 0.5)
grid.sync()
assert np.all(np.isfinite(gX)) and np.all(np.isfinite(gT))
grid.close()
print("checked clean")
'''


def test_checked_build_runs_clean():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2301_09349_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, IBM_GB300_LIB=lib, IBM_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked clean" in r.stdout
