"""The allocation-free stage-1 entry point, ibm_rhs_dt_noalloc, against the
regular entry points.

It serves callers that may not allocate device memory (a plug-in inside a
host that owns the device-memory budget, or a loop that cannot afford a
cudaMalloc): its scratch lives in a static device array.  Its L must equal
ibm_rhs's and its step size the one ibm_step computes from the same state,
within the operator tolerances of the parity tests (FP32 1e-4 relative,
FP64 1e-12; the step size is a max-reduction of identical values, so 1e-12).
Two calls in a row check that the shared scratch is reset between calls; a
state with a NaN gives a step size of 0, and the next clean call is not
affected by it.  Every grid kind is covered: 3D FP32 (the z-march kernel),
2D FP32, 2D FP64 and 3D FP64 (the tiled stage kernel).
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2301_09349_gb300 import cases as C
from paper_2301_09349_gb300 import ibm

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = a.reshape(a.shape[0], -1).astype(np.float64)
    b = b.reshape(b.shape[0], -1).astype(np.float64)
    return max(np.linalg.norm(a[c] - b[c]) / np.linalg.norm(b[c]) for c in range(a.shape[0]))


def _noalloc(L, desc, U, Lout, dt, stream):
    return L.ibm_rhs_dt_noalloc(ctypes.byref(desc), ctypes.c_void_p(U.data_ptr()),
                                ctypes.c_void_p(Lout.data_ptr()), ctypes.c_void_p(dt.data_ptr()),
                                ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("dim,n,fp,tol", [
    (3, (45, 38, 29), 4, 1e-4),
    (2, (77, 53), 4, 1e-4),
    (2, (77, 53), 8, 1e-12),
    (3, (21, 19, 13), 8, 1e-12),
])
def test_noalloc_stage1_matches_regular_entry_points(dim, n, fp, tol):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2301_09349_gb300 import build
    build.build()
    L = ibm.lib()
    g = C.small_grid(dim, n, h=0.1, fp_bytes=fp, Re=150.0, Mach=0.4)
    dtype = np.float32 if fp == 4 else np.float64
    desc = ibm.make_desc(g)
    stream = torch.cuda.current_stream()
    grid = ibm.Grid(g)
    for call, seed in enumerate((51, 52)):
        U = torch.from_numpy(C.random_state(g, seed=seed, amp=0.03).astype(dtype)).cuda()
        Lna = torch.empty_like(U)
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st = _noalloc(L, desc, U, Lna, dt, stream)
        assert st == 0, ibm.ibm_last_error(None)
        assert ibm.ibm_last_error(None) == ""
        torch.cuda.synchronize()
        L_ref = grid.rhs(U)
        grid.set_state(U)
        grid.step(1)
        dt_ref, _, _ = grid.time()
        err = _rel(Lna.cpu().numpy(), L_ref.cpu().numpy())
        assert err < tol, (call, err)
        assert abs(dt.item() - dt_ref) <= 1e-12 * dt_ref, (call, dt.item(), dt_ref)
    grid.close()


def test_noalloc_nonfinite_state_gives_zero_dt_then_recovers():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    L = ibm.lib()
    g = C.small_grid(3, (40, 24, 20), h=0.1, fp_bytes=4, Re=150.0, Mach=0.4)
    desc = ibm.make_desc(g)
    stream = torch.cuda.current_stream()
    clean = C.random_state(g, seed=53, amp=0.03).astype(np.float32)
    bad = clean.copy()
    bad[0, 7, 11, 13] = np.nan          # planted on the host
    dts = []
    for U_host in (bad, clean):
        U = torch.from_numpy(U_host).cuda()
        Lna = torch.empty_like(U)
        dt = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        assert _noalloc(L, desc, U, Lna, dt, stream) == 0
        torch.cuda.synchronize()
        dts.append(dt.item())
    assert dts[0] == 0.0
    grid = ibm.Grid(g)
    grid.set_state(torch.from_numpy(clean).cuda())
    grid.step(1)
    dt_ref, _, _ = grid.time()
    grid.close()
    assert dts[1] > 0.0 and abs(dts[1] - dt_ref) <= 1e-12 * dt_ref, (dts, dt_ref)


def test_noalloc_rejects_bad_arguments_with_their_reason():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    L = ibm.lib()
    g = C.small_grid(3, (8192, 4096, 32), h=0.1, fp_bytes=4)   # 131072 column blocks
    desc = ibm.make_desc(g)
    st = L.ibm_rhs_dt_noalloc(ctypes.byref(desc), ctypes.c_void_p(256), ctypes.c_void_p(256),
                              ctypes.c_void_p(256), None)
    assert st == ibm.IBM_OK + 1
    assert "IBM_NOALLOC_MAX_CTAS" in ibm.ibm_last_error(None)
    desc.fp_bytes = 2
    st = L.ibm_rhs_dt_noalloc(ctypes.byref(desc), ctypes.c_void_p(256), ctypes.c_void_p(256),
                              ctypes.c_void_p(256), None)
    assert st == ibm.IBM_OK + 1
    assert "fp_bytes" in ibm.ibm_last_error(None)
