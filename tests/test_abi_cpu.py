"""The C-ABI library loads and exports every entry point declared in
include/ibm.h; host-side argument checks work without a GPU (no compute
calls here)."""
import ctypes
import os
import re

import pytest

from paper_2301_09349_gb300 import build, cases, ibm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ibm.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ibm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ibm_\w+)\s*\(", src)))


def test_header_declares_the_core_calls():
    names = declared_functions()
    for n in ("ibm_create_grid", "ibm_set_markers", "ibm_step", "ibm_forces_and_nusselt",
              "ibm_backward"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_exports_nothing_the_header_does_not_declare(lib):
    """No undeclared entry point (a debug hook, a stray helper) leaves the
    library: its exported ibm_* text symbols are exactly the header's."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "--defined-only", build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = sorted({f[2] for f in (l.split() for l in out.splitlines())
                       if len(f) == 3 and f[1] == "T" and f[2].startswith("ibm_")})
    assert exported == declared_functions()


def test_binding_covers_the_header(lib):
    assert sorted(n for n, _, _ in ibm.SIGNATURES) == declared_functions()


def test_workspace_bytes(lib):
    c = cases.heated_sphere()
    d = ibm.make_desc(c.grid)
    nb = ibm.ibm_workspace_bytes(d, 20000)
    state = 5 * 256 ** 3 * 4
    assert 3 * state < nb < 3 * state + 200 * 2 ** 20
    assert ibm.ibm_workspace_bytes(d, 0) < nb
    bad = ibm.make_desc(c.grid)
    bad.dim = 4
    assert ibm.ibm_workspace_bytes(bad, 10) == 0
    bad = ibm.make_desc(c.grid)
    bad.fp_bytes = 2
    assert ibm.ibm_workspace_bytes(bad, 10) == 0
    bad = ibm.make_desc(cases.small_grid(2, (3, 8)))
    assert ibm.ibm_workspace_bytes(bad, 10) == 0
    bad = ibm.make_desc(c.grid)
    bad.bc[0] = cases.BC_PERIODIC          # unpaired periodic face
    assert ibm.ibm_workspace_bytes(bad, 10) == 0


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    c = cases.heated_cylinder()
    d = ibm.make_desc(c.grid)
    h = ctypes.c_void_p()
    st = lib.ibm_create_grid(None, 10, ctypes.c_void_p(256), 1 << 20, None, ctypes.byref(h))
    assert st == 1 and h.value is None
    assert b"null grid description" in lib.ibm_last_error(None)
    st = lib.ibm_create_grid(ctypes.byref(d), 10, None, 1 << 20, None, ctypes.byref(h))
    assert st == 1
    st = lib.ibm_create_grid(ctypes.byref(d), 10, ctypes.c_void_p(256 + 8), 1 << 30, None,
                             ctypes.byref(h))
    assert st == 1 and b"aligned" in lib.ibm_last_error(None)
    st = lib.ibm_create_grid(ctypes.byref(d), 10, ctypes.c_void_p(256), 1024, None, ctypes.byref(h))
    assert st == 5 and b"too small" in lib.ibm_last_error(None)
    st = lib.ibm_create_grid(ctypes.byref(d), -1, ctypes.c_void_p(256), 1 << 30, None,
                             ctypes.byref(h))
    assert st == 1


def test_null_handle_is_an_argument_error(lib):
    assert lib.ibm_step(None, 1, ctypes.c_double(0.0)) == 1
    assert lib.ibm_sync(None) == 1
    assert lib.ibm_destroy(None) == 1
    assert lib.ibm_set_state(None, None) == 1


def test_python_binding_raises_when_library_missing(monkeypatch):
    monkeypatch.setenv("IBM_GB300_LIB", "/nonexistent/libibm_gb300.so")
    monkeypatch.setattr(ibm, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        ibm.lib()


def test_build_compiles_every_cuda_unit_for_sm_103a_only():
    """A .cu file left out of the unit list would be missing from the library
    without any error; the flags name one architecture, sm_103a."""
    units = sorted(f for f in os.listdir(build.SRC) if f.endswith(".cu"))
    assert sorted(build.UNITS) == units
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert set(build.UNIT_FLAGS) <= set(build.UNITS)
    # subnormal flushing and the fast FP32 division / square root only in the
    # units whose FP32 arithmetic was measured and parity-tested with them
    assert set(build.UNIT_FLAGS) == {"flux.cu", "flux_zm.cu", "adjoint.cu"}
