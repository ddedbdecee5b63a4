"""Build the CUDA library libibm_gb300.so in-tree (nvcc, sm_103a only).

The translation units compile in parallel, then one nvcc call links them into
paper_2301_09349_gb300/lib/libibm_gb300.so.  The CUDA runtime is linked
statically, so the library needs only the driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libibm_gb300.so")
# the bounds-checked variant (IBM_CHECKED): every instrumented global index
# is checked, a violation is recorded in the device error word
# (IBM_ERR_BOUNDS) and the access skipped; for tests, not for timing
LIB_CHECKED = os.path.join(LIBDIR, "libibm_gb300_checked.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
UNITS = ["flux.cu", "flux_zm.cu", "markers.cu", "quadrature.cu", "api.cu", "noalloc.cu", "adjoint.cu",
         "batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]
# The FP32 fluid-stage units flush subnormals to zero: no value of the flow
# comes near 1e-38, and the approximate reciprocals and square roots then need
# no subnormal handling (4-5 % of the stage time on the 3D and 2D kernels).
# The adjoint unit also takes FP32 divisions and square roots from the fast
# approximations (FP64 code is unaffected): its FP32 reverse sweep is 23 %
# faster and stays within the FP32 gradient tolerance.
UNIT_FLAGS = {"flux.cu": ["-ftz=true"], "flux_zm.cu": ["-ftz=true"],
              "adjoint.cu": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"]}
# extra nvcc flags (e.g. -DIBM_ZM_MIN_BLOCKS=2) for build variants
EXTRA = os.environ.get("IBM_NVCC_FLAGS", "").split()


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libibm_gb300.so")


def _sources():
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    deps.append(os.path.join(INCLUDE, "ibm.h"))
    return deps


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _sources())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile the library (checked=True: the bounds-checked variant)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(lib):
        return lib
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()
    objdir = os.path.join(LIBDIR, "obj_checked" if checked else "obj")
    os.makedirs(objdir, exist_ok=True)
    variant = ["-DIBM_CHECKED"] if checked else []

    def compile_one(unit):
        obj = os.path.join(objdir, unit.replace(".cu", ".o"))
        cmd = [cc] + ARCH + FLAGS + UNIT_FLAGS.get(unit, []) + EXTRA + variant + \
            ["-c", os.path.join(SRC, unit), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s" % (unit, r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s" % r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
