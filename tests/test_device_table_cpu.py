"""The per-device record of kernel attributes (shared-memory opt-in) that
every launch of the library consults, compiled with the host compiler and
checked without a GPU: the record is per (kernel, device ordinal), so a
second device gets its own opt-in."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2301_09349_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "native", "device_table_check.cpp")


def test_device_table_is_per_device_and_thread_safe(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "device_table_check")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-I" + CSRC, SRC, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "device table ok" in r.stdout
