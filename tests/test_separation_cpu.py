"""CPU: the oracle and the CUDA path share no code.  Nothing in the package
(Python binding, CUDA sources, build script) imports, includes, loads or
runs anything under oracle/; nothing in oracle/ imports the package or
includes its headers.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU legs reach the oracle."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2301_09349_gb300")
ORACLE = os.path.join(ROOT, "oracle")
INCLUDE = os.path.join(ROOT, "include")


def _sources(top, exts):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("lib", "__pycache__", "obj")]
        for f in files:
            if os.path.splitext(f)[1] in exts:
                yield os.path.join(d, f)


def _text(p):
    with open(p, encoding="utf-8") as f:
        return f.read()


PY_IMPORT_ORACLE = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b|from\s+\.\.?\s*oracle\b)", re.M)
NAMES_ORACLE_LIB = re.compile(r"liboracle|ibm_oracle|oracle[/\\]")


def test_package_never_reaches_the_oracle():
    srcs = list(_sources(PKG, {".py", ".cu", ".cuh", ".h", ".cpp", ".c"})) + \
        list(_sources(INCLUDE, {".h"}))
    assert srcs
    for p in srcs:
        t = _text(p)
        assert not PY_IMPORT_ORACLE.search(t), p
        assert not NAMES_ORACLE_LIB.search(t), p
        for inc in re.findall(r'#include\s+"([^"]+)"', t):
            assert "oracle" not in inc, (p, inc)


def test_oracle_never_reaches_the_package():
    srcs = list(_sources(ORACLE, {".py", ".c", ".h"}))
    assert any(p.endswith(".c") for p in srcs)
    for p in srcs:
        t = _text(p)
        assert not re.search(r"^\s*(from|import)\s+paper_2301_09349_gb300", t, re.M), p
        assert "libibm_gb300" not in t, p
        for inc in re.findall(r'#include\s+"([^"]+)"', t):
            assert os.path.dirname(inc) == "" and os.path.exists(os.path.join(ORACLE, inc)), (p, inc)


def test_only_tests_smoke_and_bench_import_the_oracle():
    users = []
    for p in _sources(ROOT, {".py"}):
        rel = os.path.relpath(p, ROOT)
        if rel.startswith(("oracle" + os.sep, "tests" + os.sep, "_work" + os.sep, "baseline" + os.sep)):
            continue
        if PY_IMPORT_ORACLE.search(_text(p)):
            users.append(rel)
    assert sorted(users) == ["__graft_entry__.py", "bench.py"], users
