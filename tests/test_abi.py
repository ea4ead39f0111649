"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/qcd.h declares (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

import paper_1210_7398_gb300 as q
from paper_1210_7398_gb300 import build as qbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(qcd_[A-Za-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    path = qbuild.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 13
    for s in sorted(syms):
        assert hasattr(lib, s), "missing export %s" % s
    assert set(q.EXPORTS) <= syms


def test_binding_structs_match_header():
    # qcd_params: 2 doubles, 8 ints, 1 double, 2 ints, 2 doubles, 9 ints (with padding)
    assert ctypes.sizeof(q.qcd_params) == 120
    assert ctypes.sizeof(q.qcd_stats) == 48
    # qcd_learned_verdict: 4 doubles, 6 ints
    assert ctypes.sizeof(q.qcd_learned_verdict) == 56


def test_binding_constants_match_header():
    """Every QCD_* enumerator of the header has the same value in the binding (precisions and
    storage forms, error codes, kernel classes)."""
    text = open(os.path.join(ROOT, "include", "qcd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    consts = {}
    for body in re.findall(r"enum\s*\{([^}]*)\}", text):
        for name, val in re.findall(r"\b(QCD_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            consts[name] = int(val)
    assert consts["QCD_F32X2"] == 5 and consts["QCD_F64"] == 0
    checked = 0
    for name, val in consts.items():
        if hasattr(q, name):
            assert getattr(q, name) == val, name
            checked += 1
    assert checked >= 8


def test_null_context_is_rejected(lib):
    q.load_library()
    assert q.load_library().qcd_set_boundary(None, 1) == q.QCD_ERR_ARG
    assert q.load_library().qcd_launch_count(None) == 0


def test_plain_c_client(lib, tmp_path):
    """include/qcd.h compiles as C99 with warnings as errors; a C program linked against the
    library sees the struct layouts the binding mirrors and gets argument errors, not crashes."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(qbuild.LIB)
    exe = str(tmp_path / "abi_check")
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c", "abi_check.c"), "-L", libdir, "-lqcd",
                           "-Wl,-rpath," + libdir, "-o", exe])
    res = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert res.returncode == 0, res.stderr
    assert res.stdout.strip() == "ok"
