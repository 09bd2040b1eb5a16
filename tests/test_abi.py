"""The C-ABI library builds, loads and exports every entry point of include/mm.h
(no compute calls: these run without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1406_7635_gb300.build import build
    return build()


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mm_[a-z_0-9]+)$", out, flags=re.M))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_binding_loads_and_matches_header(lib):
    from paper_1406_7635_gb300 import mm
    assert set(declared_symbols()) == set(mm.EXPORTED)


def test_argument_errors_without_gpu(lib):
    """Argument validation happens before any device call."""
    import ctypes
    from paper_1406_7635_gb300 import mm
    h = ctypes.c_void_p()
    assert mm.mm_create(ctypes.byref(h), 0, 4, 4, 1e-9, 1e-9, 1e-9, 0, None) == -1
    assert b"grid" in mm.mm_last_error()
    assert mm.mm_create(ctypes.byref(h), 4, 4, 4, -1e-9, 1e-9, 1e-9, 0, None) == -1
    assert mm.mm_create(None, 4, 4, 4, 1e-9, 1e-9, 1e-9, 0, None) == -1
    assert mm.mm_destroy(None) == 0
    assert mm.mm_step(None, 1) == -1
