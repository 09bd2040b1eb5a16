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


def test_surrogate_and_batch_argument_errors_without_gpu(lib):
    """The surrogate and batch entry points validate their arguments before
    any device call as well."""
    import ctypes
    from paper_1406_7635_gb300 import mm
    h = ctypes.c_void_p()
    bad_mx = mm.mm_fno_cfg(32, 4, 300, 24, 4, 1)   # modes_x > W / 2
    assert mm.mm_fno_create(ctypes.byref(h), 512, 512, ctypes.byref(bad_mx), 0, None) == -1
    assert b"modes_x" in mm.mm_last_error()
    bad_my = mm.mm_fno_cfg(32, 4, 24, 300, 4, 1)   # 2 modes_y > H
    assert mm.mm_fno_create(ctypes.byref(h), 512, 512, ctypes.byref(bad_my), 0, None) == -1
    bad_w = mm.mm_fno_cfg(0, 4, 24, 24, 4, 1)      # no channels
    assert mm.mm_fno_create(ctypes.byref(h), 512, 512, ctypes.byref(bad_w), 0, None) == -1
    assert mm.mm_fno_create(ctypes.byref(h), 512, 512, None, 0, None) == -1
    assert mm.mm_fno_destroy(None) == 0
    assert mm.mm_fno_forward(None, None, None, 1) == -1
    assert mm.mm_fno_param_count(None) == 0
    assert mm.mm_batch_create(ctypes.byref(h), 0, None, 0, None) == -1
    assert mm.mm_batch_create(None, 1, None, 0, None) == -1
