"""CPU-side checks of the native library: it builds for sm_103a, loads, and
exports every entry point that include/lsn.h declares (no GPU calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lsn.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(lsn_\w+)\(", src, re.M)))


def test_header_declares_the_solver_calls():
    names = _declared()
    for n in ["lsn_create", "lsn_destroy", "lsn_last_error", "lsn_set_mesh",
              "lsn_set_material", "lsn_set_constraints", "lsn_set_cubature",
              "lsn_set_ground", "lsn_set_decoder", "lsn_set_solver", "lsn_set_optimizer",
              "lsn_set_state",
              "lsn_step", "lsn_get_positions", "lsn_eval", "lsn_fullspace_setup",
              "lsn_fullspace_set_state", "lsn_fullspace_step"]:
        assert n in names


@pytest.fixture(scope="module")
def lib():
    from paper_2409_03807_gb300.build import build
    build()
    import paper_2409_03807_gb300 as pkg
    return pkg.load()


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    import paper_2409_03807_gb300 as pkg
    assert set(_declared()) <= set(pkg.exported_symbols())


def test_noalloc_argument_checks_return_before_any_device_work(lib):
    """Host-side checks of lsn_element_system_noalloc: a misaligned tets or J
    pointer, or n not a multiple of 3, is rejected with LSN_ERR_ARG before the
    call touches a pointer or the device (host arrays stand in here)."""
    import ctypes
    import numpy as np
    buf = np.zeros(1024, dtype=np.float64)        # 8-byte aligned storage
    base = buf.ctypes.data
    assert base % 16 == 0
    call = lib.lsn_element_system_noalloc
    good = ctypes.c_void_p(base)
    out = ctypes.c_void_p(base)
    args = lambda tets, J, n=12, r=4: (1, r, n, tets, good, good, good, J, 1.0, 1.0, out, None)
    assert call(*args(ctypes.c_void_p(base + 4), good)) == -1       # tets not 16-byte aligned
    assert call(*args(ctypes.c_void_p(base + 8), good)) == -1
    assert call(*args(good, ctypes.c_void_p(base + 4))) == -1       # J rows of 16 bytes
    assert call(*args(good, good, n=13)) == -1                      # n not a multiple of 3
    assert call(*args(good, good, r=65)) == -1                      # r above 64
