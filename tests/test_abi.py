"""The C-ABI library builds for sm_103a, loads, and exports what the header
declares; argument errors are rejected on the host before any device work."""
import ctypes
import os
import re

import pytest

from paper_2402_06835_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "nuance.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nu_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = build.build_library()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ["nu_gp_factor", "nu_linear_search", "nu_periodic_search",
              "nu_batch_search", "nu_factor_info", "nu_factor_free",
              "nu_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_host_side_argument_errors(lib):
    lib.nu_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    # n < 2 is rejected before any CUDA call
    st = lib.nu_gp_factor(None, None, ctypes.c_int64(1), None, 0, None, 0, None, None,
                          ctypes.byref(out))
    assert st == 1
    assert b"n >= 2" in lib.nu_last_error()
    st = lib.nu_linear_search(None, None, ctypes.c_int64(0), None, 0, 0,
                              None, 0, None, None, None, None)
    assert st == 1
    lib.nu_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.nu_version()
