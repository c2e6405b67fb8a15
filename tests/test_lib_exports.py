"""The C-ABI library builds for sm_103a, loads, and exports every entry point of
include/trevr.h (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(trevr_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1902_08083_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "trevr_build_tree" in names and "trevr_compute_flux" in names
    for name in sorted(names):
        assert hasattr(lib, name), name


def test_binding_lists_every_symbol():
    from paper_1902_08083_gb300 import trevr
    assert set(trevr.EXPORTS) == _declared()


def test_status_strings(lib):
    lib.trevr_status_string.restype = ctypes.c_char_p
    assert lib.trevr_status_string(0) == b"ok"
    assert lib.trevr_status_string(2) == b"point outside the domain"


def test_host_side_argument_checks(lib):
    # null arguments are rejected on the host before any CUDA call
    lib.trevr_build_tree.restype = ctypes.c_int
    out = ctypes.c_void_p()
    rc = lib.trevr_build_tree(None, None, None, ctypes.c_longlong(10), None, None,
                              ctypes.c_longlong(0), None, None, None, ctypes.byref(out))
    assert rc == 1 and not out.value
    lib.trevr_compute_flux.restype = ctypes.c_int
    assert lib.trevr_compute_flux(None, None, ctypes.c_longlong(0), None, None, None, None,
                                  None) == 1
