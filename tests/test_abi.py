"""The C-ABI library builds, loads and exports every symbol include/hs.h declares.

No GPU needed: only argument validation paths (which return before any CUDA
call) are exercised here.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hs.h")
LIB = os.path.join(ROOT, "paper_1611_00606_gb300", "libhs.so")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1611_00606_gb300 import build
        build.build()
    return C.CDLL(LIB)


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hs_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("hs_plan", "hs_assemble", "hs_submit", "hs_poll", "hs_destroy", "hs_strerror",
              "hs_footprint", "hs_fallback_flags", "hs_set_t", "hs_assemble_host"):
        assert s in syms


def test_every_declared_symbol_is_exported(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_signatures_cover_header():
    from paper_1611_00606_gb300 import hs
    assert set(declared_symbols()) <= set(hs.SIGNATURES)


def test_strerror_and_argument_validation(lib):
    lib.hs_strerror.restype = C.c_char_p
    assert lib.hs_strerror(0) == b"ok"
    assert b"invalid" in lib.hs_strerror(-1)
    h = C.c_void_p()
    # bad sizes / precision / slice count are rejected before touching the device
    assert lib.hs_plan(C.byref(h), 0, 16, 100, 0, 0, C.c_size_t(0), None) == -1
    assert lib.hs_plan(C.byref(h), 4, 0, 100, 0, 0, C.c_size_t(0), None) == -1
    assert lib.hs_plan(C.byref(h), 4, 500, 100, 0, 0, C.c_size_t(0), None) == -1
    assert lib.hs_plan(C.byref(h), 4, 16, 0, 0, 0, C.c_size_t(0), None) == -1
    assert lib.hs_plan(C.byref(h), 4, 16, 100, 9, 0, C.c_size_t(0), None) == -1
    assert lib.hs_plan(C.byref(h), 4, 16, 100, 1, 1, C.c_size_t(0), None) == -1
    assert lib.hs_plan(C.byref(h), 4, 16, 100, 1, 8, C.c_size_t(0), None) == -1
    assert lib.hs_plan(None, 4, 16, 100, 0, 0, C.c_size_t(0), None) == -1
    lib.hs_footprint.restype = C.c_size_t
    assert lib.hs_footprint(None, 10) == 0
    assert lib.hs_destroy(None) == -1
