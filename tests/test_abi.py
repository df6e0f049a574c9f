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


def test_matching_argument_validation(lib):
    """hs_matching rejects bad arguments before any device call (host-side checks)."""
    from paper_1611_00606_gb300 import hs
    restype, argtypes = hs.SIGNATURES["hs_matching"]
    f = lib.hs_matching
    f.restype, f.argtypes = restype, argtypes
    p = C.c_void_p(16)   # stand-in addresses: never dereferenced on these paths
    q = C.c_void_p(32)

    def call(K=p, tau=p, R=p, u=p, omega=1.0, N_A=2, l_max=3, N_G=8, A=p, B=q, ld=32):
        return f(K, tau, R, u, omega, N_A, l_max, N_G, A, B, ld, None)

    assert call(K=None) == -1 and call(tau=None) == -1 and call(R=None) == -1
    assert call(u=None) == -1 and call(A=None) == -1 and call(B=None) == -1
    assert call(B=p) == -1                       # A and B the same buffer
    assert call(N_A=0) == -1 and call(l_max=-1) == -1 and call(l_max=12) == -1
    assert call(N_G=-1) == -1
    assert call(omega=0.0) == -1 and call(omega=-2.0) == -1 and call(omega=float("nan")) == -1
    assert call(ld=31) == -1                     # below N_A (l_max + 1)^2 = 32
    assert call(N_G=0) == 0                      # nothing to do, nothing touched
