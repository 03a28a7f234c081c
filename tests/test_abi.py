"""CPU-only checks of the C ABI: libtsvd.so builds, loads without a GPU and
exports every symbol include/tsvd.h declares; argument errors are reported
without touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "tsvd.h")).read()
    return sorted(set(re.findall(r"TSVD_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_04989_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ["tsvd_rbk", "tsvd_rbk_workspace_size", "tprod", "tprod_backward", "tproj", "tproj_backward"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_header():
    from paper_2504_04989_gb300 import _lib
    assert set(declared_symbols()) <= set(_lib.SIGNATURES)


def test_argument_errors_without_gpu(lib):
    from paper_2504_04989_gb300 import _lib
    p = _lib.TsvdParams(R=5, P=2, q=1, precision=1, seed=0, flags=0)
    n = C.c_size_t()
    assert lib.tsvd_rbk_workspace_size(32, 32, 8, C.byref(p), C.byref(n)) == 0 and n.value > 0
    bad = _lib.TsvdParams(R=40, P=2, q=1, precision=1, seed=0, flags=0)  # R > min(n1, n2)
    assert lib.tsvd_rbk_workspace_size(32, 32, 8, C.byref(bad), C.byref(n)) == -1
    big = _lib.TsvdParams(R=100, P=40, q=1, precision=1, seed=0, flags=0)  # R + P > 128
    assert lib.tsvd_rbk_workspace_size(512, 512, 8, C.byref(big), C.byref(n)) == -4
    assert lib.tsvd_rbk(None, 32, 32, 8, C.byref(p), None, None, None, None, None, None, 0, None, None) == -1
    assert lib.tprod_workspace_size(0, 3, 3, 3, 1, C.byref(n)) == -1
    assert lib.tqr_workspace_size(0, 3, 3, 0, C.byref(n)) == -1
    assert lib.tpinv_workspace_size(4, 3, 3, 2, C.byref(n)) == -1  # FP64 / FP32 only
    assert lib.tqr_workspace_size(40, 30, 8, 0, C.byref(n)) == 0 and n.value > 0
    assert lib.tqr(None, 4, 3, 3, 0, None, None, None, 0, None, None) == -1
    assert lib.tsvd_strerror(-2) == b"workspace too small"
    assert lib.tsvd_version() >= 100
