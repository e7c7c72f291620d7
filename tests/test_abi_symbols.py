"""The C-ABI library loads and exports every entry point include/ffc.h declares.

No compute call is made (no GPU needed); the library is built here if absent.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ffc.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ffc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1409_2802_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    return _build.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("ffc_sample_rows", "ffc_eval_block", "ffc_id", "ffc_id_error", "ffc_compress_tree",
                 "ffc_tree_result_free", "ffc_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_export(libpath):
    from paper_1409_2802_gb300 import ffc
    assert set(ffc.EXPORTS) == set(_declared())
    assert ffc.lib().ffc_tree_depth(65536, 256) == 8
    assert ffc.lib().ffc_tree_depth(100000, 512) == 8
    assert ffc.version().startswith("ffc")


def test_invalid_arguments_rejected_before_launch(libpath):
    """Argument validation needs no GPU: a bad call returns FFC_E_INVALID."""
    from paper_1409_2802_gb300 import ffc
    L = ffc.lib()
    rank, r22 = ctypes.c_int64(0), ctypes.c_double(0)
    # ldk < s
    st = L.ffc_id(None, 10, 5, 4, 0, 3, 0.0, None, None, 3, ctypes.byref(rank), ctypes.byref(r22), None)
    assert st == ffc.FFC_E_INVALID
    assert b"ldk" in L.ffc_last_error()
    # too many rows for the QR
    st = L.ffc_id(None, 4096, 5, 4096, 0, 3, 0.0, None, None, 3, ctypes.byref(rank), ctypes.byref(r22), None)
    assert st == ffc.FFC_E_INVALID
    # Laplace in d = 2
    err = ctypes.c_double(0)
    st = L.ffc_id_error(ffc.Kernel(ffc.LAPLACE).c_struct(), None, 0, None, 4, None, 3, 2, None, None, 1, 1,
                        ctypes.byref(err), None)
    assert st == ffc.FFC_E_INVALID
