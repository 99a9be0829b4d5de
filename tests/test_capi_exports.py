"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h (no compute calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cs_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2606_12577_gb300 import build
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc unavailable")
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("cs_setup_hierarchy", "cs_setup_cascade", "cs_vcycle", "cs_solve", "cs_smooth",
                     "cs_residual_restrict", "cs_prolong_correct", "cs_coarse_solve", "cs_export_lambda"):
        assert required in names


def test_library_exports_all_declared_symbols(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, f"missing exports: {missing}"


def test_binding_declares_every_export(lib_path):
    from paper_2606_12577_gb300 import _capi
    assert set(_capi.EXPORTED) >= _declared()
    _capi.lib()  # loads and sets every signature


def test_last_error_without_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.cs_last_error.restype = ctypes.c_char_p
    lib.cs_setup_hierarchy.restype = ctypes.c_int
    # a null stencil is rejected on the host before any CUDA call
    assert lib.cs_setup_hierarchy(None, None, None, None) == -1
    assert b"null" in lib.cs_last_error()
