"""The C ABI library loads and exports every function include/spmv_gb300.h declares (CPU only, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spmv_gb300.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:spmv_status|const char \*)\s*(\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1812_00904_gb300 import build

    return build.build()


def test_header_lists_the_boundary():
    names = header_functions()
    for required in ("spmv_plan", "spmv", "spvtm", "spmv_batch", "spmv_dvalues", "spmv_plan_destroy",
                     "spmv_last_error", "serve_create", "serve_register", "serve_submit", "serve_poll", "serve_wait",
                     "serve_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_the_header(lib_path):
    from paper_1812_00904_gb300 import _lib

    assert sorted(_lib.SIGNATURES) == header_functions()
    lib = _lib.load(lib_path)
    assert lib.spmv_version().decode().startswith("spmv_gb300")
    assert isinstance(lib.spmv_last_error().decode(), str)  # the last error of this thread, if any


def test_missing_library_fails_loudly(tmp_path):
    from paper_1812_00904_gb300 import _lib

    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="no fallback"):
            _lib.load(str(tmp_path / "absent.so"))
    finally:
        _lib._lib = saved
