"""Argument checks of the C ABI that run before any device call (CPU only).

Every entry point refuses a null handle or pointer, an unknown layout, dtype or op, and
out-of-range sizes with a status and a message from spmv_last_error(), and never aborts.
Only checks that precede the first CUDA call are exercised here: they need no GPU.
"""
import ctypes

import pytest

from paper_1812_00904_gb300 import _lib

OK, INVALID, BAD_MATRIX, UNSUPPORTED = 0, 1, 2, 8
CSC, CSR = 0, 1
F64, F32, BF16 = 0, 1, 2


@pytest.fixture(scope="module")
def lib():
    from paper_1812_00904_gb300 import build

    return _lib.load(build.build())


def _msg(lib):
    return lib.spmv_last_error().decode()


def _plan(lib, m=4, n=8, nnz=0, layout=CSC, ptr=0x1000, idx=0x2000, vals=0x3000, vt=F32, xt=F32, flags=0):
    out = ctypes.c_void_p()
    return lib.spmv_plan(ctypes.byref(out), m, n, nnz, layout, ptr, idx, vals, vt, xt, None, flags), out


def test_plan_creation_rejects_bad_arguments_before_touching_the_device(lib):
    assert lib.spmv_plan(None, 4, 8, 0, CSC, 0x1000, None, None, F32, F32, None, 0) == INVALID
    assert "out" in _msg(lib)
    st, out = _plan(lib, layout=2)
    assert st == INVALID and "layout" in _msg(lib) and out.value is None
    for m, n, nnz in ((-1, 8, 0), (4, -1, 0), (4, 8, -1), (1 << 31, 8, 0), (4, 8, 1 << 31)):
        assert _plan(lib, m=m, n=n, nnz=nnz)[0] == INVALID
    assert _plan(lib, vt=9)[0] == INVALID and "dtype" in _msg(lib)
    assert _plan(lib, vt=F32, xt=F64)[0] == UNSUPPORTED  # FP32 values need FP32 vectors
    assert _plan(lib, vt=BF16, xt=BF16)[0] == UNSUPPORTED
    assert _plan(lib, ptr=None)[0] == INVALID and "ptr" in _msg(lib)
    assert _plan(lib, nnz=3, idx=None)[0] == INVALID
    assert _plan(lib, nnz=3, m=0)[0] == BAD_MATRIX  # nonzeros of a wide matrix without rows
    assert _plan(lib, nnz=3, n=0, layout=CSR)[0] == BAD_MATRIX
    assert _plan(lib, ptr=0x1004)[0] == INVALID and "aligned" in _msg(lib)
    assert _plan(lib, nnz=3, vals=0x3002)[0] == INVALID


def test_triple_plans_reject_bad_arguments(lib):
    out = ctypes.c_void_p()

    def coo(m=4, n=8, nnz=3, layout=CSC, rows=0x1000, cols=0x2000, vals=0x3000, vt=F32, flags=0):
        return lib.spmv_plan_coo(ctypes.byref(out), m, n, nnz, layout, rows, cols, vals, vt, F32, None, flags, None)

    assert lib.spmv_plan_coo(None, 4, 8, 0, CSC, None, None, None, F32, F32, None, 0, None) == INVALID
    assert coo(layout=5) == INVALID
    assert coo(nnz=-2) == INVALID
    assert coo(rows=None) == INVALID
    assert coo(vt=7, flags=0x10) == INVALID  # unsorted triples of an unknown value type
    assert coo(n=0) == BAD_MATRIX and "nonempty" in _msg(lib)


def test_calls_on_a_null_plan_fail_with_a_status(lib):
    assert lib.spmv_plan_destroy(None) == OK
    assert lib.spmv(None, None, None, None) == INVALID and "plan" in _msg(lib)
    assert lib.spvtm(None, None, None, None) == INVALID
    assert lib.spmv_batch(None, 0, 1, None, 0, None, 0, None) == INVALID
    assert lib.spmv_dvalues(None, None, None, None, None) == INVALID
    assert lib.spmv_check(None, None) == INVALID
    assert lib.spmv_plan_export(None, None, None, None) == INVALID
    assert lib.spmv_profile_enable(None, 1) == INVALID
    assert lib.spmv_profile_reset(None) == INVALID
    ms, n = ctypes.c_double(), ctypes.c_int64()
    assert lib.spmv_profile_read(None, 0, ctypes.byref(ms), ctypes.byref(n)) == INVALID
    info = _lib.spmv_plan_info_t()
    assert lib.spmv_plan_info(None, ctypes.byref(info)) == INVALID
    chunks = (_lib.spmv_chunk_t * 1)()
    assert lib.spmv_plan_chunks(None, chunks, 1) == INVALID
    assert lib.spmv_normal(None, None, None, None, None) == INVALID
    it, rel = ctypes.c_int32(), ctypes.c_double()
    assert lib.spmv_cgls(None, None, None, 5, 1e-6, None, ctypes.byref(it), ctypes.byref(rel)) == INVALID


def test_allocation_free_entry_checks_sizes(lib):
    assert lib.spmv_noalloc(-1, 8, 0, None, None, None, None, None, None) == INVALID
    assert lib.spmv_noalloc(49153, 8, 0, 0x1000, None, None, None, 0x2000, None) == INVALID
    assert "49152" in _msg(lib)


def test_serving_calls_check_their_arguments(lib):
    srv = ctypes.c_void_p()
    assert lib.serve_create(None, 1 << 30, 32, 4) == INVALID
    assert lib.serve_create(ctypes.byref(srv), 1 << 30, 0, 4) == INVALID and srv.value is None
    assert lib.serve_create(ctypes.byref(srv), 1 << 30, 32, 17) == INVALID
    mid, rid = ctypes.c_int32(), ctypes.c_uint64()
    assert lib.serve_register(None, None, ctypes.byref(mid)) == INVALID
    assert lib.serve_register_host(None, 4, 8, 0, CSC, None, None, None, F32, F32, ctypes.byref(mid)) == INVALID
    assert lib.serve_submit(None, 0, 0, 1, None, None, ctypes.byref(rid)) == INVALID
    done, lat = ctypes.c_int32(), ctypes.c_double()
    assert lib.serve_poll(None, 1, ctypes.byref(done), ctypes.byref(lat)) == INVALID
    assert lib.serve_wait(None, 1, 10) == INVALID
    assert lib.serve_stats(None, None) == INVALID
