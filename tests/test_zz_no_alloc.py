"""The allocation-free SpMV entry point (spmv_noalloc) against the planned SpMV.

Some callers may not allocate device memory when they multiply; spmv_noalloc
serves them with scratch in the library's static device memory.  This file is
collected last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402

from paper_1812_00904_gb300 import _lib  # noqa: E402
from gpu_util import DEV, assert_close, dev_vec, host_of, make_plan  # noqa: E402


def _call_noalloc(A, t, x, y):
    lib = _lib.load()
    st = lib.spmv_noalloc(A.m, A.n, A.nnz, t["ptr"].data_ptr(), t["idx"].data_ptr(), t["vals"].data_ptr(),
                          x.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st


def test_noalloc_matches_planned_spmv_twice():
    rng = np.random.default_rng(12)
    deg = np.minimum(rng.zipf(1.9, 150_000), 2500)
    deg[rng.choice(150_000, 3000, replace=False)] = 0  # some empty columns
    A = synth.random_matrix(2500, 150_000, "csc", degrees=deg, seed=13)
    plan, stored = make_plan(A, torch.float32)
    t = {"ptr": plan.ptr, "idx": plan.idx, "vals": plan.vals}
    for call, seed in enumerate((21, 22)):  # two calls in a row share the static scratch
        x = dev_vec(synth.uniform_vector(A.n, seed), torch.float32)
        y = torch.full((A.m,), float("nan"), dtype=torch.float32, device=DEV)
        assert _call_noalloc(A, t, x, y) == 0
        torch.cuda.synchronize()
        ref = host_of(plan.spmv(x))
        xs = host_of(x)
        scale = oracle.abs_spmv(stored, xs)
        assert_close(host_of(y), ref, scale, 2e-5, f"noalloc vs planned spmv, call {call}")
        assert_close(host_of(y), oracle.spmv(stored, xs), scale, 1e-5, f"noalloc vs oracle, call {call}")


def test_noalloc_rejects_oversized_short_dimension():
    A = synth.random_matrix(49153, 10, "csc", degrees=np.ones(10, np.int64), seed=3)
    plan, _ = make_plan(A, torch.float32)
    t = {"ptr": plan.ptr, "idx": plan.idx, "vals": plan.vals}
    x = torch.ones(A.n, device=DEV)
    y = torch.zeros(A.m, device=DEV)
    assert _call_noalloc(A, t, x, y) == _lib.SPMV_ERR_INVALID_ARG
    assert "49152" in _lib.load().spmv_last_error().decode()


def test_noalloc_skips_rows_outside_the_matrix():
    """Nothing is validated on this path: a nonzero whose row index lies outside [0, m) is
    skipped, so the result is the product of the matrix without those entries."""
    A = synth.random_matrix(700, 20_000, "csc", density=0.01, seed=31)
    idx = np.asarray(A.idx, np.int32).copy()
    bad = np.arange(0, A.nnz, 97)
    idx[bad] = A.m + 5 + (bad % 3)  # rows past the end of y
    vals = np.asarray(A.vals, np.float32)
    t = {"ptr": torch.from_numpy(np.asarray(A.ptr, np.int32)).to(DEV), "idx": torch.from_numpy(idx).to(DEV),
         "vals": torch.from_numpy(vals).to(DEV)}
    x = dev_vec(synth.uniform_vector(A.n, 33), torch.float32)
    y = torch.full((A.m,), float("nan"), dtype=torch.float32, device=DEV)
    assert _call_noalloc(A, t, x, y) == 0
    torch.cuda.synchronize()
    kept = vals.astype(np.float64).copy()
    kept[bad] = 0.0
    ref_m = synth.SparseMatrix("csc", A.m, A.n, A.ptr, np.where(idx < A.m, idx, 0).astype(np.int32), kept)
    xs = host_of(x)
    assert_close(host_of(y), oracle.spmv(ref_m, xs), oracle.abs_spmv(ref_m, xs) + 1e-30, 1e-5, "rows outside skipped")
