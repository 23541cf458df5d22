"""Parity at the full workload sizes, in the launch configuration the benchmark times.

The wide matrix (m = 20,000, n = 5,000,000, about 200M nonzeros, FP32 and BF16 values)
and the tall one (m = 10,000,000, n = 2,000, about 150M nonzeros) are checked element
by element against the FP64 oracle run on the same stored values and vectors (the
oracle's straight loops take about a second at these sizes), plus the adjoint
identity v^T (A x) = (v^T A) x, which holds at any size.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
import paper_1812_00904_gb300 as pkg  # noqa: E402
from gpu_util import DEV, assert_close, host_of  # noqa: E402


def _host(A, vals_dtype=None):
    v = A.vals if vals_dtype is None else A.vals.to(vals_dtype)
    return synth.SparseMatrix(A.layout, A.m, A.n, A.ptr.cpu().numpy(), A.idx.cpu().numpy(),
                              v.double().cpu().numpy()), v


# the benchmark's plans: bank-ordered nonzeros (its row-block variant adds the row-sorted copy)
BENCH_FLAGS = pkg.SPMV_PLAN_BANK_ORDER


def _check(A, val_dtype, what, flags=BENCH_FLAGS):
    stored, vals = _host(A, val_dtype)
    plan = pkg.Plan(A.m, A.n, A.ptr, A.idx, vals, layout=A.layout, vec_dtype=torch.float32, flags=flags)
    g = torch.Generator(device=DEV)
    g.manual_seed(11)
    x = torch.rand(A.n, generator=g, device=DEV) * 2 - 1
    v = torch.rand(A.m, generator=g, device=DEV) * 2 - 1
    y = host_of(plan.spmv(x))
    u = host_of(plan.spvtm(v))
    plan.check()
    xs, vs = host_of(x), host_of(v)
    y_ref, u_ref = oracle.spmv(stored, xs), oracle.spvtm(stored, vs)
    assert_close(y, y_ref, oracle.abs_spmv(stored, xs), 1e-5, f"{what} y = A x")
    assert_close(u, u_ref, oracle.abs_spvtm(stored, vs), 1e-5, f"{what} u = v^T A")
    # adjoint identity at full size: v^T (A x) = (v^T A) x up to the accumulated rounding
    lhs, rhs = float(np.dot(vs, y)), float(np.dot(u, xs))
    scale = float(np.dot(np.abs(vs), oracle.abs_spmv(stored, xs)))
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs, scale)
    info = plan.info()
    plan.close()
    return stored, info


def test_wide_fp32_full_size():
    A = synth.wide_fp32_large(1, device=DEV)
    _, info = _check(A, None, "wide fp32")
    assert info["tile_items"] == 512 and info["stages"] == 2  # the benchmark's configuration


def test_wide_fp32_full_size_row_blocks():
    """The same matrix with the row-sorted copy: SpMV as segmented dot products over block windows."""
    A = synth.wide_fp32_large(1, device=DEV)
    _, info = _check(A, None, "wide fp32 row blocks", flags=BENCH_FLAGS | pkg.SPMV_PLAN_ROW_BLOCKS)
    assert info["row_blocks"] > 0


def test_wide_fp32_full_size_stored_order():
    """The same matrix in the caller's order, no plan-owned copies."""
    A = synth.wide_fp32_large(1, device=DEV)
    _, info = _check(A, None, "wide fp32 stored order", flags=0)
    assert info["row_blocks"] == 0


def test_wide_bf16_values_full_size():
    A = synth.wide_fp32_large(1, device=DEV)
    stored, _ = _check(A, torch.bfloat16, "wide bf16")
    # normwise against the unrounded FP32 values: the BF16 storage error stays below 1e-2
    exact, _ = _host(A)
    x = synth.uniform_vector(A.n, 3)
    y_b, y_e = oracle.spmv(stored, x), oracle.spmv(exact, x)
    assert np.linalg.norm(y_b - y_e) <= 1e-2 * np.linalg.norm(y_e)


def test_tall_fp32_full_size():
    A = synth.tall_fp32_large(2, device=DEV)
    _check(A, None, "tall fp32")
    _, info = _check(A, None, "tall fp32 row blocks", flags=BENCH_FLAGS | pkg.SPMV_PLAN_ROW_BLOCKS)
    assert info["row_blocks"] > 0


def test_wide_fp32_full_size_through_pinned_host_vectors():
    """The end-to-end configuration of the benchmark: the benchmark's plan and pinned host
    vectors staged by the library."""
    A = synth.wide_fp32_large(1, device=DEV)
    stored, _ = _host(A)
    plan = pkg.Plan(A.m, A.n, A.ptr, A.idx, A.vals, layout="csc", flags=BENCH_FLAGS)
    g = torch.Generator(device=DEV)
    g.manual_seed(12)
    xh = (torch.rand(A.n, generator=g, device=DEV) * 2 - 1).cpu().pin_memory()
    vh = (torch.rand(A.m, generator=g, device=DEV) * 2 - 1).cpu().pin_memory()
    yh = torch.empty(A.m, pin_memory=True)
    uh = torch.empty(A.n, pin_memory=True)
    pkg.spmv(plan.handle, xh, yh)
    pkg.spvtm(plan.handle, vh, uh)
    plan.check()
    xs, vs = xh.double().numpy(), vh.double().numpy()
    assert_close(yh.double().numpy(), oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), 1e-5, "host y = A x")
    assert_close(uh.double().numpy(), oracle.spvtm(stored, vs), oracle.abs_spvtm(stored, vs), 1e-5, "host u = v^T A")
    plan.close()
