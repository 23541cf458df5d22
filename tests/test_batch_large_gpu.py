"""Multi-vector products with a short vector too long for several copies on chip (m = 20,000).

Up to 8 vectors per pass are read from an interleaved global copy, so the matrix streams once
per 8 vectors: in the segmented direction (u^T = V^T A of a wide matrix) on every plan, and in
the accumulating direction (Y = A X) on plans with the row-sorted copy.  Every vector must
match the FP64 oracle, and equal its single-vector product bit for bit wherever the path adds
in a fixed order (both directions with the copy, the segmented one without).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
from types import SimpleNamespace  # noqa: E402

import paper_1812_00904_gb300 as pkg  # noqa: E402
from gpu_util import DEV, assert_close, host_of, make_plan  # noqa: E402

THREADS = 8


@pytest.fixture(scope="module")
def big():
    """m = 20,000, n = 300,000, power-law column degrees (about 30M nonzeros, repeated rows allowed)."""
    rng = np.random.default_rng(61)
    deg = np.minimum((25.0 * rng.random(300_000) ** -1.0).astype(np.int64), 20_000)
    A = synth.random_matrix(20_000, 300_000, "csc", degrees=deg, seed=62, duplicates=True)
    A.vals = np.asarray(A.vals, np.float32).astype(np.float64)
    return A


def _abs(A):
    return SimpleNamespace(layout=A.layout, m=A.m, n=A.n, ptr=A.ptr, idx=A.idx, vals=np.abs(A.vals))


@pytest.mark.parametrize("k", [8, 32])
@pytest.mark.parametrize("flags", [0, pkg.SPMV_PLAN_ROW_BLOCKS], ids=["atomic", "row_blocks"])
def test_batched_products_on_a_long_short_vector(big, k, flags):
    A = big
    plan, stored = make_plan(A, torch.float32, flags=flags)
    info = plan.info()
    assert info["batch_width"] < 8  # several short vectors do not fit on chip beside the staging
    assert (info["row_blocks"] > 0) == bool(flags)
    g = torch.Generator(device=DEV)
    g.manual_seed(63)
    X = torch.rand((k, A.n), generator=g, device=DEV) * 2 - 1
    V = torch.rand((k, A.m), generator=g, device=DEV) * 2 - 1
    Y = plan.batch(pkg.SPMV_OP_AX, X)
    U = plan.batch(pkg.SPMV_OP_VTA, V)
    plan.check()
    Aa = _abs(stored)
    for b in range(k):
        xs, vs = host_of(X[b]), host_of(V[b])
        assert_close(host_of(Y[b]), oracle.spmv_mt(stored, xs, THREADS), oracle.spmv_mt(Aa, np.abs(xs), THREADS),
                     1e-5, f"Y[{b}]")
        assert_close(host_of(U[b]), oracle.spvtm_mt(stored, vs, THREADS), oracle.spvtm_mt(Aa, np.abs(vs), THREADS),
                     1e-5, f"U[{b}]")
    for b in (0, k // 2, k - 1):
        assert torch.equal(U[b], plan.spvtm(V[b])), f"U[{b}] differs from its single-vector product"
        if flags:
            assert torch.equal(Y[b], plan.spmv(X[b])), f"Y[{b}] differs from its single-vector product"
    plan.close()
