"""Multi-vector segmented passes with one vector per lane of a lane group (MODE_VSEG).

Every vector's product must equal its single-vector product bit for bit (both passes form
each sum with the same operations in the same order: the prefix over a lane's 8 positions,
the butterfly or segmented scan over the 32 lanes of a step, the compensated carry, the zone
fix-up), whatever the batch width k, the value type, the tile size, empty or repeated
segments and unvalidated indices; and it must match the FP64 oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402

import paper_1812_00904_gb300 as pkg  # noqa: E402
from gpu_util import DEV, TOL, assert_close, dev_vec, host_of, make_plan  # noqa: E402


def _seg_op(layout):
    return pkg.SPMV_OP_VTA if layout == "csc" else pkg.SPMV_OP_AX


def _inputs(A, layout, k, seed):
    """k vectors of the segmented direction's input length (the short dimension; vector
    lengths here are multiples of 4, so that the rows of the stacked batch stay 16-byte aligned)."""
    ln = A.m if layout == "csc" else A.n
    return [synth.uniform_vector(ln, seed + b) for b in range(k)]


def _check_every_vector(plan, stored, layout, vecs, dtype, what):
    Z = torch.stack([dev_vec(v, plan.vec_dtype) for v in vecs])
    op = _seg_op(layout)
    R = plan.batch(op, Z)
    plan.check()
    for b in range(len(vecs)):
        single = plan.spvtm(Z[b]) if op == pkg.SPMV_OP_VTA else plan.spmv(Z[b])
        assert torch.equal(single, R[b]), f"{what}: vector {b} of {len(vecs)} differs from its single-vector product"
    for b in {0, len(vecs) - 1}:
        zs = host_of(Z[b])
        if op == pkg.SPMV_OP_VTA:
            ref, scale = oracle.spvtm(stored, zs), oracle.abs_spvtm(stored, zs)
        else:
            ref, scale = oracle.spmv(stored, zs), oracle.abs_spmv(stored, zs)
        assert_close(host_of(R[b]), ref, scale, TOL[dtype], f"{what}: vector {b}")


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16], ids=str)
@pytest.mark.parametrize("k", [2, 4, 6, 8, 11, 16, 19])
def test_every_vector_equals_its_single_product(layout, dtype, k):
    rng = np.random.default_rng(k)
    n_major = 60_000
    deg = np.minimum((4.0 * rng.random(n_major) ** -1.0).astype(np.int64), 1500)
    deg[rng.choice(n_major, 500, replace=False)] = 0  # empty segments
    deg[123] = 1500  # a long one, split over many steps and tiles
    m, n = (1500, n_major) if layout == "csc" else (n_major, 1500)
    A = synth.random_matrix(m, n, layout, degrees=deg, seed=30 + k)
    plan, stored = make_plan(A, dtype)
    _check_every_vector(plan, stored, layout, _inputs(A, layout, k, 100 * k), dtype, f"{layout} {dtype} k={k}")
    plan.close()


@pytest.mark.parametrize("tile_items", [40, 104, 256, 512])
@pytest.mark.parametrize("flags", [0, pkg.SPMV_PLAN_NO_VALIDATE], ids=["validated", "unvalidated"])
def test_partial_steps_repeated_indices_and_unvalidated_plans(tile_items, flags):
    rng = np.random.default_rng(tile_items)
    deg = rng.integers(0, 40, size=30_000)
    A = synth.random_matrix(900, 30_000, "csc", degrees=deg, seed=5, duplicates=True)
    plan, stored = make_plan(A, torch.float32, tile_items=tile_items, flags=flags)
    _check_every_vector(plan, stored, "csc", _inputs(A, "csc", 8, 7), torch.float32, f"T={tile_items}")
    plan.close()


@pytest.mark.parametrize("shape", ["one_column", "short_columns", "tiny"])
def test_degenerate_shapes(shape):
    if shape == "one_column":  # every tile inside one segment: head-free steps and zones only
        A = synth.random_matrix(3000, 4, "csc", degrees=np.array([0, 2900, 0, 0]), seed=1)
    elif shape == "short_columns":  # a head in nearly every virtual lane, several in most
        A = synth.random_matrix(400, 200_000, "csc", degrees=np.random.default_rng(2).integers(1, 4, 200_000), seed=2)
    else:  # fewer nonzeros than one step
        A = synth.random_matrix(52, 32, "csc", degrees=np.arange(32) % 5, seed=3)
    plan, stored = make_plan(A, torch.float32)
    _check_every_vector(plan, stored, "csc", _inputs(A, "csc", 5, 11), torch.float32, shape)
    plan.close()


def test_row_sorted_copy_batched_spmv_equals_single():
    """The accumulating direction over the row-sorted copy runs as a windowed segmented pass:
    k vectors in one pass equal their single-vector products."""
    rng = np.random.default_rng(9)
    deg = np.minimum((3.0 * rng.random(200_000) ** -1.0).astype(np.int64), 3000)
    A = synth.random_matrix(3000, 200_000, "csc", degrees=deg, seed=9)
    plan, stored = make_plan(A, torch.float32, flags=pkg.SPMV_PLAN_ROW_BLOCKS)
    assert plan.info()["row_blocks"] > 0
    X = torch.stack([dev_vec(synth.uniform_vector(A.n, 40 + b), torch.float32) for b in range(12)])
    Y = plan.batch(pkg.SPMV_OP_AX, X)
    plan.check()
    for b in range(12):
        assert torch.equal(plan.spmv(X[b]), Y[b]), f"vector {b}"
    xs = host_of(X[11])
    assert_close(host_of(Y[11]), oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), 1e-5, "row blocks k=12")
    plan.close()


def test_batch_results_do_not_depend_on_the_batch():
    """The same vector in batches of different widths and positions gives the same bits."""
    A = synth.random_matrix(2000, 80_000, "csc", density=0.003, seed=4)
    plan, _ = make_plan(A, torch.float32)
    vs = [dev_vec(v, torch.float32) for v in _inputs(A, "csc", 16, 500)]
    ref = plan.batch(pkg.SPMV_OP_VTA, torch.stack(vs))
    for k in (2, 3, 5, 9, 13):
        R = plan.batch(pkg.SPMV_OP_VTA, torch.stack(vs[16 - k:]))
        for b in range(k):
            assert torch.equal(R[b], ref[16 - k + b]), (k, b)
    plan.check()
    plan.close()
