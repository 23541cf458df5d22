"""Special values through every accumulation stage: infinities and NaNs give what the plain sum
gives (the oracle's IEEE FP64 loops), also where they meet the compensated carry of a segment
split over several tiles and chunks and the zone fix-up; subnormal products add exactly in the
segmented passes, the shared-memory atomic pass, the FP64 combines and the zone fix-up (the
widening of FP32 partials and carry records to FP64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402

import paper_1812_00904_gb300 as pkg  # noqa: E402
from gpu_util import TOL, assert_close, dev_vec, host_of, make_plan  # noqa: E402

TINY = 2.0 ** -140  # an FP32 subnormal; products of it with +-1 are exact


def _matrix(layout, n_major, n_minor, seed, long_segments):
    """Random degrees with some long segments (each split over many tiles of 64 nonzeros)."""
    rng = np.random.default_rng(seed)
    deg = rng.integers(0, 12, size=n_major)
    for j, d in long_segments.items():
        deg[j] = d
    m, n = (n_minor, n_major) if layout == "csc" else (n_major, n_minor)
    return synth.random_matrix(m, n, layout, degrees=deg, seed=seed)


def _check_classes(got, ref, scale, tol, what):
    """Non-finite expected values exactly (NaN as NaN, infinities with their sign), the rest
    within the tolerance."""
    got = np.asarray(got, dtype=np.float64)
    nan_ref = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan_ref), f"{what}: NaN positions differ"
    inf_ref = np.isinf(ref)
    assert np.array_equal(got[inf_ref], ref[inf_ref]), f"{what}: infinities differ"
    fin = np.isfinite(ref)
    assert np.all(np.isfinite(got[fin])), f"{what}: a finite sum came out non-finite"
    assert_close(got[fin], ref[fin], scale[fin], tol, what)


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64, torch.bfloat16], ids=str)
def test_infinities_and_nans_follow_the_plain_sum(layout, dtype):
    n_major, n_minor = 40_000, 3000
    A = _matrix(layout, n_major, n_minor, 3, {7: 2500, 11: 2000, 13: 1500, 17: 900})
    vals = np.asarray(A.vals, dtype=np.float64).copy()
    ptr = np.asarray(A.ptr)
    vals[ptr[7]] = np.inf          # +inf at the start and -inf at the end of one long segment: NaN
    vals[ptr[8] - 1] = -np.inf
    vals[ptr[11] + 1000] = np.inf  # one infinity inside a long segment: the carry must stay infinite
    vals[ptr[13] + 700] = np.nan   # one NaN
    vals[ptr[17] + 5] = -np.inf    # and one in a segment of two chunks
    A = synth.SparseMatrix(A.layout, A.m, A.n, A.ptr, A.idx, vals)
    plan, stored = make_plan(A, dtype, tile_items=64)
    x = dev_vec(synth.uniform_vector(A.n, 1), plan.vec_dtype)
    v = dev_vec(synth.uniform_vector(A.m, 2), plan.vec_dtype)
    y = host_of(plan.spmv(x))
    u = host_of(plan.spvtm(v))
    plan.check()
    xs, vs = host_of(x), host_of(v)
    ry, ru = oracle.spmv(stored, xs), oracle.spvtm(stored, vs)
    assert (~np.isfinite(ry)).sum() >= 3 and (~np.isfinite(ru)).sum() >= 3  # the planted values arrive
    tol = TOL[dtype]
    _check_classes(y, ry, oracle.abs_spmv(stored, xs), tol, f"{layout} {dtype} spmv")
    _check_classes(u, ru, oracle.abs_spvtm(stored, vs), tol, f"{layout} {dtype} spvtm")
    # the same through the multi-vector pass of the segmented direction
    z0 = v if layout == "csc" else x
    Z = torch.stack([z0, -z0, 2 * z0])
    R = plan.batch(pkg.SPMV_OP_VTA if layout == "csc" else pkg.SPMV_OP_AX, Z)
    plan.check()
    for b in range(3):
        zs = host_of(Z[b])
        if layout == "csc":
            ref, sc = oracle.spvtm(stored, zs), oracle.abs_spvtm(stored, zs)
        else:
            ref, sc = oracle.spmv(stored, zs), oracle.abs_spmv(stored, zs)
        _check_classes(host_of(R[b]), ref, sc, tol, f"{layout} {dtype} batch vector {b}")
    plan.close()


def _tiny_matrix(layout, seed):
    A = _matrix(layout, 30_000, 20_000, seed, {5: 15_000, 9: 6000, 21: 3000})
    sign = np.where(np.random.default_rng(seed).random(A.nnz) < 0.5, -1.0, 1.0)
    return synth.SparseMatrix(A.layout, A.m, A.n, A.ptr, A.idx, TINY * sign)


def _signs(length, seed):
    return np.where(np.random.default_rng(seed).random(length) < 0.5, -1.0, 1.0)


@pytest.mark.parametrize("layout", ["csc", "csr"])
def test_subnormal_products_add_exactly_in_the_segmented_pass(layout):
    """Sums of products +-2^-140 are multiples of 2^-149 well inside FP32: every partial, carry
    record and zone sum is exact, so the result equals the oracle's bit for bit."""
    A = _tiny_matrix(layout, 4)
    plan, stored = make_plan(A, torch.float32, tile_items=64)
    seg_len = A.m if layout == "csc" else A.n  # input length of the segmented direction
    z = dev_vec(_signs(seg_len, 6), torch.float32)
    out = plan.spvtm(z) if layout == "csc" else plan.spmv(z)
    plan.check()
    ref = oracle.spvtm(stored, host_of(z)) if layout == "csc" else oracle.spmv(stored, host_of(z))
    ref32 = torch.from_numpy(ref).float()
    assert np.count_nonzero(ref) > 1000 and np.abs(ref).max() < 2.0 ** -120
    assert torch.equal(out.cpu(), ref32), "subnormal segment sums differ from the exact ones"
    plan.close()


@pytest.mark.parametrize("layout", ["csc", "csr"])
def test_subnormal_products_add_exactly_in_the_atomic_pass(layout):
    """The accumulating direction: FP32 shared-memory atomic adds of subnormal products keep
    them (no flush to zero), and the FP64 combine of the per-CTA partials is exact."""
    A = _tiny_matrix(layout, 10)
    plan, stored = make_plan(A, torch.float32)
    acc_in = A.n if layout == "csc" else A.m  # input length of the accumulating direction
    z = dev_vec(_signs(acc_in, 11), torch.float32)
    out = plan.spmv(z) if layout == "csc" else plan.spvtm(z)
    plan.check()
    ref = oracle.spmv(stored, host_of(z)) if layout == "csc" else oracle.spvtm(stored, host_of(z))
    assert np.count_nonzero(ref) > 1000
    assert torch.equal(out.cpu(), torch.from_numpy(ref).float()), "atomic subnormal sums differ from the exact ones"
    plan.close()


def test_subnormal_partials_combine_exactly_over_row_blocks():
    """The accumulating direction over the row-sorted copy: segmented block sums of subnormal
    products, then the FP64 combine of the blocks' FP32 partials (widened exactly)."""
    B = _matrix("csc", 400_000, 500, 8, {})  # about 16 nonzeros per (block, row) segment
    sign = np.where(np.random.default_rng(8).random(B.nnz) < 0.5, -1.0, 1.0)
    A = synth.SparseMatrix(B.layout, B.m, B.n, B.ptr, B.idx, TINY * sign)
    plan, stored = make_plan(A, torch.float32, flags=pkg.SPMV_PLAN_ROW_BLOCKS)
    assert plan.info()["row_blocks"] > 0
    x = dev_vec(_signs(A.n, 9), torch.float32)
    y = plan.spmv(x)
    plan.check()
    ref = oracle.spmv(stored, host_of(x))
    assert np.count_nonzero(ref) > 400
    assert torch.equal(y.cpu(), torch.from_numpy(ref).float()), "combined subnormal partials differ from the exact sums"
    plan.close()
