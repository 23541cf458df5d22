"""Row-sorted blocks (SPMV_PLAN_ROW_BLOCKS) against the FP64 oracle.

With the flag, the product that accumulates into the short vector (y = A x of a wide
CSC matrix, u^T = v^T A of a tall CSR one) runs as segmented dot products over each
block's window of the long vector, and the per-block vectors are added in a fixed
order: results must match the oracle within the usual tolerances and repeat bit for
bit from call to call and inside a batch.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402

import paper_1812_00904_gb300 as pkg  # noqa: E402
from gpu_util import DEV, TOL, assert_close, check_products, dev_vec, host_of, make_plan  # noqa: E402

RB = pkg.SPMV_PLAN_ROW_BLOCKS


# Row indices are drawn with repetition inside a segment (repeated entries add up), which
# keeps the generators fast and puts duplicates through the sort of the copy.


def _wide(seed=21):
    """m = 256 rows, 600k columns of power-law degree, some empty, one with 256 entries."""
    rng = np.random.default_rng(seed)
    deg = np.minimum((4.0 * rng.random(600_000) ** -1.0).astype(np.int64), 256)
    deg[rng.choice(600_000, 20_000, replace=False)] = 0
    deg[123_457] = 256
    return synth.random_matrix(256, 600_000, "csc", degrees=deg, seed=seed, duplicates=True)


def _wide_mixed(seed=22):
    """m = 500, 250k columns: Zipf degrees with long runs of short columns and five of 500 entries."""
    rng = np.random.default_rng(seed)
    deg = np.minimum(rng.zipf(1.7, 250_000), 500).astype(np.int64)
    deg[rng.choice(250_000, 5, replace=False)] = 500
    deg[:3000] = 0  # a leading run of empty columns
    return synth.random_matrix(500, 250_000, "csc", degrees=deg, seed=seed, duplicates=True)


def _tall(seed=23):
    """Tall CSR, 300k rows over 100 columns: every column is a long segment of every block."""
    rng = np.random.default_rng(seed)
    deg = np.minimum(rng.zipf(1.6, 300_000), 100).astype(np.int64)
    return synth.random_matrix(300_000, 100, "csr", degrees=deg, seed=seed, duplicates=True)


CASES = {"wide": _wide, "wide_mixed": _wide_mixed, "tall": _tall}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    return request.param, CASES[request.param]()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16, torch.float16], ids=str)
def test_row_blocks_match_oracle(case, dtype):
    name, A = case
    plan, stored = make_plan(A, dtype, flags=RB)
    info = plan.info()
    assert info["row_blocks"] > 0 and info["row_blocks"] % info["ctas"] == 0, info
    assert 0 < info["row_block_window"] <= (A.n if A.layout == "csc" else A.m)
    check_products(plan, stored, synth.uniform_vector(A.n, 31), synth.uniform_vector(A.m, 32), TOL[dtype],
                   f"{name} {dtype} row blocks")
    plan.close()


def test_row_blocks_with_bank_order(case):
    name, A = case
    plan, stored = make_plan(A, torch.float32, flags=RB | pkg.SPMV_PLAN_BANK_ORDER)
    assert plan.info()["row_blocks"] > 0
    check_products(plan, stored, synth.uniform_vector(A.n, 33), synth.uniform_vector(A.m, 34), 1e-5,
                   f"{name} row blocks + bank order")
    plan.close()


def test_row_blocks_integer_data_is_exact(case):
    name, A0 = case
    A = synth.SparseMatrix(A0.layout, A0.m, A0.n, A0.ptr, A0.idx,
                           np.random.default_rng(5).integers(-7, 8, A0.nnz).astype(np.float64))
    plan, stored = make_plan(A, torch.float64, flags=RB)
    assert plan.info()["row_blocks"] > 0
    x = synth.uniform_vector(A.n, 3, int_values=5)
    v = synth.uniform_vector(A.m, 4, int_values=5)
    y = host_of(plan.spmv(dev_vec(x, torch.float64)))
    u = host_of(plan.spvtm(dev_vec(v, torch.float64)))
    plan.check()
    assert np.array_equal(y, oracle.spmv(stored, x)), name
    assert np.array_equal(u, oracle.spvtm(stored, v)), name
    plan.close()


def test_row_blocks_are_bitwise_reproducible(case):
    """No atomics on this path: repeated calls and the vectors of a batch give identical bits."""
    name, A = case
    plan, _ = make_plan(A, torch.float32, flags=RB)
    op = pkg.SPMV_OP_AX if A.layout == "csc" else pkg.SPMV_OP_VTA
    len_in = A.n if A.layout == "csc" else A.m
    X = torch.stack([dev_vec(synth.uniform_vector(len_in, 40 + b), torch.float32) for b in range(3)])
    single = plan.spmv if A.layout == "csc" else plan.spvtm
    first = [single(X[b]).clone() for b in range(3)]
    for _ in range(3):
        for b in range(3):
            assert torch.equal(single(X[b]), first[b]), f"{name}: call-to-call bits differ"
    Y = plan.batch(op, X)
    plan.check()
    for b in range(3):
        assert torch.equal(Y[b], first[b]), f"{name}: batch vector {b} differs from its single product"
    plan.close()


def test_row_blocks_match_the_atomic_path(case):
    """Same products with and without the copy, within the FP32 tolerance of each other."""
    name, A = case
    p1, stored = make_plan(A, torch.float32, flags=RB)
    p0, _ = make_plan(A, torch.float32)
    assert p1.info()["row_blocks"] > 0 and p0.info()["row_blocks"] == 0
    x = dev_vec(synth.uniform_vector(A.n, 51), torch.float32)
    v = dev_vec(synth.uniform_vector(A.m, 52), torch.float32)
    xs, vs = host_of(x), host_of(v)
    assert_close(host_of(p1.spmv(x)), host_of(p0.spmv(x)), oracle.abs_spmv(stored, xs), 2e-5, f"{name} y")
    assert_close(host_of(p1.spvtm(v)), host_of(p0.spvtm(v)), oracle.abs_spvtm(stored, vs), 2e-5, f"{name} u")
    p1.check()
    p0.check()
    p1.close()
    p0.close()


@pytest.mark.parametrize("why", ["small", "no_validate"])
def test_row_blocks_skipped_when_they_cannot_serve(why):
    """Too few nonzeros per block and short-vector entry, or an unvalidated plan: no copy, same results."""
    if why == "small":
        A = synth.random_matrix(37, 2000, "csc", density=0.05, seed=9)
        flags = RB
    else:
        A = _wide(24)
        flags = RB | pkg.SPMV_PLAN_NO_VALIDATE
    plan, stored = make_plan(A, torch.float32, flags=flags)
    assert plan.info()["row_blocks"] == 0
    check_products(plan, stored, synth.uniform_vector(A.n, 1), synth.uniform_vector(A.m, 2), 1e-5, why)
    plan.close()


def test_row_blocks_profile_kernels():
    """The copy's passes are timed as kernels 5 (dot) and 6 (zone fixup), the combine as 1."""
    A = _wide(25)
    plan, _ = make_plan(A, torch.float32, flags=RB | pkg.SPMV_PLAN_PROFILE)
    x = dev_vec(synth.uniform_vector(A.n, 1), torch.float32)
    for _ in range(3):
        plan.spmv(x)
    plan.check()
    assert plan.profile(pkg._lib.KERNEL_ROWBLOCK_DOT)[1] == 3
    assert plan.profile(pkg._lib.KERNEL_COMBINE)[1] == 3
    assert plan.profile(pkg._lib.KERNEL_SCATTER)[1] == 0
    plan.close()
