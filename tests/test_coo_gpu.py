"""Plans from coordinate triples in storage order (the column-major triple stream of the paper)."""
import json
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
import paper_1812_00904_gb300 as pkg  # noqa: E402
from gpu_util import DEV, assert_close, dev_vec, host_of  # noqa: E402


def _triples(A):
    """(rows, cols) of every stored entry, in storage order."""
    ptr = np.asarray(A.ptr, dtype=np.int64)
    major = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr)).astype(np.int32)
    minor = np.asarray(A.idx, dtype=np.int32)
    return (minor, major) if A.layout == "csc" else (major, minor)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float64], ids=str)
def test_coo_plan_matches_oracle_and_the_compressed_plan(layout, dtype):
    m, n = (700, 40_000) if layout == "csc" else (40_000, 700)
    A = synth.random_matrix(m, n, layout, density=0.004, seed=81)
    rows, cols = _triples(A)
    vals = torch.as_tensor(np.asarray(A.vals, dtype=np.float64)).to(dtype)
    stored = synth.SparseMatrix(layout, m, n, A.ptr, A.idx, vals.double().numpy())
    vt = torch.float64 if dtype == torch.float64 else torch.float32
    plan = pkg.Plan.from_coo(m, n, _dev(rows), _dev(cols), vals.to(DEV), layout=layout)
    x = dev_vec(synth.uniform_vector(n, 82), vt)
    v = dev_vec(synth.uniform_vector(m, 83), vt)
    y, u = host_of(plan.spmv(x)), host_of(plan.spvtm(v))
    plan.check()
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    xs, vs = host_of(x), host_of(v)
    assert_close(y, oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), tol, "coo y")
    assert_close(u, oracle.spvtm(stored, vs), oracle.abs_spvtm(stored, vs), tol, "coo u")
    # the same tiles as a plan over the compressed arrays: the segmented product agrees bit for bit
    ref = pkg.Plan(m, n, _dev(np.asarray(A.ptr, np.int32)), _dev(np.asarray(A.idx, np.int32)), vals.to(DEV),
                   layout=layout)
    if layout == "csc":
        assert torch.equal(plan.spvtm(v), ref.spvtm(v))
    else:
        assert torch.equal(plan.spmv(x), ref.spmv(x))


def test_coo_worked_example_and_empty_columns():
    """The 5 x 8 matrix of Figs. 1-2 (21 nonzeros) with two empty columns appended."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))
    rows = g["fig2_rows_per_column_1based"]["value"]
    idx = np.array([r - 1 for col in rows for r in col], dtype=np.int32)
    ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])])
    m, n = int(g["m"]), int(g["n"]) + 2
    ptr = np.concatenate([ptr, [ptr[-1], ptr[-1]]])
    cols = np.repeat(np.arange(n), np.diff(ptr)).astype(np.int32)
    vals = np.arange(1, len(idx) + 1, dtype=np.float64)
    A = synth.SparseMatrix("csc", m, n, ptr.astype(np.int32), idx, vals)
    plan = pkg.Plan.from_coo(m, n, _dev(idx), _dev(cols), _dev(vals), layout="csc", chunks=7)
    x = dev_vec(np.arange(1, n + 1, dtype=np.float64), torch.float64)
    v = dev_vec(np.arange(1, m + 1, dtype=np.float64), torch.float64)
    assert np.array_equal(host_of(plan.spmv(x)), oracle.spmv(A, host_of(x)))  # integer data: exact
    assert np.array_equal(host_of(plan.spvtm(v)), oracle.spvtm(A, host_of(v)))
    assert plan.info()["zones"] == 3  # Table II


def test_coo_rejects_unsorted_or_out_of_range_triples():
    rows = _dev(np.array([0, 1, 2, 0], np.int32))
    vals = _dev(np.ones(4, np.float32))
    with pytest.raises(pkg.SpmvError) as e:
        pkg.Plan.from_coo(3, 4, rows, _dev(np.array([0, 2, 1, 3], np.int32)), vals)
    assert e.value.status == 2
    with pytest.raises(pkg.SpmvError) as e:
        pkg.Plan.from_coo(3, 4, rows, _dev(np.array([0, 1, 2, 4], np.int32)), vals)
    assert e.value.status == 2


UNSORTED = pkg.SPMV_PLAN_COO_UNSORTED


def _bits(t):
    w = {2: torch.int16, 4: torch.int32, 8: torch.int64}[t.element_size()]
    return t.view(w).cpu().numpy()


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float64], ids=str)
def test_unsorted_triples_are_sorted_into_the_compressed_matrix(layout, dtype):
    """Shuffled triples: the plan's copy is exactly the compressed matrix (indices sorted inside
    each segment, values moved with them) and the products match the oracle."""
    m, n = (700, 40_000) if layout == "csc" else (40_000, 700)
    A = synth.random_matrix(m, n, layout, density=0.004, seed=87)
    rows, cols = _triples(A)
    perm = np.random.default_rng(88).permutation(A.nnz)
    vals = torch.as_tensor(np.asarray(A.vals, dtype=np.float64)).to(dtype)
    plan = pkg.Plan.from_coo(m, n, _dev(rows[perm]), _dev(cols[perm]), vals[perm].to(DEV), layout=layout,
                             flags=UNSORTED)
    idx1, val1 = plan.export()
    assert np.array_equal(idx1.cpu().numpy(), np.asarray(A.idx))
    assert np.array_equal(_bits(val1), _bits(vals))
    stored = synth.SparseMatrix(layout, m, n, A.ptr, A.idx, vals.double().numpy())
    vt = torch.float64 if dtype == torch.float64 else torch.float32
    x = dev_vec(synth.uniform_vector(n, 89), vt)
    v = dev_vec(synth.uniform_vector(m, 90), vt)
    y, u = host_of(plan.spmv(x)), host_of(plan.spvtm(v))
    plan.check()
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    xs, vs = host_of(x), host_of(v)
    assert_close(y, oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), tol, "unsorted coo y")
    assert_close(u, oracle.spvtm(stored, vs), oracle.abs_spvtm(stored, vs), tol, "unsorted coo u")


def test_unsorted_triples_with_duplicates_and_bank_order():
    m, n = 300, 20_000
    A = synth.random_matrix(m, n, "csc", density=0.01, seed=91, duplicates=True)
    rows, cols = _triples(A)
    perm = np.random.default_rng(92).permutation(A.nnz)
    vals = torch.as_tensor(np.asarray(A.vals, dtype=np.float64)).float()
    x = dev_vec(synth.uniform_vector(n, 93), torch.float32)
    stored = synth.SparseMatrix("csc", m, n, A.ptr, A.idx, vals.double().numpy())
    xs = host_of(x)
    for flags in (UNSORTED, UNSORTED | pkg.SPMV_PLAN_BANK_ORDER):
        plan = pkg.Plan.from_coo(m, n, _dev(rows[perm]), _dev(cols[perm]), vals[perm].to(DEV), flags=flags)
        assert_close(host_of(plan.spmv(x)), oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), 1e-5, "dup y")
        plan.check()
        idx1, val1 = plan.export()
        seg = np.repeat(np.arange(n), np.diff(np.asarray(A.ptr)))
        o0 = np.lexsort((_bits(vals), np.asarray(A.idx), seg))
        o1 = np.lexsort((_bits(val1), idx1.cpu().numpy(), seg))
        assert np.array_equal(np.asarray(A.idx)[o0], idx1.cpu().numpy()[o1])
        assert np.array_equal(_bits(vals)[o0], _bits(val1)[o1])


def test_unsorted_triples_large_several_passes():
    """2M nonzeros with a 30-bit key span (four 8-bit passes, about 500 sort tiles)."""
    A = synth.wide_fp32_large(1, device="cuda", scale=0.01)
    nnz = A.nnz
    major = torch.repeat_interleave(torch.arange(A.n, device=DEV, dtype=torch.int32), torch.diff(A.ptr).long())
    g = torch.Generator(device=DEV)
    g.manual_seed(94)
    perm = torch.randperm(nnz, generator=g, device=DEV)
    plan = pkg.Plan.from_coo(A.m, A.n, A.idx[perm].contiguous(), major[perm].contiguous(), A.vals[perm].contiguous(),
                             flags=UNSORTED)
    idx1, val1 = plan.export()
    assert torch.equal(idx1, A.idx) and torch.equal(val1, A.vals)
    ref = pkg.Plan(A.m, A.n, A.ptr, A.idx, A.vals)
    v = torch.rand(A.m, device=DEV) * 2 - 1
    assert torch.equal(plan.spvtm(v), ref.spvtm(v))  # same arrays, same tiles: the segmented pass agrees bit for bit
    plan.check()


def test_unsorted_triples_reject_bad_indices_and_accept_empty():
    vals = _dev(np.ones(4, np.float32))
    for rows, cols in (([0, 1, 3, 0], [2, 0, 1, 3]), ([0, 1, 2, 0], [2, 0, 4, 3]), ([0, -1, 2, 0], [2, 0, 1, 3])):
        with pytest.raises(pkg.SpmvError) as e:
            pkg.Plan.from_coo(3, 4, _dev(np.array(rows, np.int32)), _dev(np.array(cols, np.int32)), vals,
                              flags=UNSORTED)
        assert e.value.status == 2
    empty = _dev(np.zeros(0, np.int32))
    plan = pkg.Plan.from_coo(3, 4, empty, empty, _dev(np.zeros(0, np.float32)), flags=UNSORTED)
    assert torch.count_nonzero(plan.spmv(torch.ones(4, device=DEV))) == 0
    plan.check()
