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
