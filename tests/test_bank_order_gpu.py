"""Plans that keep their own copy of the nonzeros in bank order (SPMV_PLAN_BANK_ORDER).

The copy holds the same nonzeros, permuted within every column (row for CSR), so the
products equal the oracle's within the usual tolerances; the permutation itself is
checked exactly (per segment, the same (index, value) pairs), and its purpose -- fewer
shared-memory bank conflicts in the three access patterns of the streaming kernels -- is
measured on the exported order.
"""
import json
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
import paper_1812_00904_gb300 as pkg  # noqa: E402
from gpu_util import DEV, TOL, check_products, dev_vec, device_matrix, host_of, vec_dtype_for  # noqa: E402

BANK = pkg.SPMV_PLAN_BANK_ORDER


def _plan(A, dtype, flags=BANK, **kw):
    t, stored = device_matrix(A, dtype)
    plan = pkg.Plan(A.m, A.n, t["ptr"], t["idx"], t["vals"], layout=A.layout, vec_dtype=vec_dtype_for(dtype),
                    flags=flags, **kw)
    return plan, stored, t


def _same_pairs_per_segment(ptr, idx0, val0, idx1, val1):
    """Both orders hold, segment by segment, the same (index, value bits) pairs."""
    ptr = np.asarray(ptr, dtype=np.int64)
    seg = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
    o0 = np.lexsort((val0, idx0, seg))
    o1 = np.lexsort((val1, idx1, seg))
    assert np.array_equal(idx0[o0], idx1[o1])
    assert np.array_equal(val0[o0], val1[o1])


def _bits(t):
    """Value bits as integers (exact comparison for any value dtype)."""
    w = {2: torch.int16, 4: torch.int32, 8: torch.int64}[t.element_size()]
    return t.view(w).cpu().numpy()


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16], ids=str)
@pytest.mark.parametrize("tile_items", [0, 512, 256, 200, 64])
def test_bank_ordered_plan_matches_oracle(layout, dtype, tile_items):
    m, n = (900, 50_000) if layout == "csc" else (50_000, 900)
    A = synth.random_matrix(m, n, layout, density=0.006, seed=91)
    plan, stored, t = _plan(A, dtype, tile_items=tile_items)
    check_products(plan, stored, synth.uniform_vector(n, 92), synth.uniform_vector(m, 93), TOL[dtype],
                   f"bank order {layout} T={tile_items}")
    idx1, val1 = plan.export()
    _same_pairs_per_segment(A.ptr, t["idx"].cpu().numpy(), _bits(t["vals"]), idx1.cpu().numpy(), _bits(val1))
    # the batched pass reads the same copy
    X = torch.stack([dev_vec(synth.uniform_vector(n, 94 + b), plan.vec_dtype) for b in range(3)])
    Y = plan.batch(pkg.SPMV_OP_AX, X)
    plan.check()
    for b in range(3):
        xs = host_of(X[b])
        ref, scale = oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs)
        assert np.all(np.abs(host_of(Y[b]) - ref) <= TOL[dtype] * scale + 1e-300)


def _mean_max_multiplicity(rows, banks=32):
    """Mean, over warp instructions, of the most lanes (lane groups) sharing one bank (group
    of banks), for the scatter pass (32 consecutive positions), the segmented pass (lane l at
    8l + (e ^ 4((l >> 2) & 1))) and the multi-vector segmented pass with 8 vectors (4 lane
    groups at 32a + 8c + e, c = 0..3, each on the 8 banks of its index mod 4) over the whole
    256-position steps of a plan with T = 512."""
    nb = len(rows) // 256
    R = (np.asarray(rows[:nb * 256], dtype=np.int64) % banks).reshape(nb, 256)
    lane = np.arange(32)
    seg_pos = np.stack([8 * lane + (e ^ (4 * ((lane >> 2) & 1))) for e in range(8)])  # (8, 32)
    vseg_pos = np.stack([32 * a + 8 * np.arange(4) + e for a in range(8) for e in range(8)])  # (64, 4)
    out = []
    for groups, nbk in ((R.reshape(nb * 8, 32), banks), (R[:, seg_pos].reshape(nb * 8, 32), banks),
                        ((R[:, vseg_pos] % 4).reshape(nb * 64, 4), 4)):
        counts = (groups[:, :, None] == np.arange(nbk)[None, None, :]).sum(axis=1)
        out.append(counts.max(axis=1).mean())
    return out


@pytest.mark.parametrize("which", ["wide", "tall"])
def test_bank_order_spreads_the_banks(which):
    """On the power-law workloads (scaled down), all three access patterns meet fewer
    conflicting lanes per instruction in bank order than in the stored order."""
    if which == "wide":
        A = synth.wide_fp32_large(1, device="cuda", scale=0.004)
    else:
        A = synth.tall_fp32_large(2, device="cuda", scale=0.004)
    plan = pkg.Plan(A.m, A.n, A.ptr, A.idx, A.vals, layout=A.layout, flags=BANK, tile_items=512)
    idx1, val1 = plan.export()
    before = _mean_max_multiplicity(A.idx.cpu().numpy())
    after = _mean_max_multiplicity(idx1.cpu().numpy())
    # long columns leave the most freedom: the wide matrix (mean degree 40, a power-law
    # tail) gains much more than the tall one (mean degree 15)
    lim = (0.75, 0.6, 0.75) if which == "wide" else (0.95, 0.9, 0.95)
    for pattern in range(3):
        assert after[pattern] <= lim[pattern] * before[pattern], (pattern, before, after)
    _same_pairs_per_segment(A.ptr.cpu().numpy(), A.idx.cpu().numpy(), _bits(A.vals), idx1.cpu().numpy(),
                            _bits(val1))
    # the products of the bank-ordered plan and of the stored order agree within rounding
    ref = pkg.Plan(A.m, A.n, A.ptr, A.idx, A.vals, layout=A.layout, tile_items=512)
    x = torch.rand(A.n, device=DEV) * 2 - 1
    v = torch.rand(A.m, device=DEV) * 2 - 1
    for got, want in ((plan.spmv(x), ref.spmv(x)), (plan.spvtm(v), ref.spvtm(v))):
        assert torch.allclose(got, want, rtol=1e-5, atol=1e-4)
    plan.check()


def test_bank_order_worked_example_and_degenerate_matrices():
    """The 5 x 8 matrix of Figs. 1-2 with integer values (exact), an empty matrix, and one
    nonzero per column."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))
    rows = g["fig2_rows_per_column_1based"]["value"]
    idx = np.array([r - 1 for col in rows for r in col], dtype=np.int32)
    ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    m, n = int(g["m"]), int(g["n"])
    A = synth.SparseMatrix("csc", m, n, ptr, idx, np.arange(1, len(idx) + 1, dtype=np.float64))
    plan, stored, _ = _plan(A, torch.float64, chunks=7)
    x = dev_vec(np.arange(1, n + 1), torch.float64)
    v = dev_vec(np.arange(1, m + 1), torch.float64)
    assert np.array_equal(host_of(plan.spmv(x)), oracle.spmv(stored, host_of(x)))
    assert np.array_equal(host_of(plan.spvtm(v)), oracle.spvtm(stored, host_of(v)))
    assert plan.info()["zones"] == 3  # Table II

    E = synth.SparseMatrix("csc", 4, 10, np.zeros(11, np.int32), np.zeros(0, np.int32), np.zeros(0))
    pe, _, _ = _plan(E, torch.float32)
    assert torch.count_nonzero(pe.spmv(torch.ones(10, device=DEV))) == 0
    assert pe.info()["workspace_bytes"] > 0

    n1 = 3000
    D = synth.SparseMatrix("csc", 40, n1, np.arange(n1 + 1, dtype=np.int32), (np.arange(n1) * 7 % 40).astype(np.int32),
                           np.linspace(-1, 1, n1))
    pd, sd, _ = _plan(D, torch.float32)
    check_products(pd, sd, synth.uniform_vector(n1, 3), synth.uniform_vector(40, 4), 1e-5, "one per column")


def test_bank_order_owns_its_copy_and_rejects_dvalues():
    A = synth.random_matrix(300, 20_000, "csc", density=0.01, seed=95)
    plan, stored, t = _plan(A, torch.float32)
    base = pkg.Plan(A.m, A.n, t["ptr"], t["idx"], t["vals"], layout="csc").info()["workspace_bytes"]
    info = plan.info()
    assert info["workspace_bytes"] >= base + A.nnz * 8
    x = synth.uniform_vector(A.n, 96)
    v = synth.uniform_vector(A.m, 97)
    y0, u0 = check_products(plan, stored, x, v, 1e-5, "before")
    t["idx"].fill_(0)  # the caller's arrays are no longer read
    t["vals"].fill_(float("nan"))
    y1, u1 = check_products(plan, stored, x, v, 1e-5, "after the caller's arrays changed")
    assert np.array_equal(u0, u1)  # the segmented pass sums in a fixed order
    with pytest.raises(pkg.SpmvError) as e:
        plan.dvalues(dev_vec(v, torch.float32), dev_vec(x, torch.float32))
    assert e.value.status == 8
    idx_h = np.empty(A.nnz, np.int32)  # export into host buffers
    val_h = np.empty(A.nnz, np.float32)
    pkg.spmv_plan_export(plan.handle, idx_h, val_h)
    assert np.array_equal(idx_h, plan.export()[0].cpu().numpy())
    with pytest.raises(pkg.SpmvError) as e:
        pkg.spmv_plan_export(plan.handle, None, val_h)
    assert e.value.status == 1


@pytest.mark.parametrize("layout", ["csc", "csr"])
def test_unvalidated_bank_order_reports_out_of_range_indices(layout):
    """Out-of-range indices survive the permutation unchanged; the checked kernels clamp
    and report them, and nothing outside the plan's arrays is touched."""
    m, n = (300, 20_000) if layout == "csc" else (20_000, 300)
    A = synth.random_matrix(m, n, layout, density=0.01, seed=5)
    t, stored = device_matrix(A, torch.float32)
    n_minor = m if layout == "csc" else n
    for pos, val in ((3, n_minor + 7), (A.nnz // 2, 1 << 30), (A.nnz - 1, -1)):
        t["idx"][pos] = val
    plan = pkg.Plan(m, n, t["ptr"], t["idx"], t["vals"], layout=layout, vec_dtype=torch.float32,
                    flags=BANK | pkg.SPMV_PLAN_NO_VALIDATE)
    idx1, _ = plan.export()
    assert sorted(idx1.cpu().numpy().tolist()) == sorted(t["idx"].cpu().numpy().tolist())
    plan.spmv(dev_vec(synth.uniform_vector(n, 1), torch.float32))
    plan.spvtm(dev_vec(synth.uniform_vector(m, 2), torch.float32))
    with pytest.raises(pkg.SpmvError) as e:
        plan.check()
    assert e.value.status == 5
