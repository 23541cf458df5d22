"""Multi-vector products, dvalues and the autograd Function (BF16/FP16 value storage) against the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402

import paper_1812_00904_gb300 as pkg  # noqa: E402
from gpu_util import DEV, TOL, assert_close, dev_vec, host_of, make_plan  # noqa: E402


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16], ids=str)
@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 13])
def test_batch_equals_oracle_per_vector(layout, dtype, k):
    m, n = (600, 20_000) if layout == "csc" else (20_000, 600)
    A = synth.random_matrix(m, n, layout, density=0.01, seed=k)
    plan, stored = make_plan(A, dtype)
    vt = plan.vec_dtype
    X = torch.stack([dev_vec(synth.uniform_vector(n, 10 + b), vt) for b in range(k)])
    V = torch.stack([dev_vec(synth.uniform_vector(m, 50 + b), vt) for b in range(k)])
    Y = plan.batch(pkg.SPMV_OP_AX, X)
    U = plan.batch(pkg.SPMV_OP_VTA, V)
    plan.check()
    for b in range(k):
        xs, vs = host_of(X[b]), host_of(V[b])
        assert_close(host_of(Y[b]), oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), TOL[dtype], f"Y[{b}]")
        assert_close(host_of(U[b]), oracle.spvtm(stored, vs), oracle.abs_spvtm(stored, vs), TOL[dtype], f"U[{b}]")
    # the dot-product (segmented) direction adds in the same order for every batch width: bitwise equal
    seg_op = pkg.SPMV_OP_VTA if layout == "csc" else pkg.SPMV_OP_AX
    Z = V if seg_op == pkg.SPMV_OP_VTA else X
    R = U if seg_op == pkg.SPMV_OP_VTA else Y
    single = plan.spvtm(Z[k - 1]) if seg_op == pkg.SPMV_OP_VTA else plan.spmv(Z[k - 1])
    assert torch.equal(single, R[k - 1])


@pytest.mark.parametrize("layout", ["csc", "csr"])
def test_batch_on_a_wide_round_plan(layout):
    """A plan with many small tiles whose single- and multi-vector passes run different numbers
    of warps over the same tiles: the sums must agree bit for bit."""
    m, n = (900, 40_000) if layout == "csc" else (40_000, 900)
    A = synth.random_matrix(m, n, layout, density=0.004, seed=77)
    plan, stored = make_plan(A, torch.float32, tile_items=256, stages=2, warps_per_cta=24)
    assert plan.info()["warps_per_cta"] == 24
    k = 5
    X = torch.stack([dev_vec(synth.uniform_vector(n, 100 + b), torch.float32) for b in range(k)])
    V = torch.stack([dev_vec(synth.uniform_vector(m, 200 + b), torch.float32) for b in range(k)])
    Y = plan.batch(pkg.SPMV_OP_AX, X)
    U = plan.batch(pkg.SPMV_OP_VTA, V)
    plan.check()
    for b in range(k):
        xs, vs = host_of(X[b]), host_of(V[b])
        assert_close(host_of(Y[b]), oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), 1e-5, f"Y[{b}]")
        assert_close(host_of(U[b]), oracle.spvtm(stored, vs), oracle.abs_spvtm(stored, vs), 1e-5, f"U[{b}]")
    if layout == "csc":
        assert torch.equal(plan.spvtm(V[2]), U[2])
    else:
        assert torch.equal(plan.spmv(X[2]), Y[2])


def test_batch_leading_dimension_and_off_chip():
    A = synth.random_matrix(3000, 50_000, "csc", density=0.002, seed=3)
    for flags in (0, pkg.SPMV_PLAN_SHORT_IN_GLOBAL):
        plan, stored = make_plan(A, torch.float32, flags=flags)
        k, ld = 3, 50_004
        X = torch.zeros((k, ld), dtype=torch.float32, device=DEV)
        for b in range(k):
            X[b, :A.n] = dev_vec(synth.uniform_vector(A.n, b), torch.float32)
        Y = torch.full((k, 3008), 7.0, device=DEV)
        pkg.spmv_batch(plan.handle, pkg.SPMV_OP_AX, k, X, ld, Y, 3008)
        for b in range(k):
            xs = host_of(X[b, :A.n])
            assert_close(host_of(Y[b, :A.m]), oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), 1e-5, "ld")
            assert (host_of(Y[b, A.m:]) == 7.0).all()  # padding untouched


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16, torch.float16], ids=str)
def test_dvalues_matches_oracle(layout, dtype):
    m, n = (500, 30_000) if layout == "csc" else (30_000, 500)
    A = synth.random_matrix(m, n, layout, density=0.01, seed=31)
    plan, stored = make_plan(A, dtype)
    r = dev_vec(synth.uniform_vector(m, 1), plan.vec_dtype)
    x = dev_vec(synth.uniform_vector(n, 2), plan.vec_dtype)
    g = host_of(plan.dvalues(r, x))
    ref = oracle.dvalues(stored, host_of(r), host_of(x))
    # one product in the accumulation type, rounded to the value type: half an ulp relative to the
    # result, plus half the subnormal spacing for FP16 (2^-24), whose normal range starts at 2^-14
    rel = {torch.float64: 1e-15, torch.float32: 1e-6, torch.bfloat16: 2 ** -8, torch.float16: 2 ** -10}[dtype]
    tiny = 2.0 ** -25 if dtype == torch.float16 else 1e-30
    assert np.all(np.abs(g - ref) <= rel * np.abs(ref) + tiny)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16, torch.float32], ids=str)
def test_autograd_least_squares_wide_fp64_workload(dtype):
    """Loss 0.5||Ax-b||^2 on the m=1,000 x n=100,000 workload with values stored in BF16/FP16."""
    A = synth.wide_fp64_small(0)
    plan, stored = make_plan(A, dtype)
    vals = plan.vals.clone().requires_grad_(True)
    plan.vals.copy_(vals.detach())
    plan2 = pkg.Plan(A.m, A.n, plan.ptr, plan.idx, vals, layout="csc")
    x64 = synth.uniform_vector(A.n, 3)
    b64 = synth.uniform_vector(A.m, 4)
    x = dev_vec(x64, torch.float32).requires_grad_(True)
    b = dev_vec(b64, torch.float32)
    y = pkg.sparse_matvec(vals, x, plan2)
    loss = 0.5 * ((y - b) ** 2).sum()
    loss.backward()
    # oracle gradients on the stored (rounded) values and the FP32-rounded x, b
    xs, bs = host_of(x.detach()), host_of(b)
    lo, gx_ref, gv_ref, r = oracle.least_squares(stored, xs, bs)
    gx = host_of(x.grad)
    gv = host_of(vals.grad)
    r_gpu = host_of(y.detach()) - bs  # the residual the backward pass received (FP32 forward)
    # (a) the backward kernels on that residual: dx = A^T r (SpVTM), dvalues = r_i x_j rounded to the value type
    assert_close(gx, oracle.spvtm(stored, r_gpu), oracle.abs_spvtm(stored, r_gpu), 1e-5, "dx (kernel)")
    rel = {torch.bfloat16: 2 ** -8, torch.float16: 2 ** -10, torch.float32: 1e-6}[dtype]
    tiny = 2.0 ** -25 if dtype == torch.float16 else 1e-30
    gv_k = oracle.dvalues(stored, r_gpu, xs)
    assert np.all(np.abs(gv - gv_k) <= rel * np.abs(gv_k) + tiny)
    # (b) end to end against the FP64 gradient: the residual's error (forward tolerance 1e-5 |A||x| plus
    # FP32 rounding of y - b) propagates through A^T, and the backward kernel adds 1e-5 |A|^T |r|
    r_err = 1e-5 * oracle.abs_spmv(stored, xs) + 2 ** -23 * (np.abs(r) + np.abs(bs))
    gx_bound = oracle.abs_spvtm(stored, r_err) + 1e-5 * oracle.abs_spvtm(stored, np.abs(r) + r_err)
    assert_close(gx, gx_ref, gx_bound, 1.0, "dx")
    gv_prop = oracle.dvalues(stored, r_err, np.abs(xs))
    assert np.all(np.abs(gv - gv_ref) <= gv_prop + rel * (np.abs(gv_ref) + gv_prop) + tiny)
    assert abs(float(loss.detach()) - lo) <= 1e-4 * abs(lo)
    # against the unrounded FP64 matrix: normwise 1e-2 for the reduced-precision values
    y_full = oracle.spmv(A, x64)
    ynorm = np.linalg.norm(host_of(y.detach()) - y_full) / np.linalg.norm(y_full)
    assert ynorm <= 1e-2
    # directional finite difference of the GPU loss (FP32): loose check
    d = dev_vec(synth.uniform_vector(A.n, 9), torch.float32)
    h = 1e-2
    with torch.no_grad():
        lp = 0.5 * ((plan2.spmv(x.detach() + h * d) - b) ** 2).sum()
        lm = 0.5 * ((plan2.spmv(x.detach() - h * d) - b) ** 2).sum()
    fd = float(lp - lm) / (2 * h)
    an = float((x.grad * d).sum())
    assert abs(fd - an) <= 1e-2 * max(1.0, abs(an))


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("tile_items", [0, 40, 104, 256])
@pytest.mark.parametrize("k", [2, 3, 8])
def test_batch_small_tiles_match_single_vector_calls(layout, tile_items, k):
    """Multi-vector passes over small tiles (partial steps, many zones) equal the single-vector calls."""
    m, n = (900, 25_000) if layout == "csc" else (25_000, 900)
    A = synth.random_matrix(m, n, layout, density=0.01, seed=2)
    plan, stored = make_plan(A, torch.float32, tile_items=tile_items)
    X = torch.stack([dev_vec(synth.uniform_vector(n, 300 + b), torch.float32) for b in range(k)])
    V = torch.stack([dev_vec(synth.uniform_vector(m, 400 + b), torch.float32) for b in range(k)])
    Y = plan.batch(pkg.SPMV_OP_AX, X)
    U = plan.batch(pkg.SPMV_OP_VTA, V)
    plan.check()
    for b in range(k):
        xs, vs = host_of(X[b]), host_of(V[b])
        assert_close(host_of(Y[b]), oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), 1e-5, f"Y[{b}]")
        assert_close(host_of(U[b]), oracle.spvtm(stored, vs), oracle.abs_spvtm(stored, vs), 1e-5, f"U[{b}]")
    seg_single = plan.spvtm(V[k - 1]) if layout == "csc" else plan.spmv(X[k - 1])
    assert torch.equal(seg_single, U[k - 1] if layout == "csc" else Y[k - 1])
