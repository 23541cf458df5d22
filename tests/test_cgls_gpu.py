"""The normal-equation operator u = A^T (A x) and the CGLS least-squares loop on the device."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import pins  # noqa: E402
import synth  # noqa: E402
import paper_1812_00904_gb300 as pkg  # noqa: E402
from gpu_util import DEV, assert_close, dev_vec, host_of, make_plan  # noqa: E402


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5), (torch.bfloat16, 1e-5)], ids=str)
def test_normal_operator_matches_oracle(layout, dtype, tol):
    m, n = (800, 30_000) if layout == "csc" else (30_000, 800)
    A = synth.random_matrix(m, n, layout, density=0.01, seed=61)
    plan, stored = make_plan(A, dtype)
    x = dev_vec(synth.uniform_vector(n, 62), plan.vec_dtype)
    y = torch.empty(m, dtype=plan.vec_dtype, device=DEV)
    u = torch.empty(n, dtype=plan.vec_dtype, device=DEV)
    pkg.spmv_normal(plan.handle, x, u, y)
    u2 = plan.normal(x)  # the plan's own buffer for A x
    plan.check()
    xs = host_of(x)
    y_ref = oracle.spmv(stored, xs)
    assert_close(host_of(y), y_ref, oracle.abs_spmv(stored, xs), tol, "A x")
    # A^T (A x) with the scale |A|^T |A| |x| (the first product's error propagates)
    u_ref = oracle.spvtm(stored, y_ref)
    scale = oracle.abs_spvtm(stored, oracle.abs_spmv(stored, xs))
    assert_close(host_of(u), u_ref, scale, 2 * tol, "A^T A x")
    assert_close(host_of(u2), u_ref, scale, 2 * tol, "A^T A x (plan buffer)")


@pytest.mark.parametrize("layout", ["csc", "csr"])
def test_cgls_fp64_follows_the_oracle_iterates(layout):
    m, n = (300, 6_000) if layout == "csc" else (6_000, 300)
    A = synth.random_matrix(m, n, layout, density=0.02, seed=63)
    plan, stored = make_plan(A, torch.float64)
    b = dev_vec(synth.uniform_vector(m, 64), torch.float64)
    for iters in (1, 5, 12):
        x, it, rel = plan.cgls(b, max_iters=iters, tol=0.0)
        plan.check()
        assert it == iters
        x_ref, rel_ref = oracle.cgls(stored, host_of(b), np.zeros(n), iters)
        err = np.abs(host_of(x) - x_ref).max() / np.abs(x_ref).max()
        assert err < 1e-9, (iters, err)
        assert abs(rel - rel_ref) <= 1e-9 * max(rel_ref, 1e-30) + 1e-12


@pytest.mark.parametrize("layout,dtype", [("csr", torch.float32), ("csc", torch.float32), ("csr", torch.bfloat16)],
                         ids=str)
def test_cgls_converges_to_the_least_squares_solution(layout, dtype):
    """Tall full-rank: the unique solution; wide from zero: the minimum-norm solution."""
    m, n = (3_000, 200) if layout == "csr" else (200, 3_000)
    A = synth.random_matrix(m, n, layout, density=0.05, seed=65)
    plan, stored = make_plan(A, dtype)
    b = dev_vec(synth.uniform_vector(m, 66), torch.float32)
    x, it, rel = plan.cgls(b, max_iters=500, tol=1e-5)
    plan.check()
    assert rel <= 1e-5 and it <= 500
    D = pins.dense_of(stored)
    x_ref = np.linalg.lstsq(D, host_of(b), rcond=None)[0]
    err = np.linalg.norm(host_of(x) - x_ref) / np.linalg.norm(x_ref)
    assert err < 1e-3, err


def test_cgls_arguments():
    A = synth.random_matrix(50, 400, "csc", density=0.05, seed=1)
    plan, _ = make_plan(A, torch.float32)
    b = dev_vec(synth.uniform_vector(50, 2), torch.float32)
    x = torch.zeros(400, device=DEV)
    with pytest.raises(pkg.SpmvError):
        pkg.spmv_cgls(plan.handle, b, x, -1, 1e-6)
    with pytest.raises(pkg.SpmvError):
        pkg.spmv_cgls(plan.handle, b.data_ptr() + 4, x, 10, 1e-6)
    it, rel = pkg.spmv_cgls(plan.handle, b, x, 0, 1e-6)  # no iteration: x stays the start
    assert it == 0 and torch.count_nonzero(x) == 0
