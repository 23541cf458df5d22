"""spmv_pair: y = A x and u = v^T A for independent x and v in one call, with device vectors
(the two products side by side on the caller's stream and a stream of the plan, joined back
into the caller's) and with host vectors (staged, the transfers of each product overlapping
the other's kernels).  Results must match the FP64 oracle and the separate calls (bit for bit
in the segmented direction, whose sums are formed in a fixed order)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402

import paper_1812_00904_gb300 as pkg  # noqa: E402
from paper_1812_00904_gb300 import _lib  # noqa: E402
from gpu_util import DEV, assert_close, dev_vec, host_of, make_plan  # noqa: E402


def _case(layout):
    m, n = (2000, 60_000) if layout == "csc" else (60_000, 2000)
    A = synth.random_matrix(m, n, layout, density=0.004, seed=71)
    plan, stored = make_plan(A, torch.float32)
    x = synth.uniform_vector(n, 72).astype(np.float32)
    v = synth.uniform_vector(m, 73).astype(np.float32)
    return A, plan, stored, x, v


def _check(stored, x, v, y, u, what):
    xs, vs = x.astype(np.float64), v.astype(np.float64)
    assert_close(np.asarray(y, np.float64), oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), 1e-5, f"{what} y")
    assert_close(np.asarray(u, np.float64), oracle.spvtm(stored, vs), oracle.abs_spvtm(stored, vs), 1e-5, f"{what} u")


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("where", ["device", "pinned", "pageable", "mixed"])
def test_pair_matches_the_oracle_and_the_separate_calls(layout, where):
    A, plan, stored, x, v = _case(layout)
    xd, vd = dev_vec(x, torch.float32), dev_vec(v, torch.float32)
    ref_y, ref_u = plan.spmv(xd), plan.spvtm(vd)
    torch.cuda.synchronize()
    if where == "device":
        xa, va = xd, vd
        ya, ua = torch.empty(A.m, device=DEV), torch.empty(A.n, device=DEV)
    else:
        pin = where == "pinned"
        mk = (lambda a: torch.from_numpy(a).pin_memory()) if pin else (lambda a: torch.from_numpy(a.copy()))
        xa, va = mk(x), mk(v)
        ya = torch.full((A.m,), np.nan).float()
        ua = torch.full((A.n,), np.nan).float()
        if pin:
            ya, ua = ya.pin_memory(), ua.pin_memory()
        if where == "mixed":  # x and u on the host, v and y on the device
            va, ya = vd, torch.empty(A.m, device=DEV)
    pkg.spmv_pair(plan.handle, xa, ya, va, ua)
    if where == "device":
        torch.cuda.synchronize()
    # host results have landed when the call returns
    y, u = host_of(ya), host_of(ua)
    _check(stored, x, v, y, u, where)
    seg = u if layout == "csc" else y
    seg_ref = host_of(ref_u if layout == "csc" else ref_y)
    assert np.array_equal(seg, seg_ref), "segmented direction differs from the separate call"
    plan.check()
    plan.close()


@pytest.mark.parametrize("layout", ["csc", "csr"])
def test_device_pair_is_ordered_on_the_callers_stream(layout):
    """Work queued on the caller's stream before the call (here: the inputs' producer) runs
    before both products, and work queued after it (the results' consumer) sees both results,
    call after call with no host synchronisation in between."""
    A, plan, stored, x, v = _case(layout)
    s = torch.cuda.Stream()
    x0, v0 = dev_vec(x, torch.float32), dev_vec(v, torch.float32)
    torch.cuda.synchronize()
    outs = []
    with torch.cuda.stream(s):
        for rep in range(6):
            xa = x0 * float(rep + 1)
            va = v0 * float(rep - 2.5)
            ya, ua = torch.empty(A.m, device=DEV), torch.empty(A.n, device=DEV)
            pkg.spmv_pair(plan.handle, xa, ya, va, ua, s)
            outs.append((xa, va, ya.clone(), ua.clone(), ya, ua))
            ya.fill_(float("nan"))  # overwritten on the stream once the consumer has copied them
            ua.fill_(float("nan"))
    s.synchronize()
    for rep, (xa, va, y, u, _, _) in enumerate(outs):
        _check(stored, host_of(xa).astype(np.float32), host_of(va).astype(np.float32), host_of(y), host_of(u),
               f"{layout} call {rep}")
    plan.check()
    plan.close()


def test_pair_repeated_calls_and_errors():
    A, plan, stored, x, v = _case("csc")
    xa, va = torch.from_numpy(x).pin_memory(), torch.from_numpy(v).pin_memory()
    ya, ua = torch.empty(A.m).pin_memory(), torch.empty(A.n).pin_memory()
    for rep in range(5):  # the staging buffers, copy stream and events are reused
        xa.mul_(-1.0)
        pkg.spmv_pair(plan.handle, xa, ya, va, ua)
        _check(stored, xa.numpy(), v, ya.numpy(), ua.numpy(), f"repeat {rep}")
    lib = _lib.load()
    assert lib.spmv_pair(plan.handle, None, ya.data_ptr(), va.data_ptr(), ua.data_ptr(), None) == _lib.SPMV_ERR_INVALID_ARG
    yd = torch.empty(A.m + 4, device=DEV)
    assert lib.spmv_pair(plan.handle, xa.data_ptr(), yd.data_ptr() + 4, va.data_ptr(), ua.data_ptr(),
                         None) == _lib.SPMV_ERR_INVALID_ARG  # misaligned device vector
    assert "aligned" in lib.spmv_last_error().decode()
    plan.check()
    plan.close()


@pytest.mark.parametrize("where", ["host", "device"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.bfloat16], ids=str)
@pytest.mark.parametrize("flags", [0, pkg.SPMV_PLAN_ROW_BLOCKS, pkg.SPMV_PLAN_BANK_ORDER, pkg.SPMV_PLAN_PROFILE],
                         ids=["stored", "row_blocks", "bank_order", "profiled"])
def test_pair_value_types_and_plan_copies(dtype, flags, where):
    """Pairs (host-staged, and device vectors with the two products side by side) on FP64 and
    BF16-value plans, on plans that multiply their own copies of the nonzeros (row-sorted
    blocks, bank order) and with every launch timed, against the FP64 oracle."""
    from gpu_util import TOL, vec_dtype_for

    A = synth.random_matrix(1500, 80_000, "csc", density=0.003, seed=81)
    plan, stored = make_plan(A, dtype, flags=flags)
    vt = vec_dtype_for(dtype)
    x = synth.uniform_vector(A.n, 82)
    v = synth.uniform_vector(A.m, 83)
    if where == "host":
        xa = torch.from_numpy(x).to(vt).pin_memory()
        va = torch.from_numpy(v).to(vt).pin_memory()
        ya = torch.empty(A.m, dtype=vt).pin_memory()
        ua = torch.empty(A.n, dtype=vt).pin_memory()
    else:
        xa, va = dev_vec(x, vt), dev_vec(v, vt)
        ya, ua = torch.empty(A.m, dtype=vt, device=DEV), torch.empty(A.n, dtype=vt, device=DEV)
    pkg.spmv_pair(plan.handle, xa, ya, va, ua)
    torch.cuda.synchronize()
    xs, vs = host_of(xa), host_of(va)
    assert_close(host_of(ya), oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), TOL[dtype], "pair y")
    assert_close(host_of(ua), oracle.spvtm(stored, vs), oracle.abs_spvtm(stored, vs), TOL[dtype], "pair u")
    if flags == pkg.SPMV_PLAN_PROFILE:  # both products' launches were timed, on either stream
        assert pkg.spmv_profile_read(plan.handle, 0)[1] == 1 and pkg.spmv_profile_read(plan.handle, 2)[1] == 1
    plan.check()
    plan.close()


@pytest.mark.parametrize("layout", ["csc", "csr"])
def test_device_pair_with_the_short_vector_off_chip(layout):
    """A short dimension too long for shared memory: the accumulating pass adds into a global
    FP64 accumulator and the segmented pass reads the short vector through L2, side by side."""
    m, n = (60_000, 40_000) if layout == "csc" else (40_000, 60_000)
    A = synth.random_matrix(m, n, layout, density=0.0005, seed=91)
    plan, stored = make_plan(A, torch.float32)
    assert plan.info()["short_on_chip"] == 0
    x, v = synth.uniform_vector(n, 92), synth.uniform_vector(m, 93)
    xd, vd = dev_vec(x, torch.float32), dev_vec(v, torch.float32)
    y, u = torch.empty(m, device=DEV), torch.empty(n, device=DEV)
    for _ in range(3):
        pkg.spmv_pair(plan.handle, xd, y, vd, u)
    torch.cuda.synchronize()
    _check(stored, host_of(xd), host_of(vd), host_of(y), host_of(u), f"{layout} off chip")
    plan.check()
    plan.close()
