"""CUDA path (through the C ABI) against the FP64 oracle: SpMV and SpVTM, plan set-up, edge cases."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle import plan as plan_oracle  # noqa: E402

import paper_1812_00904_gb300 as pkg  # noqa: E402
from gpu_util import (DEV, TOL, assert_close, check_products, dev_vec, device_matrix, host_of,  # noqa: E402
                      make_plan)

DTYPES = [torch.float64, torch.float32, torch.bfloat16, torch.float16]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("dtype", DTYPES, ids=str)
@pytest.mark.parametrize("shape", [(37, 2000), (500, 40_000), (1, 777), (2000, 3)])
def test_random_matches_oracle(layout, dtype, shape):
    m, n = shape if layout == "csc" else shape[::-1]
    A = synth.random_matrix(m, n, layout, density=min(0.05, 40.0 / max(1, min(m, n)) + 0.01), seed=m + n)
    plan, stored = make_plan(A, dtype)
    check_products(plan, stored, synth.uniform_vector(n, 1), synth.uniform_vector(m, 2), TOL[dtype],
                   f"{layout} {dtype} {shape}")
    info = plan.info()
    assert info["zones"] <= max(info["chunks"] - 1, 0)


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=str)
def test_integer_data_is_exact(layout, dtype):
    """Integer values and vectors: every partial sum is exact, so any order gives the oracle's bits."""
    m, n = (300, 20_000) if layout == "csc" else (20_000, 300)
    A = synth.random_matrix(m, n, layout, density=0.02, seed=5, int_values=7)
    plan, stored = make_plan(A, dtype)
    x = synth.uniform_vector(n, 3, int_values=5)
    v = synth.uniform_vector(m, 4, int_values=5)
    y = host_of(plan.spmv(dev_vec(x, plan.vec_dtype)))
    u = host_of(plan.spvtm(dev_vec(v, plan.vec_dtype)))
    plan.check()
    assert np.array_equal(y, oracle.spmv(stored, x))
    assert np.array_equal(u, oracle.spvtm(stored, v))


def _worked_example_matrix():
    g = json.load(open(GOLDEN))
    rows = g["fig2_rows_per_column_1based"]["value"]
    ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    idx = np.array([r - 1 for col in rows for r in col], dtype=np.int32)
    vals = np.arange(1, len(idx) + 1, dtype=np.float64)
    return synth.SparseMatrix("csc", g["m"], g["n"], ptr, idx, vals), g


def test_worked_example_setup_on_device():
    """Sec. II / IV-B on the GPU with P = 7 reproduces Tables II and III."""
    A, g = _worked_example_matrix()
    plan, stored = make_plan(A, torch.float64, chunks=g["P"])
    ch = plan.chunks()
    for name in ("needLeft", "needRight", "leftGroupEnd", "rightGroup", "leftGroup", "procsOnLeft", "procsOnRight"):
        assert [c[name] for c in ch] == g["table3"][name], name
    assert [c["nz_end"] - c["nz_begin"] for c in ch] == g["nonzeros_per_processor"]["value"]
    assert plan.info()["zones"] == len(g["zones"]["value"])
    assert plan.info()["max_zone_size"] == 3
    x = np.arange(1.0, 9.0)
    v = np.arange(1.0, 6.0) - 2.5
    y = host_of(plan.spmv(dev_vec(x, torch.float64)))
    u = host_of(plan.spvtm(dev_vec(v, torch.float64)))
    assert np.array_equal(y, oracle.spmv(stored, x))
    assert np.array_equal(u, oracle.spvtm(stored, v))


def _ptr_cases(rng):
    cases = {}
    cases["powerlaw"] = np.minimum(rng.zipf(1.8, 3000), 800)
    d = rng.integers(0, 3, 3000) * rng.integers(0, 2, 3000)
    cases["empties"] = d
    one = np.zeros(500, np.int64)
    one[123] = 20_000
    cases["one_column"] = one
    cases["singletons"] = np.ones(50_000, np.int64)
    runs = np.zeros(40_000, np.int64)
    runs[::4000] = 300
    cases["empty_runs"] = runs
    lead = np.concatenate([np.zeros(5000, np.int64), rng.integers(1, 5, 2000), np.zeros(7000, np.int64)])
    cases["leading_trailing_empty"] = lead
    return cases


@pytest.mark.parametrize("case", ["powerlaw", "empties", "one_column", "singletons", "empty_runs",
                                  "leading_trailing_empty"])
@pytest.mark.parametrize("P", [1, 2, 7, 64, 333, 1216, 5000])
def test_setup_and_products_match_oracle(case, P):
    """Device set-up values equal the oracle's Sec. IV-B steps; products match for every chunk count."""
    rng = np.random.default_rng(7)
    deg = _ptr_cases(rng)[case]
    m = max(64, int(deg.max()))
    A = synth.random_matrix(m, deg.shape[0], "csc", degrees=deg, seed=P)
    plan, stored = make_plan(A, torch.float32, chunks=P)
    po = plan_oracle.plan(A.ptr, P)
    ch = plan.chunks()
    for name in ("needLeft", "needRight", "leftGroupEnd", "rightGroup", "leftGroup", "procsOnLeft", "procsOnRight"):
        assert [c[name] for c in ch] == getattr(po, name).tolist(), name
    assert [c["nz_begin"] for c in ch] == po.begin.tolist()
    assert [c["nz_end"] for c in ch] == po.end.tolist()
    ne = po.nonempty
    assert [c["jf"] for c, e in zip(ch, ne) if e] == po.jf[ne].tolist()
    assert [c["jl"] for c, e in zip(ch, ne) if e] == po.jl[ne].tolist()
    assert plan.info()["zones"] == po.z
    check_products(plan, stored, synth.uniform_vector(A.n, 1), synth.uniform_vector(A.m, 2), 1e-5, f"{case} P={P}")


@pytest.mark.parametrize("tile_items,stages,warps", [(64, 2, 1), (128, 4, 3), (992, 2, 4), (256, 3, 16), (40, 4, 7), (256, 2, 24), (384, 2, 20), (256, 2, 16), (512, 2, 16)])
def test_tiling_options(tile_items, stages, warps):
    A = synth.random_matrix(700, 30_000, "csc", degrees=np.minimum(np.random.default_rng(1).zipf(1.9, 30_000), 700),
                            seed=9)
    plan, stored = make_plan(A, torch.float32, tile_items=tile_items, stages=stages, warps_per_cta=warps)
    assert plan.info()["tile_items"] == tile_items
    check_products(plan, stored, synth.uniform_vector(A.n, 1), synth.uniform_vector(A.m, 2), 1e-5, "tiling")


@pytest.mark.parametrize("layout", ["csc", "csr"])
def test_short_vector_in_global_memory(layout):
    """Forced and natural off-chip paths (short dimension too long for shared memory)."""
    m, n = (3000, 60_000) if layout == "csc" else (60_000, 3000)
    A = synth.random_matrix(m, n, layout, density=0.001, seed=21)
    plan, stored = make_plan(A, torch.float32, flags=pkg.SPMV_PLAN_SHORT_IN_GLOBAL)
    assert plan.info()["short_on_chip"] == 0
    check_products(plan, stored, synth.uniform_vector(n, 1), synth.uniform_vector(m, 2), 1e-5, "forced global")
    m, n = (120_000, 400_000) if layout == "csc" else (400_000, 120_000)
    A = synth.random_matrix(m, n, layout, density=2e-5, seed=22)
    plan, stored = make_plan(A, torch.float32)
    assert plan.info()["short_on_chip"] == 0
    check_products(plan, stored, synth.uniform_vector(n, 1), synth.uniform_vector(m, 2), 1e-5, "large short dim")


def test_short_vector_at_shared_memory_limit():
    """The longest short dimension kept on chip, and one element more."""
    A0 = synth.random_matrix(2, 5000, "csc", density=0.5, seed=1)
    plan0, _ = make_plan(A0, torch.float32)
    smem_left = plan0.info()  # noqa: F841 (configuration only)
    # find the boundary by bisection over m with cheap empty-ish matrices
    lo, hi = 1000, 60_000
    while lo + 1 < hi:
        mid = (lo + hi) // 2
        A = synth.random_matrix(mid, 10, "csc", degrees=np.ones(10, np.int64), seed=2)
        if make_plan(A, torch.float32)[0].info()["short_on_chip"]:
            lo = mid
        else:
            hi = mid
    for m in (lo, hi):
        A = synth.random_matrix(m, 50_000, "csc", density=2.0 / m, seed=m)
        plan, stored = make_plan(A, torch.float32)
        assert plan.info()["short_on_chip"] == (1 if m == lo else 0)
        check_products(plan, stored, synth.uniform_vector(A.n, 1), synth.uniform_vector(m, 2), 1e-5, f"m={m}")


def test_zero_nonzeros_and_empty_shapes():
    for (m, n) in [(5, 7), (1, 1), (0, 4), (4, 0)]:
        A = synth.SparseMatrix("csc", m, n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0))
        plan, stored = make_plan(A, torch.float32)
        y = host_of(plan.spmv(dev_vec(np.ones(n), torch.float32)))
        u = host_of(plan.spvtm(dev_vec(np.ones(m), torch.float32)))
        assert not y.any() and not u.any() and y.shape == (m,) and u.shape == (n,)


def test_duplicates_and_unsorted_indices():
    A = synth.random_matrix(50, 3000, "csc", density=0.1, seed=4, duplicates=True)
    plan, stored = make_plan(A, torch.float64)
    check_products(plan, stored, synth.uniform_vector(A.n, 1), synth.uniform_vector(A.m, 2), 1e-12, "dups")


def test_host_pointers_match_device():
    A = synth.random_matrix(400, 30_000, "csc", density=0.01, seed=8)
    plan, stored = make_plan(A, torch.float32)
    x = synth.uniform_vector(A.n, 1).astype(np.float32)
    v = synth.uniform_vector(A.m, 2).astype(np.float32)
    y_dev = host_of(plan.spmv(torch.from_numpy(x).to(DEV)))
    u_dev = host_of(plan.spvtm(torch.from_numpy(v).to(DEV)))
    y_host = np.empty(A.m, np.float32)
    u_host = np.empty(A.n, np.float32)
    pkg.spmv(plan.handle, x, y_host)
    pkg.spvtm(plan.handle, torch.from_numpy(v).pin_memory(), u_host)
    assert np.array_equal(y_host.astype(np.float64), y_dev) or np.allclose(y_host, y_dev, rtol=1e-6, atol=1e-6)
    assert np.array_equal(u_host.astype(np.float64), u_dev)


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=str)
def test_host_vectors_pinned_misaligned_or_pageable(layout, dtype):
    """Host inputs and outputs of every kind (pinned, a pinned view off the 16-byte grid,
    pageable) go through the staging buffers and agree with the device-vector results (the
    segmented pass bit for bit) and with the oracle."""
    m, n = (400, 30_000) if layout == "csc" else (30_000, 400)
    A = synth.random_matrix(m, n, layout, density=0.01, seed=18)
    plan, stored = make_plan(A, dtype)
    vt = plan.vec_dtype
    x = dev_vec(synth.uniform_vector(n, 1), vt)
    v = dev_vec(synth.uniform_vector(m, 2), vt)
    y_dev, u_dev = plan.spmv(x).cpu(), plan.spvtm(v).cpu()
    seg_dev = u_dev if layout == "csc" else y_dev
    for kind in ("pinned", "pinned_offset", "pageable"):
        if kind == "pageable":
            y_h, u_h = torch.empty(m, dtype=vt), torch.empty(n, dtype=vt)
        else:
            off = 1 if kind == "pinned_offset" else 0
            y_h = torch.empty(m + off, dtype=vt, pin_memory=True)[off:]
            u_h = torch.empty(n + off, dtype=vt, pin_memory=True)[off:]
        for src in (x, x.cpu().pin_memory()):
            pkg.spmv(plan.handle, src, y_h)
            pkg.spvtm(plan.handle, v if src.is_cuda else v.cpu().pin_memory(), u_h)
            plan.check()
            xs, vs = host_of(x), host_of(v)
            tol = TOL[dtype]
            assert_close(y_h.double().numpy(), oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), tol, kind)
            assert_close(u_h.double().numpy(), oracle.spvtm(stored, vs), oracle.abs_spvtm(stored, vs), tol, kind)
            seg_host = u_h if layout == "csc" else y_h
            assert torch.equal(seg_host, seg_dev), kind


@pytest.mark.parametrize("which", ["wide", "tall"])
def test_host_vectors_on_large_plans(which):
    """Pageable and pinned host vectors, and pinned long vectors with the short side on the
    device, on power-law matrices of a few million nonzeros: all agree with the oracle, and
    repeated calls agree bit for bit on the segmented pass."""
    if which == "wide":
        A = synth.wide_fp32_large(1, device="cuda", scale=0.06)
    else:
        A = synth.tall_fp32_large(2, device="cuda", scale=0.03)
    stored = synth.SparseMatrix(A.layout, A.m, A.n, A.ptr.cpu().numpy(), A.idx.cpu().numpy(),
                                A.vals.double().cpu().numpy())
    plan = pkg.Plan(A.m, A.n, A.ptr, A.idx, A.vals, layout=A.layout)
    g = torch.Generator(device=DEV)
    g.manual_seed(19)
    x = (torch.rand(A.n, generator=g, device=DEV) * 2 - 1).cpu()
    v = (torch.rand(A.m, generator=g, device=DEV) * 2 - 1).cpu()
    xs, vs = x.double().numpy(), v.double().numpy()
    y_ref, u_ref = oracle.spmv(stored, xs), oracle.spvtm(stored, vs)
    y_sc, u_sc = oracle.abs_spmv(stored, xs), oracle.abs_spvtm(stored, vs)
    seg = []
    for kind in ("pageable", "pinned", "pinned", "pinned_short_on_device"):
        pin = kind != "pageable"
        xh, vh = (x.pin_memory(), v.pin_memory()) if pin else (x.clone(), v.clone())
        yh, uh = torch.empty(A.m, pin_memory=pin), torch.empty(A.n, pin_memory=pin)
        if kind == "pinned_short_on_device":  # the short side on the device, the long one pinned
            if A.layout == "csc":
                yd = torch.empty(A.m, device=DEV)
                pkg.spmv(plan.handle, xh, yd)
                yh = yd.cpu()
                pkg.spvtm(plan.handle, v.to(DEV), uh)
            else:
                ud = torch.empty(A.n, device=DEV)
                pkg.spvtm(plan.handle, vh, ud)
                uh = ud.cpu()
                pkg.spmv(plan.handle, x.to(DEV), yh)
        else:
            pkg.spmv(plan.handle, xh, yh)
            pkg.spvtm(plan.handle, vh, uh)
        plan.check()
        assert_close(yh.double().numpy(), y_ref, y_sc, 1e-5, f"{which} {kind} y")
        assert_close(uh.double().numpy(), u_ref, u_sc, 1e-5, f"{which} {kind} u")
        if pin:
            seg.append((uh if A.layout == "csc" else yh).clone())
    assert torch.equal(seg[0], seg[1]) and torch.equal(seg[0], seg[2])


def test_segdot_is_bitwise_deterministic():
    A = synth.random_matrix(3000, 200_000, "csc", density=0.002, seed=10)
    plan, _ = make_plan(A, torch.float32)
    v = dev_vec(synth.uniform_vector(A.m, 3), torch.float32)
    u1 = plan.spvtm(v).clone()
    for _ in range(3):
        assert torch.equal(plan.spvtm(v), u1)


def test_errors_are_reported_not_raised_on_device():
    A = synth.random_matrix(20, 100, "csc", density=0.2, seed=1)
    t, _ = device_matrix(A, torch.float32)
    bad = t["ptr"].clone()
    bad[5] = bad[6] + 3  # decreasing pointer
    with pytest.raises(pkg.SpmvError) as e:
        pkg.Plan(20, 100, bad, t["idx"], t["vals"])
    assert e.value.status == 2
    bidx = t["idx"].clone()
    bidx[0] = 20
    with pytest.raises(pkg.SpmvError) as e:
        pkg.Plan(20, 100, t["ptr"], bidx, t["vals"])
    assert e.value.status == 2
    with pytest.raises(pkg.SpmvError) as e:  # (f32 values, f64 vectors) is not a supported pair
        pkg.Plan(20, 100, t["ptr"], t["idx"], t["vals"], vec_dtype=torch.float64)
    assert e.value.status == 8
    plan = pkg.Plan(20, 100, t["ptr"], t["idx"], t["vals"])
    x = torch.zeros(101, dtype=torch.float32, device=DEV)
    y = torch.zeros(20, dtype=torch.float32, device=DEV)
    with pytest.raises(pkg.SpmvError) as e:  # misaligned device pointer
        pkg.spmv(plan.handle, x.data_ptr() + 4, y)
    assert e.value.status == 1
    plan.check()


@pytest.mark.parametrize("layout", ["csc", "csr"])
@pytest.mark.parametrize("flags", [0, pkg.SPMV_PLAN_SHORT_IN_GLOBAL])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=str)
def test_unvalidated_out_of_range_indices_set_the_device_error(layout, flags, dtype):
    """With validation skipped, out-of-range indices are never dereferenced: every
    product runs to completion, spmv_check reports SPMV_ERR_DEVICE, and the next plan
    on a valid matrix is unaffected."""
    m, n = (300, 20_000) if layout == "csc" else (20_000, 300)
    A = synth.random_matrix(m, n, layout, density=0.01, seed=5)
    t, stored = device_matrix(A, dtype)
    bidx = t["idx"].clone()
    n_minor = m if layout == "csc" else n
    for pos, val in ((3, n_minor + 7), (A.nnz // 2, 1 << 30), (A.nnz - 1, -1)):
        bidx[pos] = val
    plan = pkg.Plan(m, n, t["ptr"], bidx, t["vals"], layout=layout, vec_dtype=torch.float32,
                    flags=flags | pkg.SPMV_PLAN_NO_VALIDATE, tile_items=512, stages=2)
    x = dev_vec(synth.uniform_vector(n, 1), torch.float32)
    v = dev_vec(synth.uniform_vector(m, 2), torch.float32)
    plan.spmv(x)
    plan.spvtm(v)
    plan.dvalues(v, x)
    plan.batch(pkg.SPMV_OP_AX, torch.stack([x, x, x]))
    plan.batch(pkg.SPMV_OP_VTA, torch.stack([v, v]))
    torch.cuda.synchronize()
    with pytest.raises(pkg.SpmvError) as e:
        plan.check()
    assert e.value.status == 5
    plan.close()
    good, stored = make_plan(A, dtype)
    check_products(good, stored, synth.uniform_vector(n, 1), synth.uniform_vector(m, 2), 1e-5, "after error")


def test_wide_fp64_workload_matches_oracle():
    """The m=1,000 x n=100,000 FP64 workload (Zipf(2) degrees, 5 dense columns)."""
    A = synth.wide_fp64_small(0)
    plan, stored = make_plan(A, torch.float64)
    check_products(plan, stored, synth.uniform_vector(A.n, 100), synth.uniform_vector(A.m, 101), 1e-12, "wide fp64")
    info = plan.info()
    assert info["imbalance"] * A.nnz / info["chunks"] <= 1.0  # chunk sizes differ by at most one (Sec. II)


@pytest.mark.parametrize("layout", ["csc", "csr"])
def test_stale_slot_contents_do_not_leak(layout):
    """A partial last step reads slot positions past the tile's end: whatever a previous launch
    left there (here: infinities and NaNs of a matrix that holds only those) must not reach the
    sums of the next launch."""
    m, n = (25_000, 900) if layout == "csr" else (900, 25_000)
    A = synth.random_matrix(m, n, layout, density=0.01, seed=2)
    t, stored = device_matrix(A, torch.float32)
    poison = torch.full_like(t["vals"], float("inf"))
    poison[::2] = float("nan")
    bad = pkg.Plan(m, n, t["ptr"], t["idx"], poison, layout=layout, tile_items=64)
    good = pkg.Plan(m, n, t["ptr"], t["idx"], t["vals"], layout=layout, tile_items=64)
    x = dev_vec(synth.uniform_vector(n, 1), torch.float32)
    v = dev_vec(synth.uniform_vector(m, 2), torch.float32)
    for _ in range(3):
        bad.spmv(x)
        bad.spvtm(v)
        y = host_of(good.spmv(x))
        u = host_of(good.spvtm(v))
        xs, vs = host_of(x), host_of(v)
        assert_close(y, oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), 1e-5, "y after a poisoned launch")
        assert_close(u, oracle.spvtm(stored, vs), oracle.abs_spvtm(stored, vs), 1e-5, "u after a poisoned launch")
    good.check()


def test_kernel_timers_count_launches_and_switch_on_and_off():
    A = synth.random_matrix(200, 30_000, "csc", density=0.01, seed=7)
    plan, _ = make_plan(A, torch.float32, flags=pkg.SPMV_PLAN_PROFILE)
    x = dev_vec(synth.uniform_vector(A.n, 1), torch.float32)
    v = dev_vec(synth.uniform_vector(A.m, 2), torch.float32)
    plan.spmv(x)
    plan.spvtm(v)
    ms, n = pkg.spmv_profile_read(plan.handle, 0)  # chunk scatter
    assert n == 1 and ms > 0
    assert pkg.spmv_profile_read(plan.handle, 2)[1] == 1  # chunk dot
    pkg.spmv_profile_enable(plan.handle, False)
    plan.spmv(x)
    assert pkg.spmv_profile_read(plan.handle, 0)[1] == 1
    pkg.spmv_profile_enable(plan.handle, True)
    plan.spmv(x)
    assert pkg.spmv_profile_read(plan.handle, 0)[1] == 2
    pkg.spmv_profile_reset(plan.handle)
    assert pkg.spmv_profile_read(plan.handle, 0) == (0.0, 0)
    quiet, _ = make_plan(A, torch.float32)
    quiet.spmv(x)
    assert pkg.spmv_profile_read(quiet.handle, 0)[1] == 0
    pkg.spmv_profile_enable(quiet.handle, True)
    quiet.spmv(x)
    assert pkg.spmv_profile_read(quiet.handle, 0)[1] == 1
    plan.check()
    quiet.check()
