"""Serving runtime: continuous batching over resident matrices (serve_* of the C ABI).

Every served vector must equal what the single-vector call computes on the same
plan: bit for bit in the segmented (dot-product) direction, whose summation order
does not depend on the batch, and within the FP32 tolerance against the FP64 oracle
in the scatter direction, whose shared-memory additions are unordered.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
import paper_1812_00904_gb300 as pkg  # noqa: E402
from gpu_util import DEV, assert_close, dev_vec, device_matrix, host_of  # noqa: E402

GB = 1 << 30


def _segmented(layout, op):
    return (layout == "csc" and op == pkg.SPMV_OP_VTA) or (layout == "csr" and op == pkg.SPMV_OP_AX)


def _matrices():
    specs = [(700, 30_000, "csc", torch.float32, 1), (25_000, 900, "csr", torch.float32, 2),
             (1_200, 20_000, "csc", torch.bfloat16, 3), (500, 8_000, "csc", torch.float32, 4)]
    out = []
    for m, n, layout, dt, seed in specs:
        A = synth.random_matrix(m, n, layout, density=0.01, seed=seed)
        t, stored = device_matrix(A, dt)
        plan = pkg.Plan(m, n, t["ptr"], t["idx"], t["vals"], layout=layout, vec_dtype=torch.float32)
        out.append((A, stored, plan))
    return out


def test_each_result_is_the_same_alone_and_in_the_mix():
    mats = _matrices()
    rng = np.random.default_rng(7)
    reqs = []
    for r in range(48):
        i = int(rng.integers(len(mats)))
        op = int(rng.integers(2))
        k = int(rng.integers(1, 6))
        A = mats[i][0]
        len_in, len_out = (A.n, A.m) if op == pkg.SPMV_OP_AX else (A.m, A.n)
        X = torch.stack([dev_vec(synth.uniform_vector(len_in, 1000 + 7 * r + b), torch.float32) for b in range(k)])
        Y = torch.full((k, len_out), float("nan"), device=DEV)
        reqs.append((i, op, k, X, Y))
    # alone: the single-vector calls
    alone = []
    for i, op, k, X, _ in reqs:
        plan = mats[i][2]
        alone.append(torch.stack([plan.spmv(X[b]) if op == pkg.SPMV_OP_AX else plan.spvtm(X[b]) for b in range(k)]))
    torch.cuda.synchronize()
    # in the mix: all submitted at once to 3 stream slots, coalesced up to 8 vectors per launch
    srv = pkg.serve_create(8 * GB, k_max=8, n_streams=3)
    try:
        ids = [pkg.serve_register(srv, plan.handle) for _, _, plan in mats]
        rids = [pkg.serve_submit(srv, ids[i], op, k, X, Y) for i, op, k, X, Y in reqs]
        for rid in rids:
            pkg.serve_wait(srv, rid, 60_000)
        lat = [pkg.serve_poll(srv, rid) for rid in rids]
        st = pkg.serve_stats(srv)
    finally:
        pkg.serve_destroy(srv)
    assert all(done for done, _ in lat) and all(ms >= 0.0 for _, ms in lat)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["vectors"] == sum(k for _, _, k, _, _ in reqs)
    assert st["launches"] < st["vectors"]  # vectors of waiting requests were coalesced
    for (i, op, k, X, Y), ref in zip(reqs, alone):
        A, stored, plan = mats[i]
        layout = "csc" if A.layout == "csc" else "csr"
        if _segmented(layout, op):
            assert torch.equal(Y, ref), f"request on matrix {i} op {op}: differs from the single-vector call"
        for b in range(k):
            xs = host_of(X[b])
            if op == pkg.SPMV_OP_AX:
                assert_close(host_of(Y[b]), oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), 1e-5, "served Ax")
            else:
                assert_close(host_of(Y[b]), oracle.spvtm(stored, xs), oracle.abs_spvtm(stored, xs), 1e-5, "served vTA")
            scale = oracle.abs_spmv(stored, xs) if op == pkg.SPMV_OP_AX else oracle.abs_spvtm(stored, xs)
            assert_close(host_of(Y[b]), host_of(ref[b]), scale, 1e-5, "alone vs in the mix")


def test_host_registered_matrices_are_admitted_and_evicted_within_the_budget():
    hosts = []
    for seed in range(3):
        A = synth.random_matrix(2_000, 150_000, "csc", density=0.01, seed=40 + seed)
        vals = np.asarray(A.vals, dtype=np.float32)
        hosts.append((A, np.ascontiguousarray(A.ptr, np.int32), np.ascontiguousarray(A.idx, np.int32), vals))

    def register(srv, i):
        A, p, ix, v = hosts[i]
        return pkg.serve_register_host(srv, A.m, A.n, A.nnz, pkg.SPMV_CSC_WIDE, p, ix, v, pkg.SPMV_F32, pkg.SPMV_F32)

    def run(srv, mid, i, seed):
        A = hosts[i][0]
        x = dev_vec(synth.uniform_vector(A.n, seed), torch.float32)
        y = torch.empty(A.m, device=DEV)
        torch.cuda.synchronize()
        pkg.serve_wait(srv, pkg.serve_submit(srv, mid, pkg.SPMV_OP_AX, 1, x, y), 60_000)
        return x, y

    # footprint of one resident matrix, then a budget that holds two of them but not three
    srv = pkg.serve_create(64 * GB, k_max=4, n_streams=2)
    try:
        run(srv, register(srv, 0), 0, 1)
        one = pkg.serve_stats(srv)["resident_bytes"]
    finally:
        pkg.serve_destroy(srv)
    budget = int(2.5 * one)
    srv = pkg.serve_create(budget, k_max=4, n_streams=2)
    try:
        ids = [register(srv, i) for i in range(3)]
        for r, i in enumerate([0, 1, 2, 0, 1, 2, 2, 0]):
            x, y = run(srv, ids[i], i, 500 + r)
            A = hosts[i][0]
            stored = synth.SparseMatrix("csc", A.m, A.n, A.ptr, A.idx, hosts[i][3].astype(np.float64))
            xs = host_of(x)
            assert_close(host_of(y), oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), 1e-5, f"host matrix {i}")
            assert pkg.serve_stats(srv)["resident_bytes"] <= budget
        st = pkg.serve_stats(srv)
        assert st["evictions"] >= 1 and st["admissions"] >= 4 and st["failed"] == 0
    finally:
        pkg.serve_destroy(srv)


def test_serving_errors_are_statuses():
    A = synth.random_matrix(300, 5_000, "csc", density=0.02, seed=9)
    hp, hi, hv = (np.ascontiguousarray(A.ptr, np.int32), np.ascontiguousarray(A.idx, np.int32),
                  np.asarray(A.vals, np.float32))  # borrowed by the runtime until serve_destroy
    srv = pkg.serve_create(1 << 20, k_max=4, n_streams=1)  # 1 MiB: nothing fits
    try:
        mid = pkg.serve_register_host(srv, A.m, A.n, A.nnz, pkg.SPMV_CSC_WIDE, hp, hi, hv, pkg.SPMV_F32, pkg.SPMV_F32)
        x = torch.zeros(A.n, device=DEV)
        y = torch.zeros(A.m, device=DEV)
        with pytest.raises(pkg.SpmvError) as e:
            pkg.serve_submit(srv, mid + 5, pkg.SPMV_OP_AX, 1, x, y)
        assert e.value.status == 9  # unknown matrix
        with pytest.raises(pkg.SpmvError) as e:
            pkg.serve_submit(srv, mid, pkg.SPMV_OP_AX, 0, x, y)
        assert e.value.status == 1
        rid = pkg.serve_submit(srv, mid, pkg.SPMV_OP_AX, 1, x, y)
        with pytest.raises(pkg.SpmvError) as e:
            pkg.serve_wait(srv, rid, 10_000)
        assert e.value.status == 7  # the matrix can never fit the budget
        with pytest.raises(pkg.SpmvError) as e:
            pkg.serve_wait(srv, rid + 100, 10)
        assert e.value.status == 9
    finally:
        pkg.serve_destroy(srv)


def _serving_sized():
    """A dozen matrices of the serving workload's ranges (m 1k-50k short side, wide and tall),
    the widest short sides near the shared-memory limit, nonzeros kept to a few million each."""
    specs = [("csc", 1_000, 400_000, 2_000_000), ("csr", 900_000, 1_500, 3_000_000),
             ("csc", 4_000, 1_000_000, 4_000_000), ("csr", 2_000_000, 8_000, 5_000_000),
             ("csc", 12_000, 300_000, 3_000_000), ("csr", 500_000, 20_000, 2_000_000),
             ("csc", 30_000, 600_000, 4_000_000), ("csr", 700_000, 36_000, 3_000_000),
             ("csc", 44_000, 200_000, 2_500_000), ("csr", 400_000, 50_000, 2_000_000),
             ("csc", 2_500, 5_000_000, 6_000_000), ("csr", 3_000_000, 3_000, 4_000_000)]
    out = []
    for i, (layout, m, n, z) in enumerate(specs):
        A = synth.serving_matrix(dict(id=100 + i, layout=layout, m=m, n=n, nnz=z, seed=9000 + i), device=DEV)
        plan = pkg.Plan(A.m, A.n, A.ptr, A.idx, A.vals, layout=layout)
        stored = synth.SparseMatrix(layout, A.m, A.n, A.ptr.cpu().numpy(), A.idx.cpu().numpy(),
                                    A.vals.double().cpu().numpy())
        out.append((A, stored, plan))
    return out


def test_serving_sized_matrices_alone_and_in_the_mix():
    mats = _serving_sized()
    assert sum(1 for A, _, p in mats if not p.info()["short_on_chip"]) >= 1  # an off-chip short vector is served
    rng = np.random.default_rng(17)
    reqs = []
    for r in range(60):
        i = r % len(mats) if r < 2 * len(mats) else int(rng.integers(len(mats)))
        op = (r // len(mats)) % 2 if r < 2 * len(mats) else int(rng.integers(2))  # every matrix, both ops
        k = int(rng.integers(1, 5))
        A = mats[i][0]
        len_in, len_out = (A.n, A.m) if op == pkg.SPMV_OP_AX else (A.m, A.n)
        g = torch.Generator(device=DEV)
        g.manual_seed(3000 + r)
        X = torch.rand((k, len_in), generator=g, device=DEV) * 2 - 1
        Y = torch.full((k, len_out), float("nan"), device=DEV)
        reqs.append((i, op, k, X, Y))
    alone = []
    for i, op, k, X, _ in reqs:
        plan = mats[i][2]
        alone.append(torch.stack([plan.spmv(X[b]) if op == pkg.SPMV_OP_AX else plan.spvtm(X[b]) for b in range(k)]))
    torch.cuda.synchronize()
    srv = pkg.serve_create(64 * GB, k_max=16, n_streams=4)
    try:
        ids = [pkg.serve_register(srv, plan.handle) for _, _, plan in mats]
        rids = [pkg.serve_submit(srv, ids[i], op, k, X, Y) for i, op, k, X, Y in reqs]
        for rid in rids:
            pkg.serve_wait(srv, rid, 120_000)
        st = pkg.serve_stats(srv)
    finally:
        pkg.serve_destroy(srv)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    for (i, op, k, X, Y), ref in zip(reqs, alone):
        A, stored, plan = mats[i]
        for b in range(k):
            xs = host_of(X[b])
            if op == pkg.SPMV_OP_AX:
                ref_o, scale = oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs)
            else:
                ref_o, scale = oracle.spvtm(stored, xs), oracle.abs_spvtm(stored, xs)
            assert_close(host_of(Y[b]), ref_o, scale, 1e-5, f"served matrix {i} op {op}")
            assert_close(host_of(Y[b]), host_of(ref[b]), scale, 1e-5, f"matrix {i} op {op} alone vs in the mix")
        if _segmented(A.layout, op):
            assert torch.equal(Y, ref), f"matrix {i} op {op}: segmented result differs from the single call"
    for _, _, p in mats:
        p.close()


def test_resident_requests_run_while_another_matrix_is_admitted():
    """A host-registered matrix is copied and planned on the admission thread; requests on an
    already resident matrix submitted right after it complete before that admission ends."""
    big = synth.wide_fp32_large(7, device=DEV, scale=0.2)  # about 40M nonzeros, 320 MB to copy
    hp, hi, hv = big.ptr.cpu().numpy(), big.idx.cpu().numpy(), big.vals.cpu().numpy()
    small = synth.random_matrix(500, 20_000, "csc", density=0.01, seed=71)
    t, stored = device_matrix(small, torch.float32)
    plan = pkg.Plan(small.m, small.n, t["ptr"], t["idx"], t["vals"])
    srv = pkg.serve_create(64 * GB, k_max=4, n_streams=2)
    try:
        rid_small = pkg.serve_register(srv, plan.handle)
        rid_big = pkg.serve_register_host(srv, big.m, big.n, big.nnz, pkg.SPMV_CSC_WIDE, hp, hi, hv, pkg.SPMV_F32,
                                          pkg.SPMV_F32)
        xb = torch.rand(big.n, device=DEV)
        yb = torch.empty(big.m, device=DEV)
        xs = [dev_vec(synth.uniform_vector(small.n, 80 + r), torch.float32) for r in range(20)]
        ys = [torch.empty(small.m, device=DEV) for _ in range(20)]
        torch.cuda.synchronize()
        r_big = pkg.serve_submit(srv, rid_big, pkg.SPMV_OP_AX, 1, xb, yb)
        r_small = [pkg.serve_submit(srv, rid_small, pkg.SPMV_OP_AX, 1, x, y) for x, y in zip(xs, ys)]
        for r in r_small:
            pkg.serve_wait(srv, r, 60_000)
        admitted_meanwhile = pkg.serve_stats(srv)["admissions"]
        pkg.serve_wait(srv, r_big, 120_000)
        st = pkg.serve_stats(srv)
    finally:
        pkg.serve_destroy(srv)
    assert admitted_meanwhile == 0, "the resident requests waited for the admission"
    assert st["admissions"] == 1 and st["failed"] == 0
    for x, y in zip(xs, ys):
        xh = host_of(x)
        assert_close(host_of(y), oracle.spmv(stored, xh), oracle.abs_spmv(stored, xh), 1e-5, "resident request")
    plan.close()


def test_request_table_stays_bounded():
    """10,000 requests, each waited for: the runtime keeps none of them in its table, and a poll
    after the wait still reports the request (from the window of recently reported ones)."""
    A = synth.random_matrix(64, 1_000, "csc", density=0.05, seed=72)
    t, stored = device_matrix(A, torch.float32)
    plan = pkg.Plan(A.m, A.n, t["ptr"], t["idx"], t["vals"])
    x = dev_vec(synth.uniform_vector(A.n, 1), torch.float32)
    y = torch.empty((4, A.m), device=DEV)
    torch.cuda.synchronize()
    srv = pkg.serve_create(GB, k_max=8, n_streams=2)
    try:
        mid = pkg.serve_register(srv, plan.handle)
        peak = 0
        for r in range(10_000):
            rid = pkg.serve_submit(srv, mid, pkg.SPMV_OP_AX, 1, x, y[r % 4])
            pkg.serve_wait(srv, rid, 60_000)
            if r % 1000 == 999:
                peak = max(peak, pkg.serve_stats(srv)["tracked_requests"])
        done, lat = pkg.serve_poll(srv, rid)
        st = pkg.serve_stats(srv)
    finally:
        pkg.serve_destroy(srv)
    assert done and lat >= 0.0
    assert peak == 0 and st["tracked_requests"] == 0 and st["completed"] == 10_000
    plan.close()
