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
