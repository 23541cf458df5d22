"""The nonzero-partitioned products over several ranks, on CPU gloo ranks.

Each rank runs the partition of Sec. II, the set-up of Sec. IV-B over the ranks and the
two exchange steps (the FP64 all-reduce of the short vector, Sec. III step 2; the
all-gather of boundary partial sums that completes the columns split between ranks,
Sec. IV-A); the local products are the FP64 oracle's loops on the rank's group.  The
assembled results must equal the single-process oracle, and every copy of a shared
long-vector entry must be the same on all ranks that hold it.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth
from oracle import plan as plan_oracle
from paper_1812_00904_gb300 import distributed

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _OracleLocal:
    """Local products of a rank's group by the FP64 oracle (test stand-in for the device plan)."""

    def __init__(self, layout, m, n, ptr, idx, vals):
        self.A = synth.SparseMatrix(layout, m, n, np.asarray(ptr, np.int32), np.asarray(idx, np.int32),
                                    np.asarray(vals, np.float64))

    def spmv(self, x):
        return oracle.spmv(self.A, np.asarray(x, np.float64))

    def spvtm(self, v):
        return oracle.spvtm(self.A, np.asarray(v, np.float64))


def _matrix(case):
    rng = np.random.default_rng(5)
    if case == "wide":
        deg = np.minimum(rng.zipf(1.8, 3000), 120).astype(np.int64)
        deg[1500] = 120  # a full column, split over several ranks
        deg[10:40] = 0
        return synth.random_matrix(120, 3000, "csc", degrees=deg, seed=7)
    if case == "tall":
        deg = np.minimum(rng.zipf(1.8, 2500), 90).astype(np.int64)
        deg[700] = 90
        return synth.random_matrix(2500, 90, "csr", degrees=deg, seed=8)
    if case == "one_column":  # every rank inside the one column
        return synth.random_matrix(400, 1, "csc", degrees=np.array([400]), seed=9)
    # fewer nonzeros than ranks: the trailing groups are empty
    return synth.random_matrix(6, 5, "csc", degrees=np.array([0, 2, 0, 1, 0]), seed=10)


def _rank(rank, world, port, case, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A = _matrix(case)
        D = distributed.DistributedMatrix(A.layout, A.m, A.n, A.ptr, A.idx, np.asarray(A.vals, np.float64),
                                          local=_OracleLocal)
        x = synth.uniform_vector(A.n, 11)
        v = synth.uniform_vector(A.m, 12)
        f, l = D.window
        if A.layout == "csc":
            short = D.spmv(x[f:l + 1]).numpy().tolist()
            win = D.spvtm(v).numpy().tolist()
        else:
            win = D.spmv(x).numpy().tolist()
            short = D.spvtm(v[f:l + 1]).numpy().tolist()
        out[rank] = json.dumps(dict(first=f, last=l, short=short, win=win, zones=D.setup.zones))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("wide", 2), ("wide", 3), ("tall", 3), ("one_column", 4), ("tiny", 5)])
def test_partitioned_products_match_the_single_process_oracle(case, world):
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, case, out), nprocs=world, join=True)
        res = {r: json.loads(out[r]) for r in range(world)}
    A = _matrix(case)
    x = synth.uniform_vector(A.n, 11)
    v = synth.uniform_vector(A.m, 12)
    if A.layout == "csc":
        short_ref, short_scale = oracle.spmv(A, x), oracle.abs_spmv(A, x)
        long_ref, long_scale = oracle.spvtm(A, v), oracle.abs_spvtm(A, v)
    else:
        short_ref, short_scale = oracle.spvtm(A, v), oracle.abs_spvtm(A, v)
        long_ref, long_scale = oracle.spmv(A, x), oracle.abs_spmv(A, x)
    # the short vector is the same on every rank and equals the oracle's
    for r in range(world):
        assert res[r]["short"] == res[0]["short"]
    assert np.all(np.abs(np.array(res[0]["short"]) - short_ref) <= 1e-12 * short_scale + 1e-300)
    # the long vector: every rank's window, shared entries equal on all ranks that hold them
    got = {}
    for r in range(world):
        f, l = res[r]["first"], res[r]["last"]
        for j, val in zip(range(f, l + 1), res[r]["win"]):
            assert got.setdefault(j, val) == val, f"entry {j} differs between ranks"
    covered = np.zeros(len(long_ref), bool)
    for j, val in got.items():
        covered[j] = True
        assert abs(val - long_ref[j]) <= 1e-12 * long_scale[j] + 1e-300, (j, val, long_ref[j])
    # entries held by no rank are segments without nonzeros at the ends of the matrix
    assert np.all(long_ref[~covered] == 0.0)
    # the zones are the set-up's of the same partition computed by the plan oracle
    ptr = np.asarray(A.ptr, np.int64)
    po = plan_oracle.plan(ptr, world)
    assert [tuple(z) for z in res[0]["zones"]] == [(S[0], S[-1], j) for (k, j, S) in po.zones]


def test_zone_setup_reproduces_table_iii():
    """The set-up over ranks on the worked example of Figs. 1-3 gives the printed Table III."""
    g = json.load(open(GOLDEN))
    ptr = np.concatenate([[0], np.cumsum(g["column_counts"]["value"])]).astype(np.int64)
    P = g["P"]
    first, last, nonempty = [], [], []
    for r in range(P):
        a, b = distributed.group_range(int(ptr[-1]), P, r)
        nonempty.append(b > a)
        first.append(distributed.owner_of(ptr, a) if b > a else 0)
        last.append(distributed.owner_of(ptr, b - 1) if b > a else -1)
    st = distributed.zone_setup(first, last, nonempty)
    for name in ("needLeft", "needRight", "leftGroupEnd", "rightGroup", "leftGroup", "procsOnLeft", "procsOnRight"):
        assert getattr(st, name) == g["table3"][name], name
    assert [[k, j + 1, list(range(f, l + 1))] for k, (f, l, j) in enumerate(st.zones)] == g["zones"]["value"]


def test_zone_setup_matches_the_plan_oracle_on_random_partitions():
    rng = np.random.default_rng(13)
    for _ in range(60):
        deg = np.minimum(rng.zipf(1.7, int(rng.integers(1, 400))), 500)
        deg[rng.random(deg.size) < 0.1] = 0
        ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
        P = int(rng.integers(1, 70))
        po = plan_oracle.plan(ptr, P)
        first, last, nonempty = [], [], []
        for r in range(P):
            a, b = distributed.group_range(int(ptr[-1]), P, r)
            nonempty.append(b > a)
            first.append(distributed.owner_of(ptr, a) if b > a else 0)
            last.append(distributed.owner_of(ptr, b - 1) if b > a else -1)
        st = distributed.zone_setup(first, last, nonempty)
        for name in ("needLeft", "needRight", "leftGroupEnd", "rightGroup", "leftGroup", "procsOnLeft", "procsOnRight"):
            assert getattr(st, name) == getattr(po, name).tolist(), name
