"""The nonzero-partitioned products with the device plans as local products.

Two gloo ranks share cuda:0: each multiplies its Sec. II group with the library on the GPU
and the exchanges go through gloo on the host (the kernels never wait on the other rank).
The assembled results must match the FP64 oracle within the FP32 tolerance.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _matrix(layout):
    rng = np.random.default_rng(21)
    if layout == "csc":
        deg = np.minimum(rng.zipf(1.8, 60_000), 700).astype(np.int64)
        deg[30_000] = 700
        return synth.random_matrix(700, 60_000, "csc", degrees=deg, seed=22, duplicates=True)
    deg = np.minimum(rng.zipf(1.8, 60_000), 500).astype(np.int64)
    deg[30_000] = 500
    return synth.random_matrix(60_000, 500, "csr", degrees=deg, seed=23, duplicates=True)


def _rank(rank, world, port, layout, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    from paper_1812_00904_gb300 import distributed

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A = _matrix(layout)
        D = distributed.DistributedMatrix(A.layout, A.m, A.n, A.ptr, A.idx,
                                          torch.from_numpy(np.asarray(A.vals, np.float32)), device=dev)
        x = synth.uniform_vector(A.n, 11).astype(np.float32)
        v = synth.uniform_vector(A.m, 12).astype(np.float32)
        f, l = D.window
        if A.layout == "csc":
            short = D.spmv(torch.from_numpy(x[f:l + 1].copy()).to(dev))
            win = D.spvtm(torch.from_numpy(v).to(dev))
        else:
            win = D.spmv(torch.from_numpy(x).to(dev))
            short = D.spvtm(torch.from_numpy(v[f:l + 1].copy()).to(dev))
        torch.cuda.synchronize()
        out[rank] = json.dumps(dict(first=f, last=l, short=short.cpu().tolist(), win=win.cpu().tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("layout", ["csc", "csr"])
def test_two_ranks_on_device_plans_match_the_oracle(layout):
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, layout, out), nprocs=world, join=True)
        res = {r: json.loads(out[r]) for r in range(world)}
    A = _matrix(layout)
    A32 = synth.SparseMatrix(A.layout, A.m, A.n, A.ptr, A.idx, np.asarray(A.vals, np.float32).astype(np.float64))
    x = synth.uniform_vector(A.n, 11).astype(np.float32).astype(np.float64)
    v = synth.uniform_vector(A.m, 12).astype(np.float32).astype(np.float64)
    if layout == "csc":
        sref, sscale, lref, lscale = oracle.spmv(A32, x), oracle.abs_spmv(A32, x), oracle.spvtm(A32, v), \
            oracle.abs_spvtm(A32, v)
    else:
        sref, sscale, lref, lscale = oracle.spvtm(A32, v), oracle.abs_spvtm(A32, v), oracle.spmv(A32, x), \
            oracle.abs_spmv(A32, x)
    assert res[0]["short"] == res[1]["short"]
    assert np.all(np.abs(np.array(res[0]["short"]) - sref) <= 1e-5 * sscale + 1e-30)
    got = {}
    for r in range(world):
        for j, val in zip(range(res[r]["first"], res[r]["last"] + 1), res[r]["win"]):
            assert got.setdefault(j, val) == val, f"entry {j} differs between ranks"
    for j, val in got.items():
        assert abs(val - lref[j]) <= 1e-5 * lscale[j] + 1e-30, (j, val, lref[j])
