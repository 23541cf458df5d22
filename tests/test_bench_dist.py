"""The multi-rank benchmark path on CPU: two gloo ranks, as `bench.py --gpus 2` runs replicas.

Each rank times its own replica; the job's time is the maximum over the ranks and
the value aggregates the bytes of all ranks (weak scaling).  The data path itself
has no collective: only the timing is reduced.
"""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 * (rank + 1)  # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, world, torch.device("cpu"))
        out[rank] = (ms_max, bench.whole_job_gbs(1_000_000_000, 10, world, ms_max))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_max_time_and_the_whole_job_value():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]  # every rank sees the same job time
    ms_max, gbs = res[0]
    assert ms_max == 20.0
    assert abs(gbs - 1_000_000_000 * 10 * 2 / 0.020 / 1e9) < 1e-9  # 1000 GB/s over both replicas
