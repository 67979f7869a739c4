"""The multi-GPU path of bench.py is replicas only: every rank solves its own batch (seeds offset by
rank) and only the timing (max over ranks) and the counted solves (sum over ranks) are combined.
This covers that host logic with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        seeds = [x.seed for x in bench.workload(16, rank)]
        ms, ok = bench.rank_reduce([10.0 + 5.0 * rank, 3 + rank], ["max", "sum"], ws, "cpu")
        out.put((rank, seeds, ms, ok))
    finally:
        dist.destroy_process_group()


def test_two_replicas_shard_the_seeds_and_combine_time_and_counts():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, seeds, ms, ok = q.get(timeout=120)
        res[r] = (seeds, ms, ok)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert not set(res[0][0]) & set(res[1][0])           # each replica has its own instances
    for r in range(2):
        assert res[r][1] == 15.0 and res[r][2] == 7.0     # max of the times, sum of the counts


def test_one_rank_is_a_no_op():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_reduce([2.5, 4], ["max", "sum"], 1, "cpu") == [2.5, 4.0]
