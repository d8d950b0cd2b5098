"""Multi-rank host logic of the replica mode, run as two gloo ranks on CPU:
stream sharding covers every stream once, and the timing reduction gives every
rank the slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2505_07158_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.shard_streams(32, rank, world)
        mx = replicas.max_over_ranks(10.0 + 5.0 * rank)
        dist.barrier()
        q.put((rank, mine, mx))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert res[0][1] + res[1][1] == list(range(32))
    assert res[0][2] == res[1][2] == 15.0


def test_single_process_helpers():
    assert replicas.shard_streams(5, 0, 1) == [0, 1, 2, 3, 4]
    assert sum(len(replicas.shard_streams(7, r, 3)) for r in range(3)) == 7
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(30, 100.0, world=2) == pytest.approx(600.0)
