"""Multi-GPU form is replicas: each rank evaluates its own systems and only
the timing is reduced (max over ranks).  Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


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
    import bench
    t = bench.reduce_max(1.5 + rank, "cpu")
    seeds = bench.rank_seeds(rank, 8)
    q.put((rank, t, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_max_and_disjoint_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert all(t == 2.5 for _, t, _ in res)          # max over ranks
    assert not set(res[0][2]) & set(res[1][2])        # independent systems per rank
