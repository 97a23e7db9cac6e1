"""Multi-GPU form is replicas: each rank evaluates its own systems and only
the timing is reduced (max over ranks), the whole-job value dividing the
points of all ranks by it.  Checked with two gloo ranks on CPU: each rank
builds its inputs as the bench does (the same grids on every rank, its own
densities), and the point count is summed over the ranks."""
import os
import socket

import numpy as np
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
    from paper_1703_06999_gb300 import inputs
    t = bench.reduce_max(1.5 + rank, "cpu")
    seeds = bench.rank_seeds(rank, 8)
    # the 64-grid workload's recipe on a few small systems: grids from seed 0
    # on every rank, densities from the rank
    sys_r = inputs.uneven_batch(rank, count=5, sizes=(16, 20, 24, 32), shape_seed=0)
    local = sum(x.npts for x in sys_r)
    total = bench.job_points(local, world, "cpu")
    cub = bench.make_workload("cubic24", rank, "cpu")[0]
    q.put((rank, t, seeds, [x.shape for x in sys_r], [x.cell.tolist() for x in sys_r],
           [float(x.n.sum()) for x in sys_r], local, total, float(cub.n.sum())))
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
    res.sort(key=lambda r: r[0])
    assert all(r[1] == 2.5 for r in res)              # max over ranks
    assert not set(res[0][2]) & set(res[1][2])        # independent dimer seeds per rank
    (_, _, _, sh0, c0, n0, l0, t0, k0), (_, _, _, sh1, c1, n1, l1, t1, k1) = res
    assert sh0 == sh1 and c0 == c1                    # the same work on every rank (weak scaling)
    assert all(a != b for a, b in zip(n0, n1))        # independent densities
    assert k0 != k1
    assert l0 == l1 and t0 == t1 == 2 * l0            # job points: the sum over the ranks


def test_rank_zero_keeps_the_single_gpu_workload():
    from paper_1703_06999_gb300 import inputs
    a = inputs.uneven_batch(0, count=4, sizes=(16, 20, 24, 32))
    b = inputs.uneven_batch(0, count=4, sizes=(16, 20, 24, 32), shape_seed=0)
    for x, y in zip(a, b):
        assert x.shape == y.shape and x.functional == y.functional
        assert np.array_equal(x.cell, y.cell) and torch.equal(x.n, y.n)
