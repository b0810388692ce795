"""Multi-rank benchmark logic on CPU (gloo, world size 2): each rank
integrates its own batch (weak scaling), the job time is the slowest rank's
and the throughput counts every rank's neurons."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, n = bench.reduce_over_ranks(1.0 + rank, 100.0 * (rank + 1), "cpu")
    out[rank] = (t, n)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.0, 300.0)


def test_ranks_get_distinct_batches():
    a, _, _ = bench.make_workload("plain20", 0)
    b, _, _ = bench.make_workload("plain20", 1)
    assert a.n_neurons == b.n_neurons
    assert not np.array_equal(a.i_const, b.i_const)
