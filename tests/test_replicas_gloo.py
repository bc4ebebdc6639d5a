"""The multi-GPU path is replicas only (independent solves per rank, weak
scaling): the bench's whole-job aggregation is checked with two gloo ranks on
the CPU (slowest rank's time, sum of the units all ranks processed)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    def red(op):
        def f(v):
            t = torch.tensor([v], dtype=torch.float64)
            dist.all_reduce(t, op=op)
            return float(t.item())
        return f

    local_ms = 100.0 + 50.0 * rank            # rank 1 is the slower replica
    units = 1000.0 * (rank + 1)
    ms, total, value = bench.replica_aggregate(local_ms, units, world, red(dist.ReduceOp.MAX),
                                               red(dist.ReduceOp.SUM))
    dist.barrier()
    out[rank] = (ms, total, value)
    dist.destroy_process_group()


def test_two_replicas_aggregate_over_gloo():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        ms, total, value = out[r]
        assert ms == 150.0 and total == 3000.0
        assert value == pytest.approx(3000.0 / 0.150)


def test_single_replica_needs_no_collective():
    import bench
    boom = lambda v: (_ for _ in ()).throw(AssertionError("no collective at N=1"))
    assert bench.replica_aggregate(20.0, 500.0, 1, boom, boom) == (20.0, 500.0, 500.0 / 0.02)
