"""The multi-GPU launch path of bench.py, exercised on CPU with two gloo ranks: each rank works on
its own volume (no data-path collective), and the reported throughput is the units of all ranks
over the slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 * (rank + 1)              # rank 1 is the slow one
    value, ms = bench.aggregate(ms_local, units_per_step_per_rank=1000.0, steps=5, world=world)
    out[rank] = (value, ms, bench.rank_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    mgr = mp.get_context("spawn").Manager()   # no fork of a process that may run threads
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    v0, ms0, s0 = out[0]
    v1, ms1, s1 = out[1]
    assert ms0 == ms1 == 200.0                       # max over ranks, seen by every rank
    assert v0 == v1 == pytest.approx(2 * 1000.0 * 5 / 0.2)   # all ranks' units / slowest time
    assert s0 != s1                                  # independent volumes per rank


def test_single_rank_aggregation_needs_no_process_group():
    import bench
    value, ms = bench.aggregate(50.0, 100.0, 4, 1)
    assert ms == 50.0 and value == pytest.approx(100.0 * 4 / 0.05)
