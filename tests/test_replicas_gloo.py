"""Multi-GPU runs are replicas (each rank reconstructs its own scan, no
data-path collective): the benchmark's only cross-rank steps are a barrier,
the maximum of the ranks' times and the whole-job rate.  This runs those
steps as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        elapsed = 2.0 + rank                        # rank 1 is the slower replica
        dist.barrier()
        t = bench.max_over_ranks(elapsed, world, torch.device("cpu"))
        units = 1000.0                              # the same work on every rank (weak scaling)
        out[rank] = (t, bench.whole_job_rate(units, world, t))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    assert res[0] == res[1]                         # every rank agrees on the job's time and rate
    t, rate = res[0]
    assert t == 3.0
    assert rate == pytest.approx(world * 1000.0 / 3.0)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5, 1, torch.device("cpu")) == 1.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
