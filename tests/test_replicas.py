"""Several GPUs run independent replicas of the step (the method has no
exchange between problems): the benchmark's host logic takes the slowest
rank's time and reports the whole-job rate over it.  Checked here with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [2.0, 3.0][rank]                    # rank 1 is the slow one
    slowest = bench.max_over_ranks(seconds, world, device="cpu")
    out[rank] = (slowest, bench.whole_job_rate(600.0, world, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    world = 2
    with mp.get_context("spawn").Manager() as m:   # no fork of a threaded process
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (3.0, 400.0)   # 2 x 600 units over the slower rank's 3 s


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.whole_job_rate(600.0, 1, 2.0) == 300.0
