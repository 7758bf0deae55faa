"""The multi-GPU path of bench.py on CPU: two gloo ranks.

bench.py runs one independent chain per GPU (the MH chain is serial, so the
only collective is the timing): every rank must get the slowest rank's time,
the same whole-job rate, and a chain seed of its own.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = 1.0 + 0.5 * rank  # rank 1 is the slower one
    t = bench.max_over_ranks(t_local, dist, "cpu")
    out[rank] = (t, bench.whole_job_rate(1000.0, world, t), bench.replica_seed(5, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timing_and_keep_own_seeds():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 1.5
    assert res[0][1] == res[1][1] == pytest.approx(2 * 1000.0 / 1.5)
    assert res[0][2] != res[1][2]
    # without a process group the value is the rank's own
    assert bench.max_over_ranks(2.5) == 2.5
