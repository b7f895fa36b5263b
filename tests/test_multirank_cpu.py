"""The benchmark's multi-rank bookkeeping with two gloo ranks on CPU (no GPU): the job time
is the slowest rank's, the job throughput counts every rank's replica, and the reference
arm runs on rank 0 only."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, device="cpu")
    out[rank] = (ms, bench.job_throughput(1000.0, 4, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 15.0
        assert value == pytest.approx(2 * 4 * 1000.0 / 0.015)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench

    class Args:
        seed = 0
        steps = 1
        warmup = 1
    bench.run_reference(Args(), rank=1)
    assert capsys.readouterr().out == ""
