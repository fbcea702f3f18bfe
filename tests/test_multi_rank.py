"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own
replica, combine into the slowest rank's time and the units of both ranks
(weak scaling, no data exchange between replicas); the reference arm runs on
rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        own_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        total = bench.slowest_rank_ms(own_ms, world)
        rate = bench.whole_job_rate(1e6, world, total)
        out[rank] = (total, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_to_slowest_time_and_total_units():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        total, rate = res[r]
        assert total == 150.0
        assert rate == pytest.approx(2e6 / 0.150)


def test_single_rank_is_its_own_time():
    import bench

    assert bench.slowest_rank_ms(123.0, 1) == 123.0
    assert bench.whole_job_rate(10.0, 1, 1000.0) == pytest.approx(10.0)


def test_reference_arm_other_ranks_exit_without_work(capsys):
    import argparse

    import bench

    args = argparse.Namespace(steps=1, warmup=3)
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""
