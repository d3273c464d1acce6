"""The replica path of bench.py (world size 2 over gloo, on CPU): every rank
rotates its own batch, the timing is the maximum over ranks, the rate counts
every rank's units, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        secs = [2.0, 3.0][rank]
        worst = bench.barrier_max(secs, world, device="cpu")
        rate = bench.replica_rate(256 * 5, secs, world, device="cpu")
        q.put((rank, worst, rate))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_count_all_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, worst, rate in got:
        assert worst == 3.0
        assert rate == pytest.approx(2 * 256 * 5 / 3.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    args = argparse.Namespace(gpus=2, steps=1, warmup=0)
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""
