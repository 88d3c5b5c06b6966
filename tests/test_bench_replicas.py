"""The replica logic of bench.py under torch.distributed (world size 2, gloo on CPU): every rank
times its own independent problem, the job's time per step is the slowest rank's, and the reported
rate counts the applications of all ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [1.0 + rank, 2.0 * (rank + 1), 0.5 - 0.1 * rank]
        out[rank] = (bench.job_times(local), bench.whole_job_rate(world, bench.job_times(local)[0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_replica():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        times, rate = res[r]
        assert times == [2.0, 4.0, 0.5]
        assert rate == pytest.approx(world * 1000.0 / 2.0)


def test_single_process_keeps_local_times():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_times([3.0, 1.0]) == [3.0, 1.0]
    assert bench.whole_job_rate(1, 0.1) == pytest.approx(10000.0)
