"""The N > 1 host logic of bench.py on CPU ranks (gloo, world size 2): each
rank times its own replica of the workload; the job's time is the slowest
rank's and its throughput counts every rank's units.  No GPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out_path):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        worst = bench.max_over_ranks(torch, dist, world, times[rank], "cpu")
        value = bench.job_throughput(1000, 7, world, worst)
        with open(out_path + ".%d" % rank, "w") as f:
            f.write("%r %r\n" % (worst, value))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp
    world, times = 2, [0.25, 0.75]
    out = str(tmp_path / "res")
    mp.start_processes(_rank_main, args=(world, _free_port(), times, out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        worst, value = map(float, open(out + ".%d" % r).read().split())
        assert worst == 0.75
        assert value == pytest.approx(world * 1000 * 7 / 0.75)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(torch, None, 1, 1.5, "cpu") == 1.5
    assert bench.job_throughput(10, 3, 1, 2.0) == 15.0
