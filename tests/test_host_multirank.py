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


def _shard_main(rank, world, port, out_path):
    import torch.distributed as dist
    import bench
    import synthetic as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [S.ensemble_instance_shape(i)[0] for i in range(4096)]
        mine = bench.shard_instances(sizes, world, rank)
        # gather every rank's shard (a test-only exchange; the bench needs none)
        got = [None] * world
        dist.all_gather_object(got, mine)
        with open(out_path + ".%d" % rank, "w") as f:
            f.write(repr(got))
    finally:
        dist.destroy_process_group()


def test_ensemble_shards_cover_every_instance_once_and_balance_nodes(tmp_path):
    """The full 4096-instance ensemble split over two gloo ranks: each rank
    derives its shard by itself, the shards are disjoint and cover every
    instance, and their node counts agree within 5 %."""
    import torch.multiprocessing as mp
    import synthetic as S
    world = 2
    out = str(tmp_path / "shard")
    mp.start_processes(_shard_main, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    shards = [eval(open(out + ".%d" % r).read()) for r in range(world)]
    assert shards[0] == shards[1]                      # both ranks agree on the assignment
    parts = shards[0]
    allidx = sorted(i for part in parts for i in part)
    assert allidx == list(range(4096))
    sizes = [S.ensemble_instance_shape(i)[0] for i in range(4096)]
    nodes = [sum(sizes[i] for i in part) for part in parts]
    assert max(nodes) <= 1.05 * min(nodes)
