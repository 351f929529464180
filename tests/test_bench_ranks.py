"""Host logic of bench.py's multi-rank path, on CPU with two gloo ranks:
every rank reports the slowest rank's time, and throughput aggregates the
units of all ranks over that time (weak scaling, one replica per rank)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank
    ms = bench.max_over_ranks(local_ms, world, "cpu")
    rate = bench.aggregate_rate(100, ms / 1e3, world)
    out[rank] = (ms, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] == res[1][1] == pytest.approx(2 * 100 / 0.015)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.aggregate_rate(10, 2.0, 1) == 5.0


def _shard_main(rank, world, port, out):
    import torch.distributed as dist
    import workloads as W
    from paper_2311_18783_gb300.api import shard_problems
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ps = W.many_problems(24, seed=3)
    mine = shard_problems(ps, rank, world)
    cells = sum(int(w.active.sum()) for i, w in enumerate(ps) if i in mine)
    t = torch.tensor([float(cells), float(len(mine))])
    parts = [torch.zeros(2) for _ in range(world)]
    dist.all_gather(parts, t)
    out[rank] = (mine, [p.tolist() for p in parts])
    dist.barrier()
    dist.destroy_process_group()


def test_independent_problems_shard_gloo():
    """The batching workload's independent problems split over two gloo
    ranks with no overlap and no gap, and the active-cell loads stay within
    the largest problem of each other."""
    import torch.multiprocessing as mp
    import workloads as W
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_shard_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    got = sorted(res[0][0] + res[1][0])
    assert got == list(range(24))
    assert not set(res[0][0]) & set(res[1][0])
    loads = [p[0] for p in res[0][1]]
    assert res[0][1] == res[1][1]
    biggest = max(int(w.active.sum()) for w in W.many_problems(24, seed=3))
    assert abs(loads[0] - loads[1]) <= biggest
