"""The multi-rank host logic on CPU: two gloo ranks partition a batch of
independent molecules (disjoint, complete, balanced) and reduce timings with
a max over ranks, as bench.py does under torchrun."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, costs, out):
    import torch.distributed as dist
    from paper_2412_13203_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = shard.shard(costs, world, rank)
        got = [None] * world
        dist.all_gather_object(got, mine)
        tmax = shard.max_over_ranks([10.0 * (rank + 1), -rank])
        out.put((rank, got, tmax))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    costs = [float((7 * i) % 13 + 1) for i in range(64)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    got0, got1 = res[0][1], res[1][1]
    assert got0 == got1
    a, b = set(got0[0]), set(got0[1])
    assert not (a & b) and a | b == set(range(64))
    la, lb = sum(costs[i] for i in a), sum(costs[i] for i in b)
    assert abs(la - lb) <= max(costs)
    for _, _, tmax in res:
        assert tmax == [20.0, 0.0]


def test_shard_single_rank_and_errors():
    from paper_2412_13203_gb300 import shard
    assert shard.shard([3, 1, 2], 1, 0) == [0, 1, 2]
    with pytest.raises(ValueError):
        shard.shard([1], 2, 2)
    assert shard.max_over_ranks([1.5, 2.0]) == [1.5, 2.0]
