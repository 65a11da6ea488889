"""Host-side logic of the multi-GPU path: independent problems (molecules of a
batch, or one replica of a workload per rank) are partitioned over ranks with
no collective on the data path; the only collectives are the timing
reductions of a benchmark.

One process drives one GPU.  J and K of a molecule are never split across
ranks, so no all-reduce of J or K is needed."""
from __future__ import annotations


def shard(costs, world: int, rank: int) -> list[int]:
    """Indices of the problems rank `rank` of `world` owns: longest-processing-
    time-first greedy assignment by estimated cost (e.g. screened quartets x
    primitive quartets), ties broken by index, identical on every rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += float(costs[i])
    return [i for i in range(len(costs)) if owner[i] == rank]


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks of the default
    process group (the input itself when torch.distributed is not
    initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]
