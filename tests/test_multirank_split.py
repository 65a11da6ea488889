"""The multi-GPU split of one molecule on CPU (no GPU needed): the library's
cost-balanced partition rule (``jk_partition``, host code exported by the C
ABI) and the one-collective reduction of partial J and K
(``allreduce_jk``), run as two gloo ranks.  Each rank takes its cost-balanced
range of a molecule's unique shell quartets, the oracle gives that range's
J/K contributions, and the all-reduce must give the oracle's full J and K:
the data path of ``jk_build_distributed`` with the oracle standing in for
the GPU part build (Sec. 4, stage 2: quartet blocks are independent)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    from paper_2412_13203_gb300 import build
    build.build()
    import paper_2412_13203_gb300 as g
    g.load()
    return g


def _check_bounds(b, cost, nparts):
    n = len(cost)
    assert b[0] == 0 and b[-1] == n and len(b) == nparts + 1
    assert np.all(np.diff(b) >= 0)  # contiguous, ordered: every unit in exactly one part
    pre = np.concatenate([[0.0], np.cumsum(cost)])
    parts = pre[b[1:]] - pre[b[:-1]]
    cmax = float(np.max(cost)) if n else 0.0
    assert np.all(np.abs(parts - pre[-1] / nparts) <= cmax * (1 + 1e-12) + 1e-9), (parts, cmax)
    return parts


def test_partition_rule(g):
    rng = np.random.Generator(np.random.PCG64(5))
    for n, nparts in ((1000, 2), (1000, 8), (37, 5), (5, 8), (1, 3), (64, 64)):
        cost = rng.gamma(0.7, 100.0, size=n)  # skewed, like rows of very different primitive counts
        b = g.partition(cost, nparts)
        _check_bounds(b, cost, nparts)
    # one dominant unit: the rule cannot split it, the others share what is left
    cost = np.ones(100)
    cost[10] = 1e6
    _check_bounds(g.partition(cost, 4), cost, 4)
    # zero total cost: equal counts
    b = g.partition(np.zeros(10), 4)
    assert list(b) == [0, 2, 5, 7, 10]
    # empty input and one part
    assert list(g.partition(np.zeros(0), 3)) == [0, 0, 0, 0]
    assert list(g.partition(np.arange(5.0), 1)) == [0, 5]


def test_partition_rejects_bad_input(g):
    with pytest.raises(g.JKError):
        g.partition([1.0, -2.0], 2)
    with pytest.raises(g.JKError):
        g.partition([1.0, float("nan")], 2)
    with pytest.raises(g.JKError):
        g.partition([1.0, 2.0], 0)


def _unique_quartets(S):
    out = []
    for a in range(S):
        for b in range(a + 1):
            ab = a * (a + 1) // 2 + b
            for c in range(S):
                for d in range(c + 1):
                    if c * (c + 1) // 2 + d <= ab:
                        out.append((a, b, c, d))
    return np.array(out, dtype=np.int32)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import molgen
    import oracle
    import paper_2412_13203_gb300 as g
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mol = molgen.random_molecule(41, 3, [0, 1, 2], 1, 3, 0.15, 8.0, layout="cube", box=4.0, min_spacing=1.2)
        D = molgen.density(mol, 13)
        q = _unique_quartets(mol.nshell)
        k = np.asarray(mol.shell_nprim, dtype=np.float64)
        cost = k[q[:, 0]] * k[q[:, 1]] * k[q[:, 2]] * k[q[:, 3]]  # primitive quartets of every quartet
        b = g.partition(cost, world)
        Jp, Kp = oracle.jk_quartets(mol, D, q[b[rank]:b[rank + 1]])
        JK = torch.from_numpy(np.stack([Jp, Kp]))
        J, K = JK[0], JK[1]
        g.allreduce_jk(J, K)
        # a separate pair of tensors (not views of one buffer) takes the stacked path
        J2, K2 = torch.from_numpy(Jp.copy()), torch.from_numpy(Kp.copy())
        g.allreduce_jk(J2, K2)
        out.put((rank, J.numpy().copy(), K.numpy().copy(), J2.numpy().copy(), K2.numpy().copy(),
                 [int(x) for x in b], float(cost[b[rank]:b[rank + 1]].sum()), float(cost.sum()), float(cost.max())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_one_molecule(g):
    import torch.multiprocessing as mp
    import molgen
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in procs], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mol = molgen.random_molecule(41, 3, [0, 1, 2], 1, 3, 0.15, 8.0, layout="cube", box=4.0, min_spacing=1.2)
    D = molgen.density(mol, 13)
    Jo, Ko, _ = oracle.jk(mol, D, mode="all")
    for _, J, K, J2, K2, b, mine, tot, cmax in res:
        assert res[0][5] == b  # every rank derives the same partition
        assert abs(mine - tot / 2) <= cmax
        for X, Xo in ((J, Jo), (K, Ko), (J2, Jo), (K2, Ko)):
            assert np.abs(X - Xo).max() <= 1e-12 * np.abs(Xo).max()
    # the two parts are both real work
    assert 0 < res[0][5][1] < res[0][5][2]
