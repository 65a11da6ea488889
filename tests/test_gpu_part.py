"""Partial builds for the multi-GPU split of one molecule (Sec. 4, stage 2:
quartet blocks are independent; Sec. 7, several GPUs), through the C ABI on
one GPU: the parts of every class's cost-balanced row partition sum to the
whole build (J, K in both precisions, the nuclear gradient), the partition
covers every quartet row exactly once, every part holds its share of every
class within one row's cost, and malformed part arguments are rejected."""
import numpy as np
import pytest

import molgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_13203_gb300 as g
    g.load()
    return g


@pytest.fixture(scope="module")
def case(g):
    mol, D = molgen.config(1, natom=8)
    pairs = g.ShellPairs(mol, molgen.CONFIG_THRESH[1])
    yield mol, torch.from_numpy(D).cuda(), pairs
    pairs.free()


def _rel(x, ref):
    return float((x - ref).abs().max() / ref.abs().max())


@pytest.mark.parametrize("nparts", [2, 3, 7])
def test_fp64_parts_sum_to_whole(g, case, nparts):
    _, D, pairs = case
    J, K = g.jk_build(pairs, D, "fp64")
    Js, Ks = torch.zeros_like(J), torch.zeros_like(K)
    for p in range(nparts):
        Jp, Kp = g.jk_build_part(pairs, D, p, nparts, "fp64")
        assert _rel(Jp, J) > 1e-4  # every part carries real work
        Js += Jp
        Ks += Kp
    assert _rel(Js, J) < 1e-12 and _rel(Ks, K) < 1e-12


def test_mixed_parts_sum_to_whole(g, case):
    _, D, pairs = case
    J, K = g.jk_build(pairs, D, "mixed")
    n32, n64 = g.last_split(pairs)
    Js, Ks = torch.zeros_like(J), torch.zeros_like(K)
    s32 = s64 = 0
    for p in range(3):
        Jp, Kp = g.jk_build_part(pairs, D, p, 3, "mixed")
        a, b = g.last_split(pairs)
        s32 += a
        s64 += b
        Js += Jp
        Ks += Kp
    # the same quartets take the same precision in the parts as in the whole
    assert (s32, s64) == (n32, n64)
    assert _rel(Js, J) < 1e-10 and _rel(Ks, K) < 1e-10


def test_partition_covers_and_balances(g, case):
    _, _, pairs = case
    for nparts in (2, 5):
        rows = g.part_rows(pairs, nparts)
        by_cls = {}
        for r in rows:
            by_cls.setdefault(r["cls"], []).append(r)
        assert len(by_cls) == len(g.class_stats(pairs))
        items_total = 0
        for cls, rs in by_cls.items():
            rs.sort(key=lambda r: r["part"])
            assert [r["part"] for r in rs] == list(range(nparts))
            assert rs[0]["r0"] == 0
            for a, b in zip(rs, rs[1:]):
                assert a["r1"] == b["r0"]  # contiguous: every row in exactly one part
            tot = sum(r["cost"] for r in rs)
            for r in rs:
                assert abs(r["cost"] - tot / nparts) <= r["max_row_cost"] + 1
            items_total += sum(r["items"] for r in rs)
        assert items_total > pairs.nquartets / 2


def test_gradient_parts_sum_to_whole(g, case):
    _, D, pairs = case
    G = g.jk_grad(pairs, D, "fp64")
    Gs = sum(g.jk_grad_part(pairs, D, p, 3, "fp64") for p in range(3))
    assert _rel(Gs, G) < 1e-12


def test_part_arguments_rejected(g, case):
    _, D, pairs = case
    with pytest.raises(g.JKError):
        g.jk_build_part(pairs, D, 3, 3)
    with pytest.raises(g.JKError):
        g.jk_build_part(pairs, D, 0, 0)
    with pytest.raises(g.JKError):
        g.jk_grad_part(pairs, D, -1, 2)


def test_distributed_without_group_is_plain_build(g, case):
    _, D, pairs = case
    J, K = g.jk_build(pairs, D, "fp64")
    J2, K2 = g.jk_build_distributed(pairs, D, "fp64")
    assert _rel(J2, J) < 1e-14 and _rel(K2, K) < 1e-14
