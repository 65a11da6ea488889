"""Failure handling through the C ABI, made on the host (no GPU fault is
provoked): malformed densities caught by the optional check (a NaN or an
infinity, a non-symmetric D), an injected device-allocation failure in the
middle of a pair build and of a J/K build, and a corrupted tuner
configuration.  Each call must return its error status with a message, leave
the library usable, and change nothing it should not."""
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
    mol, D = molgen.config(1, natom=4)
    pairs = g.ShellPairs(mol, 1e-10)
    yield mol, torch.from_numpy(D).cuda(), pairs
    pairs.free()


def _status(e):
    return e.value.code


def test_density_check(g, case):
    _, D, pairs = case
    J0, K0 = g.jk_build(pairs, D, "fp64")
    g.set_option("check_symmetry", 1)
    try:
        J, K = g.jk_build(pairs, D, "fp64")  # a symmetric D passes
        assert float((J - J0).abs().max()) <= 1e-14 * float(J0.abs().max())
        bad = D.clone()
        bad[1, 2] += 1e-3
        with pytest.raises(g.JKError) as e:
            g.jk_build(pairs, bad, "fp64")
        assert _status(e) == -6 and "not symmetric" in str(e.value)
        for v in (float("nan"), float("inf")):
            bad = D.clone()
            bad[3, 3] = v
            with pytest.raises(g.JKError) as e:
                g.jk_build(pairs, bad, "mixed")
            assert _status(e) == -1 and "non-finite" in str(e.value)
    finally:
        g.set_option("check_symmetry", 0)
    J, K = g.jk_build(pairs, D, "fp64")  # still usable
    assert float((J - J0).abs().max()) <= 1e-14 * float(J0.abs().max())
    assert float((K - K0).abs().max()) <= 1e-14 * float(K0.abs().max())


def test_injected_allocation_failure(g, case):
    mol, D, pairs = case
    J0, K0 = g.jk_build(pairs, D, "fp64")
    try:
        for n in (0, 3, 9):  # fail at different points of the pair build
            g.set_option("fail_alloc_after", n)
            with pytest.raises(g.JKError) as e:
                g.ShellPairs(mol, 1e-10)
            assert _status(e) == -2 and "injected" in str(e.value)
        g.set_option("fail_alloc_after", -1)
        fresh = g.ShellPairs(mol, 1e-10)  # nothing leaked into the next build
        g.set_option("fail_alloc_after", 0)
        with pytest.raises(g.JKError) as e:
            g.jk_build(fresh, D, "fp64")  # its compensation scratch is not there yet
        assert _status(e) == -2
    finally:
        g.set_option("fail_alloc_after", -1)
    J, K = g.jk_build(fresh, D, "fp64")
    assert float((J - J0).abs().max()) <= 1e-14 * float(J0.abs().max())
    assert float((K - K0).abs().max()) <= 1e-14 * float(K0.abs().max())
    fresh.free()


def test_corrupted_tuning_changes_nothing(g, case):
    _, D, pairs = case
    cfg = g.tuning(pairs)
    assert cfg
    J0, K0 = g.jk_build(pairs, D, "mixed")
    cls = next(iter(cfg))
    for bad in ((33, 1, 128, 1), (128, 0, 128, 1), (128, 1, 512, 1), (128, 1, 128, -4)):
        broken = dict(cfg)
        broken[cls] = bad
        with pytest.raises(g.JKError) as e:
            g.set_tuning(pairs, broken)
        assert _status(e) == -1
        assert g.tuning(pairs) == cfg  # rejected as a whole
    J, K = g.jk_build(pairs, D, "mixed")
    assert float((J - J0).abs().max()) <= 1e-12 * float(J0.abs().max())
