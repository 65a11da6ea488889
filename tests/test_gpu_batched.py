"""GPU parity of the batched launch (many molecules, one launch per angular
class, CUDA-graph capture) and of the autotuner (the paper's Algorithm 2):
neither may change the result."""
import numpy as np
import pytest

import molgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_13203_gb300 as g
    g.load()
    return g


def _mols():
    out = []
    for i in range(5):  # uneven sizes and class mixes
        mol = molgen.random_molecule(500 + i, 2 + i % 3, [0, 1, 2] if i % 2 == 0 else [0, 0, 1], 1, 2 + i % 3,
                                     0.1, 30.0, layout="lattice", spacing=2.2)
        out.append((mol, molgen.density(mol, 600 + i)))
    return out


@pytest.mark.parametrize("graph", [1, 0])
def test_batched_matches_oracle_and_single(g, graph):
    g.set_option("graph", graph)
    mols = _mols()
    pairs = [g.ShellPairs(m, 1e-12) for m, _ in mols]
    Ds = [torch.from_numpy(D).cuda() for _, D in mols]
    for rep in range(2):  # second call replays the captured graph
        Js, Ks = g.jk_build_batched(pairs, Ds, precision="fp64")
        torch.cuda.synchronize()
        for (mol, D), p, J, K, Dt in zip(mols, pairs, Js, Ks, Ds):
            Jo, Ko, _ = oracle.jk(mol, D, thresh=1e-12, mode="unique")
            assert np.abs(J.cpu().numpy() - Jo).max() <= 1e-10 * max(1.0, np.abs(Jo).max())
            assert np.abs(K.cpu().numpy() - Ko).max() <= 1e-10 * max(1.0, np.abs(Ko).max())
            J1, K1 = g.jk_build(p, Dt, "fp64")
            assert float((J1 - J).abs().max()) <= 1e-12 * max(1.0, float(J1.abs().max()))
    g.set_option("graph", 1)


@pytest.mark.parametrize("graph", [1, 0])
def test_batched_mixed(g, graph):
    """The batched mixed form (density-weighted FP64 selection, pre-pass outside
    the captured graph) against FP64 builds, and against the single-molecule
    mixed path, which selects the same quartets (its FP32 sums are grouped
    over other warp lanes, so the two agree to FP32 rounding of the small
    contributions, not bit for bit); a second call replays."""
    g.set_option("graph", graph)
    mols = _mols()
    pairs = [g.ShellPairs(m, 1e-12) for m, _ in mols]
    Ds = [torch.from_numpy(D).cuda() for _, D in mols]
    try:
        for rep in range(2):
            if rep == 1:  # new density values under the same pointers: the pre-pass re-reads them
                for D in Ds:
                    D.mul_(1.5)
            Js, Ks = g.jk_build_batched(pairs, Ds, precision="mixed")
            torch.cuda.synchronize()
            for p, J, K, Dt in zip(pairs, Js, Ks, Ds):
                J1, K1 = g.jk_build(p, Dt, "fp64")
                assert float((J1 - J).abs().max()) <= 1e-6 and float((K1 - K).abs().max()) <= 1e-6
                Jm, Km = g.jk_build(p, Dt, "mixed")
                assert float((Jm - J).abs().max()) <= 1e-8 * max(1.0, float(Jm.abs().max()))
                assert float((Km - K).abs().max()) <= 1e-8 * max(1.0, float(Km.abs().max()))
    finally:
        g.set_option("graph", 1)


def test_autotune_keeps_results(g):
    mol, D = molgen.config(1, natom=6)
    p = g.ShellPairs(mol, 1e-10)
    Dt = torch.from_numpy(D).cuda()
    J0, K0 = g.jk_build(p, Dt, "fp64")
    J0, K0 = J0.clone(), K0.clone()
    cfg = g.autotune(p, Dt, "fp64")
    assert cfg and all(v[1] >= 1 for v in cfg.values())
    J1, K1 = g.jk_build(p, Dt, "fp64")
    assert float((J1 - J0).abs().max()) <= 1e-11 * float(J0.abs().max())
    assert float((K1 - K0).abs().max()) <= 1e-11 * float(K0.abs().max())
    # the configuration can be saved and restored (tuner cache)
    q = g.ShellPairs(mol, 1e-10)
    g.set_tuning(q, cfg)
    assert g.tuning(q) == cfg
