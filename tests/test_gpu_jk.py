"""GPU parity: the sm_103a McMurchie-Davidson J/K path against the CPU
Obara-Saika oracle on the same seeded inputs (called through the C ABI)."""
import numpy as np
import pytest

import molgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10  # Eh, absolute, on every J/K element and on energies


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_13203_gb300 as g
    g.load()
    return g


def _run(g, mol, D, thresh=None, prec="fp64"):
    pairs = g.ShellPairs(mol, thresh)
    Dt = torch.from_numpy(D).cuda()
    J, K = g.jk_build(pairs, Dt, prec)
    E = g.jk_energy(Dt, J, K)
    torch.cuda.synchronize()
    return pairs, J.cpu().numpy(), K.cpu().numpy(), E


def test_boys_against_oracle(g):
    Ts = np.concatenate([np.linspace(0, 2, 97), np.linspace(2, 45, 301), [79.99, 80.0, 80.01, 120.0, 1e3]])
    F = g.boys(13, torch.from_numpy(Ts).cuda()).cpu().numpy()
    for T, row in zip(Ts, F):
        ref = oracle.boys(13, float(T))
        assert np.all(np.abs(row - ref) <= 2e-14 * ref + 1e-300), (T, row, ref)
    F32 = g.boys(13, torch.from_numpy(Ts).cuda(), "mixed").cpu().numpy()
    for T, row in zip(Ts, F32):
        ref = oracle.boys(13, float(T))
        assert np.all(np.abs(row - ref) <= 2e-6 * ref + 1e-37)


def test_config0_fp64_matches_oracle(g):
    mol, D = molgen.config(0)
    pairs, J, K, E = _run(g, mol, D)
    Jo, Ko, n = oracle.jk(mol, D, mode="all")
    assert pairs.nquartets == 78 * 79 // 2
    assert np.abs(J - Jo).max() <= FP64_TOL and np.abs(K - Ko).max() <= FP64_TOL
    assert abs(E - oracle.energy(D, Jo, Ko)) <= FP64_TOL


@pytest.mark.parametrize("seed,shells,natom,kmax", [(1, [0, 1, 2], 3, 3), (2, [2, 2, 0], 2, 4), (3, [1, 2], 4, 2),
                                                    (4, [0, 0, 1, 2], 3, 6)])
def test_all_l2_classes_fp64(g, seed, shells, natom, kmax):
    mol = molgen.random_molecule(100 + seed, natom, shells, 1, kmax, 0.05, 5e3, layout="lattice", spacing=2.0)
    D = molgen.density(mol, 200 + seed)
    pairs, J, K, E = _run(g, mol, D)
    Jo, Ko, _ = oracle.jk(mol, D, mode="unique")
    scale = max(1.0, np.abs(Jo).max())
    assert np.abs(J - Jo).max() <= FP64_TOL * scale, np.abs(J - Jo).max()
    assert np.abs(K - Ko).max() <= FP64_TOL * scale, np.abs(K - Ko).max()
    assert abs(E - oracle.energy(D, Jo, Ko)) <= FP64_TOL * max(1.0, abs(E))


def test_screened_fp64_matches_screened_oracle(g):
    mol = molgen.random_molecule(7, 8, [0, 0, 1, 2], 1, 4, 0.05, 5e3, layout="lattice", spacing=2.5)
    D = molgen.density(mol, 8)
    thresh = 1e-8
    pairs, J, K, E = _run(g, mol, D, thresh)
    Jo, Ko, n = oracle.jk(mol, D, thresh=thresh, mode="unique")
    # quartets on the threshold boundary may flip between the two Q evaluations;
    # each flip moves an element by < 8 * thresh * ncomp * max|D|
    assert abs(pairs.nquartets - n) <= max(3, n // 10000)
    bound = FP64_TOL + 8 * 36 * thresh * np.abs(D).max() * abs(pairs.nquartets - n)
    assert np.abs(J - Jo).max() <= bound and np.abs(K - Ko).max() <= bound


def test_mixed_precision_within_target(g):
    mol = molgen.random_molecule(9, 6, [0, 0, 1, 2], 1, 4, 0.05, 5e3, layout="lattice", spacing=2.5)
    D = molgen.density(mol, 10)
    pairs, J, K, E = _run(g, mol, D, 1e-10, "mixed")
    n32, n64 = g.last_split(pairs)
    assert n32 + n64 == pairs.nquartets
    Jo, Ko, _ = oracle.jk(mol, D, thresh=1e-10, mode="unique")
    assert np.abs(J - Jo).max() <= 1e-6 and np.abs(K - Ko).max() <= 1e-6
    assert abs(E - oracle.energy(D, Jo, Ko)) <= 1e-6


@pytest.mark.parametrize("seed,shells,natom,kmax", [(21, [3], 2, 2), (22, [0, 3], 2, 2), (23, [1, 3], 2, 2),
                                                    (24, [2, 3], 2, 2), (25, [3, 3, 0], 2, 1),
                                                    (26, [0, 1, 2, 3], 2, 2)])
def test_f_classes_fp64(g, seed, shells, natom, kmax):
    """Every class with an f shell (the ket-component-chunked kernels), FP64,
    against the oracle's Obara-Saika/HRR J and K."""
    mol = molgen.random_molecule(100 + seed, natom, shells, 1, kmax, 0.1, 200.0, layout="lattice", spacing=1.9)
    D = molgen.density(mol, 200 + seed)
    pairs, J, K, E = _run(g, mol, D)
    Jo, Ko, _ = oracle.jk(mol, D, mode="unique")
    scale = max(1.0, np.abs(Jo).max())
    assert np.abs(J - Jo).max() <= FP64_TOL * scale, np.abs(J - Jo).max()
    assert np.abs(K - Ko).max() <= FP64_TOL * scale, np.abs(K - Ko).max()
    assert abs(E - oracle.energy(D, Jo, Ko)) <= FP64_TOL * max(1.0, abs(E))


def test_f_classes_mixed(g):
    mol = molgen.random_molecule(31, 3, [0, 1, 2, 3], 1, 3, 0.05, 1e3, layout="lattice", spacing=2.6)
    D = molgen.density(mol, 32)
    pairs, J, K, E = _run(g, mol, D, 1e-11, "mixed")
    n32, n64 = g.last_split(pairs)
    assert n32 > 0 and n32 + n64 == pairs.nquartets
    Jo, Ko, _ = oracle.jk(mol, D, thresh=1e-11, mode="unique")
    assert np.abs(J - Jo).max() <= 1e-6 and np.abs(K - Ko).max() <= 1e-6
    assert abs(E - oracle.energy(D, Jo, Ko)) <= 1e-6


@pytest.mark.parametrize("seed,shells,natom,kmax", [(41, [0, 1, 2], 3, 3), (42, [2, 2, 1], 2, 4), (43, [2, 0, 1, 2], 3, 2)])
def test_all_fp32_kernels_against_oracle(g, seed, shells, natom, kmax):
    """Every quartet through the FP32 kernels (cutoff above every bound): the
    per-class FP32 code, whatever its thread mapping, agrees with the oracle
    to FP32 accuracy (an indexing slip would be an O(1) error)."""
    mol = molgen.random_molecule(500 + seed, natom, shells, 1, kmax, 0.05, 5e3, layout="lattice", spacing=2.2)
    D = molgen.density(mol, 600 + seed)
    old = g.get_option("mixed_tau")
    g.set_option("mixed_tau", 1e300)
    try:
        pairs, J, K, E = _run(g, mol, D, None, "mixed")
        n32, n64 = g.last_split(pairs)
    finally:
        g.set_option("mixed_tau", old)
    assert n64 == 0 and n32 == pairs.nquartets
    Jo, Ko, _ = oracle.jk(mol, D, mode="unique")
    assert np.abs(J - Jo).max() <= 2e-6 * np.abs(Jo).max(), np.abs(J - Jo).max() / np.abs(Jo).max()
    assert np.abs(K - Ko).max() <= 2e-6 * np.abs(Ko).max(), np.abs(K - Ko).max() / np.abs(Ko).max()


@pytest.mark.parametrize("seed,shells,natom,kmax", [(44, [0, 1, 2], 3, 3), (45, [2, 2, 1], 2, 4)])
def test_double_float_tier(g, seed, shells, natom, kmax):
    """Every quartet through the double-float kernels (cutoff 0: every quartet
    is FP64-selected, and the double-float tier takes them): the oracle's J, K
    and E to FP64-like accuracy, far inside the FP32 kernels' 2e-6; with the
    tier off the same quartets run in FP64 and the two agree to 1e-11."""
    mol = molgen.random_molecule(500 + seed, natom, shells, 1, kmax, 0.05, 5e3, layout="lattice", spacing=2.2)
    D = molgen.density(mol, 600 + seed)
    tau, df, ptau = g.get_option("mixed_tau"), g.get_option("df_tier"), g.get_option("prim_tau")
    g.set_option("mixed_tau", 0.0)
    g.set_option("prim_tau", 0.0)  # every primitive quartet of every quartet in the tier
    try:
        g.set_option("df_tier", 1)
        pairs, J, K, E = _run(g, mol, D, None, "mixed")
        n32, n64 = g.last_split(pairs)
        g.set_option("df_tier", 0)
        _, J64, K64, E64 = _run(g, mol, D, None, "mixed")
    finally:
        g.set_option("mixed_tau", tau)
        g.set_option("df_tier", df)
        g.set_option("prim_tau", ptau)
    assert n32 == 0 and n64 == pairs.nquartets
    Jo, Ko, _ = oracle.jk(mol, D, mode="unique")
    sJ, sK = max(1.0, np.abs(Jo).max()), max(1.0, np.abs(Ko).max())
    assert np.abs(J - Jo).max() <= 1e-11 * sJ, np.abs(J - Jo).max() / sJ
    assert np.abs(K - Ko).max() <= 1e-11 * sK, np.abs(K - Ko).max() / sK
    assert abs(E - oracle.energy(D, Jo, Ko)) <= 1e-11 * max(1.0, abs(E))
    assert np.abs(J - J64).max() <= 1e-11 * sJ and np.abs(K - K64).max() <= 1e-11 * sK


@pytest.mark.parametrize("df", [1, 0])
@pytest.mark.parametrize("seed,shells,natom,kmax", [(46, [0, 1, 2], 3, 4), (47, [2, 1], 3, 3)])
def test_primitive_split(g, df, seed, shells, natom, kmax):
    """The primitive split of the FP64-selected quartets (JK_OPT_PRIM_TAU) with
    every quartet FP64-selected (tau 0): a vanishing cut leaves every primitive
    quartet in the FP64 / double-float tier (the unsplit result); an
    unreachable cut sends every primitive quartet to the FP32 complement (the
    all-FP32 result, to FP32 rounding of the oracle); a cut in between splits
    the work and stays within FP32 rounding of the part below it."""
    mol = molgen.random_molecule(500 + seed, natom, shells, 1, kmax, 0.05, 5e3, layout="lattice", spacing=2.2)
    D = molgen.density(mol, 600 + seed)
    Jo, Ko, _ = oracle.jk(mol, D, mode="unique")
    sJ, sK = max(1.0, np.abs(Jo).max()), max(1.0, np.abs(Ko).max())
    old = {k: g.get_option(k) for k in ("mixed_tau", "df_tier", "prim_tau")}
    res = {}
    try:
        g.set_option("mixed_tau", 0.0)
        g.set_option("df_tier", df)
        for ptau in (0.0, 1e-300, 1e300, 1e-3):
            g.set_option("prim_tau", ptau)
            pairs, J, K, E = _run(g, mol, D, None, "mixed")
            st = g.split_stats(pairs)
            res[ptau] = (J, K, sum(s["fp64"]["nprimq"] for s in st), sum(s["fp32"]["nprimq"] for s in st))
    finally:
        for k, v in old.items():
            g.set_option(k, v)
    J0, K0, p64, p32 = res[0.0]
    assert p32 == 0 and p64 == pairs.nprimquartets
    J, K, q64, q32 = res[1e-300]
    assert (q64, q32) == (p64, 0)
    assert np.abs(J - J0).max() <= 1e-12 * sJ and np.abs(K - K0).max() <= 1e-12 * sK
    J, K, q64, q32 = res[1e300]
    assert (q64, q32) == (0, p64)
    assert np.abs(J - Jo).max() <= 2e-6 * np.abs(Jo).max() and np.abs(K - Ko).max() <= 2e-6 * np.abs(Ko).max()
    J, K, q64, q32 = res[1e-3]
    assert q64 > 0 and q32 > 0 and q64 + q32 == p64
    assert np.abs(J - Jo).max() <= 2e-6 * sJ and np.abs(K - Ko).max() <= 2e-6 * sK
