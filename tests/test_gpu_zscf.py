"""GPU parity of the one-electron kernel (jk_one_electron) against the
oracle's Obara-Saika S, T, V, and of the SCF driver around jk_build against
the oracle's RHF and the H2 / STO-3G textbook example."""
import json
import os

import numpy as np
import pytest

import molgen
import oracle
from oracle import one_electron as oe
from oracle import scf as oscf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "h2_sto3g.json")


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_13203_gb300 as g
    g.load()
    return g


@pytest.mark.parametrize("seed,shells,natom", [(1, [0, 1], 3), (3, [3, 1], 2), (5, [0, 1, 2, 3], 2)])
def test_one_electron_matches_oracle(g, seed, shells, natom):
    mol = molgen.random_molecule(950 + seed, natom, shells, 1, 3, 0.1, 20.0, layout="lattice", spacing=1.7)
    z = np.arange(1, natom + 1, dtype=np.float64) * 1.5
    mol.charges = z
    pairs = g.ShellPairs(mol)
    S, T, V = (M.cpu().numpy() for M in g.one_electron(pairs, z))
    So, To, Vo = oe.one_electron(mol)
    for M, Mo in ((S, So), (T, To), (V, Vo)):
        np.testing.assert_allclose(M, Mo, rtol=0, atol=1e-12 * np.abs(Mo).max())


def test_one_electron_of_a_screened_handle(g):
    """Elements of pairs the Schwarz threshold drops (Q_ab Q_max < thresh) are
    0; the elements of every kept pair match the oracle."""
    mol = molgen.random_molecule(960, 4, [0, 1], 1, 2, 0.5, 20.0, layout="lattice", spacing=4.0)
    z = np.full(4, 2.0)
    mol.charges = z
    thresh = 1e-6
    Q = oracle.schwarz(mol)
    qq = Q * Q.max()
    assert not np.any(np.abs(qq / thresh - 1.0) < 1e-6)  # no pair on the boundary
    pairs = g.ShellPairs(mol, thresh)
    S_, L_ = mol.nshell, mol.shell_l
    assert pairs.npairs == sum(1 for a in range(S_) for b in range(a + 1) if qq[a, b] >= thresh) < S_ * (S_ + 1) // 2
    off = np.concatenate([mol.shell_offsets(), [mol.nbf]])
    kept = np.zeros((mol.nbf, mol.nbf), bool)
    for a in range(S_):
        for b in range(S_):
            kept[off[a]:off[a + 1], off[b]:off[b + 1]] = qq[a, b] >= thresh
    S, _, V = (M.cpu().numpy() for M in g.one_electron(pairs, z))
    So, _, Vo = oe.one_electron(mol)
    assert (~kept).any()
    np.testing.assert_allclose(S[kept], So[kept], rtol=0, atol=1e-12)
    np.testing.assert_allclose(V[kept], Vo[kept], rtol=0, atol=1e-12 * np.abs(Vo).max())
    np.testing.assert_array_equal(S[~kept], 0.0)
    np.testing.assert_array_equal(V[~kept], 0.0)


def test_scf_h2_sto3g_textbook(g):
    from paper_2412_13203_gb300 import scf
    gold = json.load(open(GOLDEN))
    mol = molgen.h2_sto3g(gold["R_bohr"])
    r = scf.rhf(mol, mol.charges, nocc=1)
    assert r.converged
    assert round(r.energy, 4) == gold["E_total"]
    assert round(r.electronic, 4) == gold["E_electronic"]
    Eo, _, _ = oscf.rhf(mol, 1)
    assert abs(r.energy - Eo) <= 1e-10


@pytest.mark.parametrize("diis", [0, 6])
def test_scf_polarised_h2_matches_oracle(g, diis):
    from paper_2412_13203_gb300 import scf
    mol = molgen.h2_polarised()
    r = scf.rhf(mol, mol.charges, nocc=1, diis=diis)
    assert r.converged
    Eo, _, Po = oscf.rhf(mol, 1)
    assert abs(r.energy - Eo) <= 1e-9
    assert float(np.abs(r.D.cpu().numpy() - Po).max()) <= 1e-6


def test_scf_mixed_precision(g):
    from paper_2412_13203_gb300 import scf
    mol = molgen.h2_polarised(1.5)
    e64 = scf.rhf(mol, mol.charges, nocc=1).energy
    emx = scf.rhf(mol, mol.charges, nocc=1, precision="mixed").energy
    assert abs(emx - e64) <= 1e-6


def test_scf_incremental_density_screening(g):
    """Incremental Fock builds J(D_n) = J(D_m) + J(D_n - D_m) with density
    screening at 1e-10 reach the full SCF's energy while the difference
    builds skip quartets (H6 chain, where distant pairs have small bounds)."""
    from paper_2412_13203_gb300 import scf
    mol = molgen.h_chain(6, 2.0)
    z = np.ones(6)
    tau0 = g.get_option("mixed_tau")
    full = scf.rhf(mol, z, nocc=3)
    inc = scf.rhf(mol, z, nocc=3, incremental_eps=1e-10)
    assert full.converged and inc.converged
    Eo, _, _ = oscf.rhf(mol, 3)
    assert abs(full.energy - Eo) <= 1e-9
    assert abs(inc.energy - full.energy) <= 1e-8
    assert min(inc.quartets) < 0.8 * full.quartets[0]
    assert g.get_option("density_screen") == 0.0 and g.get_option("mixed_tau") == tau0


def test_scf_pure_shells(g):
    """SCF over pure d shells against the oracle's pure-basis RHF (integrals
    with every index transformed)."""
    from paper_2412_13203_gb300 import scf
    mol = molgen.h2_polarised()
    r = scf.rhf(mol, mol.charges, nocc=1, pure=True)
    assert r.converged and r.D.shape == (18, 18)
    Ep, _, Pp = oscf.rhf(mol, 1, pure=True)
    assert abs(r.energy - Ep) <= 1e-9
    assert float(np.abs(r.D.cpu().numpy() - Pp).max()) <= 1e-6
