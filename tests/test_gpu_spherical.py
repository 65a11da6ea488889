"""GPU parity of pure (real solid-harmonic) d/f shells: the Cartesian <-> pure
transform kernel against the oracle's transform matrix, and pure-basis J, K,
energy and gradient against the oracle's pure-basis definitions (through the
C ABI)."""
import numpy as np
import pytest

import molgen
import oracle
from oracle import spherical as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# The coefficients of one pure function sum to at most 4 in magnitude (f, m = 0),
# so a transformed J/K element carries at most 4^2 = 16 times the Cartesian
# elements' rounding.
AMPL = 16.0


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_13203_gb300 as g
    g.load()
    return g


def _mol(seed, shells, natom, kmax=2):
    return molgen.random_molecule(100 + seed, natom, shells, 1, kmax, 0.1, 200.0, layout="lattice", spacing=1.9)


def _pure_density(n, seed, nocc=5):
    """PSD, with T D T^T of the size of the Cartesian tests' densities."""
    C = np.random.default_rng(seed).normal(0, 0.1, (n, nocc))
    return C @ C.T


@pytest.mark.parametrize("seed,shells,natom", [(51, [0, 1, 2, 3], 2), (52, [3, 2, 2, 1], 2), (53, [2], 3)])
def test_transform_matches_oracle(g, seed, shells, natom):
    mol = _mol(seed, shells, natom)
    pairs = g.ShellPairs(mol)
    T = sp.transform_matrix(mol)
    assert (pairs.nbf, pairs.nsph) == T.shape
    rng = np.random.default_rng(seed)
    Dp = rng.normal(size=(pairs.nsph,) * 2)  # not symmetric: checks the orientation
    Mc = rng.normal(size=(pairs.nbf,) * 2)
    Dc = g.sph_transform(pairs, torch.from_numpy(Dp).cuda(), "to_cartesian").cpu().numpy()
    Mp = g.sph_transform(pairs, torch.from_numpy(Mc).cuda(), "to_pure").cpu().numpy()
    np.testing.assert_allclose(Dc, T @ Dp @ T.T, rtol=0, atol=1e-14 * AMPL * np.abs(Dp).max())
    np.testing.assert_allclose(Mp, T.T @ Mc @ T, rtol=0, atol=1e-14 * AMPL * np.abs(Mc).max())


def test_s_and_p_shells_pass_through(g):
    mol = _mol(54, [0, 1, 0], 3)
    pairs = g.ShellPairs(mol)
    assert pairs.nsph == pairs.nbf
    M = torch.from_numpy(np.random.default_rng(1).normal(size=(pairs.nbf,) * 2)).cuda()
    for d in ("to_cartesian", "to_pure"):
        assert torch.equal(g.sph_transform(pairs, M, d), M)
    with pytest.raises(g.JKError) as e:  # in place is refused
        g.sph_transform(pairs, M, "to_pure", out=M)
    assert e.value.code == -1


@pytest.mark.parametrize("seed,shells,natom", [(55, [0, 1, 2, 3], 2), (56, [2, 3, 0], 2)])
def test_pure_jk_fp64(g, seed, shells, natom):
    """J, K and E over pure shells against the oracle's definition (every index
    of the Cartesian ERI tensor transformed, then contracted)."""
    mol = _mol(seed, shells, natom)
    pairs = g.ShellPairs(mol)
    Dp = _pure_density(pairs.nsph, seed)
    Dt = torch.from_numpy(Dp).cuda()
    J, K = g.jk_build_pure(pairs, Dt, "fp64")
    E = g.jk_energy(Dt, J, K)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    Jo, Ko = sp.jk_pure(mol, Dp)
    scale = max(1.0, np.abs(Jo).max())
    assert np.abs(J - Jo).max() <= 1e-10 * AMPL * scale, np.abs(J - Jo).max()
    assert np.abs(K - Ko).max() <= 1e-10 * AMPL * scale, np.abs(K - Ko).max()
    Eo = 0.5 * np.sum(Dp * Jo) - 0.25 * np.sum(Dp * Ko)
    assert abs(E - Eo) <= 1e-10 * AMPL * max(1.0, abs(Eo))


def test_pure_jk_mixed(g):
    mol = molgen.random_molecule(57, 3, [0, 1, 2, 3], 1, 3, 0.05, 1e3, layout="lattice", spacing=2.6)
    pairs = g.ShellPairs(mol, 1e-11)
    Dp = _pure_density(pairs.nsph, 58)
    Dt = torch.from_numpy(Dp).cuda()
    J, K = g.jk_build_pure(pairs, Dt, "mixed")
    E = g.jk_energy(Dt, J, K)
    T = sp.transform_matrix(mol)
    Jc, Kc, _ = oracle.jk(mol, T @ Dp @ T.T, thresh=1e-11, mode="unique")
    Jo, Ko = T.T @ Jc @ T, T.T @ Kc @ T
    assert np.abs(J.cpu().numpy() - Jo).max() <= 1e-6 and np.abs(K.cpu().numpy() - Ko).max() <= 1e-6
    assert abs(E - (0.5 * np.sum(Dp * Jo) - 0.25 * np.sum(Dp * Ko))) <= 1e-6


def test_pure_gradient(g):
    """dE/dR at fixed pure density = the Cartesian gradient at T D T^T (T does
    not depend on the geometry)."""
    mol = molgen.random_molecule(359, 3, [0, 1, 2, 2], 1, 2, 0.1, 50.0, layout="lattice", spacing=1.8)
    pairs = g.ShellPairs(mol)
    Dp = _pure_density(pairs.nsph, 60)
    gg = g.jk_grad_pure(pairs, torch.from_numpy(Dp).cuda(), "fp64").cpu().numpy()
    T = sp.transform_matrix(mol)
    go = oracle.grad(mol, T @ Dp @ T.T, mode="unique")
    scale = max(1.0, np.abs(go).max())
    assert np.abs(gg - go).max() <= 1e-10 * AMPL * scale, (gg, go)
    assert np.abs(gg.sum(axis=0)).max() <= 1e-10 * AMPL * scale
