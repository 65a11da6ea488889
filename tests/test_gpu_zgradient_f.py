"""GPU parity of the derivative kernels of classes with an f shell (one thread
per work item and ket component) against the oracle's analytic gradient."""
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


@pytest.mark.parametrize("seed,shells,natom,kmax", [(33, [0, 3], 2, 1), (34, [3, 1], 2, 2), (35, [2, 3], 2, 2),
                                                    (36, [0, 1, 2, 3], 2, 2)])
def test_gradient_f_classes(g, seed, shells, natom, kmax):
    mol = molgen.random_molecule(300 + seed, natom, shells, 1, kmax, 0.1, 50.0, layout="lattice", spacing=1.8)
    D = molgen.density(mol, 400 + seed)
    pairs = g.ShellPairs(mol)
    gg = g.jk_grad(pairs, torch.from_numpy(D).cuda(), "fp64").cpu().numpy()
    go = oracle.grad(mol, D, mode="unique")
    scale = max(1.0, np.abs(go).max())
    assert np.abs(gg - go).max() <= 1e-10 * scale, (gg, go)
    assert np.abs(gg.sum(axis=0)).max() <= 1e-10 * scale


def test_pure_gradient_with_f_shells(g):
    """dE/dR at fixed pure density with f shells (the Cartesian gradient at T D T^T)."""
    from oracle import spherical as sp
    mol = molgen.random_molecule(337, 2, [0, 2, 3], 1, 2, 0.1, 50.0, layout="lattice", spacing=1.8)
    pairs = g.ShellPairs(mol)
    C = np.random.default_rng(338).normal(0, 0.1, (pairs.nsph, 5))
    Dp = C @ C.T
    gg = g.jk_grad_pure(pairs, torch.from_numpy(Dp).cuda(), "fp64").cpu().numpy()
    T = sp.transform_matrix(mol)
    go = oracle.grad(mol, T @ Dp @ T.T, mode="unique")
    scale = max(1.0, np.abs(go).max())
    assert np.abs(gg - go).max() <= 1.6e-9 * scale


def test_autograd_pure_with_f_shells(g):
    """jk_energy_fn over pure d/f shells: E, dE/dxyz and dE/dD against the
    oracle's pure-basis J/K and its gradient at T D T^T."""
    from oracle import spherical as sp
    mol = molgen.random_molecule(339, 2, [0, 1, 2, 3], 1, 2, 0.2, 20.0, layout="lattice", spacing=2.0)
    T = sp.transform_matrix(mol)
    C = np.random.default_rng(340).normal(0, 0.1, (T.shape[1], 5))
    Dp = C @ C.T
    xyz = torch.tensor(mol.xyz, dtype=torch.float64, device="cuda", requires_grad=True)
    Dt = torch.tensor(Dp, dtype=torch.float64, device="cuda", requires_grad=True)
    E = g.jk_energy_fn(xyz, Dt, mol, pure=True)
    E.backward()
    Jo, Ko = sp.jk_pure(mol, Dp)
    Eo = 0.5 * np.sum(Dp * Jo) - 0.25 * np.sum(Dp * Ko)
    assert abs(float(E.detach()) - Eo) <= 1.6e-9 * max(1.0, abs(Eo))
    go = oracle.grad(mol, T @ Dp @ T.T, mode="unique")
    assert np.abs(xyz.grad.cpu().numpy() - go).max() <= 1.6e-9 * max(1.0, np.abs(go).max())
    assert np.abs(Dt.grad.cpu().numpy() - (Jo - 0.5 * Ko)).max() <= 1.6e-9 * max(1.0, np.abs(Jo).max())
