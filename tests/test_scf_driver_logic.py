"""Host logic of the GPU SCF driver (paper_2412_13203_gb300/scf.py) on the CPU:
the iteration, DIIS, incremental Fock builds, option handling and the pure-
shell mode, with the driver's library calls replaced inside this test by CPU
stand-ins that compute the same quantities with the oracle.  The GPU path
itself is covered by tests/test_gpu_zscf.py."""
import numpy as np
import pytest

import molgen
import oracle
from oracle import one_electron as oe
from oracle import scf as oscf
from oracle import spherical as sp

torch = pytest.importorskip("torch")


class _Pairs:
    def __init__(self, mol, thresh=None):
        self.mol, self.nbf, self.natom = mol, mol.nbf, mol.natom
        self.nsph = sp.transform_matrix(mol).shape[1]
        S = mol.nshell * (mol.nshell + 1) // 2
        self.nquartets = S * (S + 1) // 2


@pytest.fixture
def drv(monkeypatch):
    from paper_2412_13203_gb300 import scf
    opts = {"density_screen": 0.0, "mixed_tau": 1e-2}
    calls = []

    def one_electron(pairs, charges):
        m = pairs.mol
        m.charges = np.asarray(charges, dtype=np.float64)
        return tuple(torch.from_numpy(x) for x in oe.one_electron(m))

    def jk_build(pairs, D, prec, J=None, K=None):
        calls.append((prec, dict(opts)))
        Jo, Ko, _ = oracle.jk(pairs.mol, D.numpy(), mode="all")
        if J is None:
            return torch.from_numpy(Jo), torch.from_numpy(Ko)
        J.copy_(torch.from_numpy(Jo))
        K.copy_(torch.from_numpy(Ko))
        return J, K

    def sph_transform(pairs, M, direction, out=None):
        T = torch.from_numpy(sp.transform_matrix(pairs.mol))
        r = T @ M @ T.T if direction == "to_cartesian" else T.T @ M @ T
        if out is None:
            return r.contiguous()
        out.copy_(r)
        return out

    monkeypatch.setattr(scf, "ShellPairs", _Pairs)
    monkeypatch.setattr(scf, "one_electron", one_electron)
    monkeypatch.setattr(scf, "jk_build", jk_build)
    monkeypatch.setattr(scf, "sph_transform", sph_transform)
    monkeypatch.setattr(scf, "get_option", lambda k: opts[k])
    monkeypatch.setattr(scf, "set_option", lambda k, v: opts.__setitem__(k, v))
    monkeypatch.setattr(scf, "last_split", lambda p: (0, 7))
    return scf, opts, calls


def test_h2_textbook_and_oracle(drv):
    scf, _, _ = drv
    mol = molgen.h2_sto3g(1.4)
    r = scf.rhf(mol, mol.charges, nocc=1)
    assert r.converged and round(r.energy, 4) == -1.1167
    assert r.energy == pytest.approx(oscf.rhf(mol, 1)[0], abs=1e-12)
    assert r.nuclear_repulsion == pytest.approx(1.0 / 1.4)


@pytest.mark.parametrize("diis", [0, 6])
def test_diis_and_plain_iterations_reach_the_oracle(drv, diis):
    """DIIS starts from the second iteration: the core guess D = 0 commutes
    with every Fock matrix and would otherwise pin the extrapolation."""
    scf, _, _ = drv
    mol = molgen.h2_polarised()
    r = scf.rhf(mol, mol.charges, nocc=1, diis=diis)
    Eo, _, Po = oscf.rhf(mol, 1)
    assert r.converged
    assert r.energy == pytest.approx(Eo, abs=1e-11)
    np.testing.assert_allclose(r.D.numpy(), Po, atol=1e-7)


def test_incremental_builds_and_options(drv):
    scf, opts, calls = drv
    mol = molgen.h_chain(4, 2.0)
    full = scf.rhf(mol, np.ones(4), nocc=2)
    calls.clear()
    inc = scf.rhf(mol, np.ones(4), nocc=2, incremental_eps=1e-10, rebuild=3)
    assert inc.converged and inc.energy == pytest.approx(full.energy, abs=1e-11)
    # full builds at iterations 1, 4, 7, ... and for the final energy; the rest are
    # difference builds with the screen set (tau 0 for an FP64 SCF)
    n = inc.iterations
    kinds = [("diff" if (c[1]["density_screen"] == 1e-10) else "full") for c in calls]
    assert kinds[-1] == "full" and len(kinds) == n + 1
    for it, k in enumerate(kinds[:-1], start=1):
        assert k == ("full" if (it - 1) % 3 == 0 else "diff"), kinds
    assert all(c[0] == "mixed" and c[1]["mixed_tau"] == 0.0 for c in calls if c[1]["density_screen"] > 0)
    assert inc.quartets[0] == _Pairs(mol).nquartets and 7 in inc.quartets
    assert opts == {"density_screen": 0.0, "mixed_tau": 1e-2}  # restored


def test_pure_mode(drv):
    scf, _, _ = drv
    mol = molgen.h2_polarised()
    r = scf.rhf(mol, mol.charges, nocc=1, pure=True)
    Ep, _, Pp = oscf.rhf(mol, 1, pure=True)
    assert r.D.shape == (18, 18)
    assert r.energy == pytest.approx(Ep, abs=1e-11)
    np.testing.assert_allclose(r.D.numpy(), Pp, atol=1e-7)


def test_nuclear_repulsion():
    from paper_2412_13203_gb300 import scf
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 2.0], [0.0, 3.0, 0.0]])
    z = np.array([1.0, 2.0, 3.0])
    want = 1 * 2 / 2.0 + 1 * 3 / 3.0 + 2 * 3 / np.sqrt(13.0)
    assert scf.nuclear_repulsion(xyz, z) == pytest.approx(want, rel=1e-15)
