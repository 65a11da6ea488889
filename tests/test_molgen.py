"""The seeded synthetic workloads: sizes follow the shell recipes, draws are
reproducible, densities are symmetric PSD."""
import numpy as np

import molgen


def test_config_sizes():
    expect = {0: (4, 12, 20), 1: (32, 192, 480), 3: (24, 144, 360), 4: (200, 2000, 7000)}
    for c, (na, ns, nbf) in expect.items():
        mol, D = molgen.config(c)
        assert (mol.natom, mol.nshell, mol.nbf) == (na, ns, nbf)
        assert D.shape == (nbf, nbf)
        assert np.array_equal(D, D.T)


def test_reproducible_and_psd():
    m1, D1 = molgen.config(1)
    m2, D2 = molgen.config(1)
    assert np.array_equal(m1.xyz, m2.xyz) and np.array_equal(m1.exps, m2.exps) and np.array_equal(D1, D2)
    assert np.linalg.eigvalsh(D1).min() > -1e-12
    assert m1.exps.min() >= 0.05 and m1.exps.max() <= 5e3
    assert m1.shell_nprim.min() >= 1 and m1.shell_nprim.max() <= 6
    d = np.linalg.norm(m1.xyz[:, None] - m1.xyz[None], axis=-1) + 10 * np.eye(32)
    assert d.min() > 2.5 * 0.6 - 1e-12


def test_config2_batch():
    b = molgen.config2_batch(8)
    for mol, D in b:
        assert 8 <= mol.natom <= 48 and D.shape == (mol.nbf, mol.nbf)


def test_config0_spacing():
    mol, _ = molgen.config(0)
    d = np.linalg.norm(mol.xyz[:, None] - mol.xyz[None], axis=-1) + 10 * np.eye(4)
    assert d.min() >= 1.8 and mol.xyz.min() >= 0 and mol.xyz.max() <= 6


def test_small_scf_molecules():
    import molgen
    h2 = molgen.h2_polarised()
    assert list(h2.shell_l) == [0, 1, 2, 0, 1, 2] and list(h2.shell_atom) == [0, 0, 0, 1, 1, 1]
    assert h2.nbf == 20 and list(h2.charges) == [1.0, 1.0]
    np.testing.assert_array_equal(h2.exps[:3], molgen.h2_sto3g().exps[:3])
    ch = molgen.h_chain(5, 1.8)
    assert ch.natom == 5 and ch.nbf == 5 * 4 and ch.nshell == 10
    np.testing.assert_allclose(np.diff(ch.xyz[:, 2]), 1.8)
    assert np.all(ch.shell_prim_offset[1:] > ch.shell_prim_offset[:-1])
