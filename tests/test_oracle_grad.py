"""Pins for the oracle's nuclear gradient of E = tr(DJ)/2 - tr(DK)/4 at a
fixed density (the adjoint the GPU's gradient kernel computes)."""
import numpy as np
import pytest

import molgen
import oracle


def _energy(mol, D):
    J, K, _ = oracle.jk(mol, D, mode="unique")
    return oracle.energy(D, J, K)


@pytest.mark.parametrize("shells", [[0, 1], [0, 2], [1, 3]])
def test_gradient_finite_difference(shells):
    mol = molgen.random_molecule(41 + len(shells) + sum(shells), 3, shells, 1, 2, 0.2, 6.0,
                                 layout="cube", box=3.5, min_spacing=1.2)
    D = molgen.density(mol, 9)
    g_all = oracle.grad(mol, D, mode="all")
    g_uni = oracle.grad(mol, D, mode="unique")
    assert np.abs(g_all - g_uni).max() < 1e-11 * max(1.0, np.abs(g_all).max())
    # translational invariance: the four centre derivatives are taken independently
    assert np.abs(g_all.sum(axis=0)).max() < 1e-11 * max(1.0, np.abs(g_all).max())
    # 4-point central differences, h = 1e-3 (truncation O(h^4))
    h = 1e-3
    fd = np.zeros_like(g_all)
    for a in range(mol.natom):
        for x in range(3):
            def E(s):
                xyz = mol.xyz.copy()
                xyz[a, x] += s
                return _energy(mol.with_xyz(xyz), D)
            fd[a, x] = (8 * (E(h) - E(-h)) - (E(2 * h) - E(-2 * h))) / (12 * h)
    assert np.abs(fd - g_all).max() < 1e-8 * max(1.0, np.abs(g_all).max()), (fd, g_all)
