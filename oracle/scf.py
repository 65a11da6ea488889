"""Closed-shell Hartree-Fock (test infrastructure).

Pins the oracle's integrals and J/K to the textbook H2 / STO-3G worked
example (R = 1.4 bohr), and is the reference SCF for the GPU driver: the SCF
structure the paper describes in Sec. 2.1 -- build the Fock matrix from the
current orbitals, form the density, evaluate the energy, repeat until the
density is stable.  Plain Roothaan iterations with symmetric orthogonalisation
X = S^(-1/2); the one-electron integrals come from one_electron.py.
"""
from __future__ import annotations

import numpy as np

from . import jk
from .one_electron import one_electron  # noqa: F401  (re-exported)


def nuclear_repulsion(mol) -> float:
    e = 0.0
    for i in range(mol.natom):
        for j in range(i):
            e += mol.charges[i] * mol.charges[j] / np.linalg.norm(mol.xyz[i] - mol.xyz[j])
    return e


def rhf(mol, nocc: int, tol: float = 1e-10, maxiter: int = 99, pure: bool = False):
    """Returns (E_total, E_electronic, P) with P the total density.  With
    `pure`, in the basis of pure d and f shells: S and H transformed by the
    Cartesian-to-pure matrix, J and K from the pure-basis integrals
    (spherical.jk_pure: every tensor index transformed)."""
    S, T, V = one_electron(mol)
    H = T + V
    if pure:
        from . import spherical
        Tm = spherical.transform_matrix(mol)
        S, H = Tm.T @ S @ Tm, Tm.T @ H @ Tm

        def jkf(P):
            return spherical.jk_pure(mol, P)
    else:
        def jkf(P):
            return jk(mol, P, mode="all")[:2]
    w, U = np.linalg.eigh(S)
    X = U @ np.diag(w ** -0.5) @ U.T
    P = np.zeros_like(S)
    e_old = 0.0
    for _ in range(maxiter):
        J, K = jkf(P)
        F = H + J - 0.5 * K
        e, Cp = np.linalg.eigh(X.T @ F @ X)
        Cmo = X @ Cp
        Pn = 2.0 * Cmo[:, :nocc] @ Cmo[:, :nocc].T
        Jn, Kn = jkf(Pn)
        e_el = 0.5 * float(np.sum(Pn * (H + H + Jn - 0.5 * Kn)))
        if abs(e_el - e_old) < tol and np.abs(Pn - P).max() < 1e-8:
            P = Pn
            break
        P, e_old = Pn, e_el
    J, K = jkf(P)
    e_el = 0.5 * float(np.sum(P * (2.0 * H + J - 0.5 * K)))
    return e_el + nuclear_repulsion(mol), e_el, P
