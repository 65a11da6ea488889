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


def rhf(mol, nocc: int, tol: float = 1e-10, maxiter: int = 99):
    """Returns (E_total, E_electronic, P) with P the total density."""
    S, T, V = one_electron(mol)
    H = T + V
    w, U = np.linalg.eigh(S)
    X = U @ np.diag(w ** -0.5) @ U.T
    P = np.zeros_like(S)
    e_old = 0.0
    for _ in range(maxiter):
        J, K, _ = jk(mol, P, mode="all")
        F = H + J - 0.5 * K
        e, Cp = np.linalg.eigh(X.T @ F @ X)
        Cmo = X @ Cp
        Pn = 2.0 * Cmo[:, :nocc] @ Cmo[:, :nocc].T
        e_el = 0.5 * float(np.sum(Pn * (H + H + _g(mol, Pn))))
        if abs(e_el - e_old) < tol and np.abs(Pn - P).max() < 1e-8:
            P = Pn
            break
        P, e_old = Pn, e_el
    J, K, _ = jk(mol, P, mode="all")
    e_el = 0.5 * float(np.sum(P * (2.0 * H + J - 0.5 * K)))
    return e_el + nuclear_repulsion(mol), e_el, P


def _g(mol, P):
    J, K, _ = jk(mol, P, mode="all")
    return J - 0.5 * K
