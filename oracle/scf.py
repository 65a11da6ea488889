"""Closed-shell Hartree-Fock for small s-only molecules (test infrastructure).

Used only to pin the oracle's two-electron integrals and J/K to the textbook
H2 / STO-3G worked example (R = 1.4 bohr), the SCF structure the paper
describes in Sec. 2.1: build the Fock matrix from the current orbitals, form
the density, evaluate the energy, repeat until the density is stable.

One-electron integrals use the closed forms for s Gaussians:
  S = (pi/p)^(3/2) exp(-mu R_AB^2)
  T = mu (3 - 2 mu R_AB^2) (pi/p)^(3/2) exp(-mu R_AB^2)
  V = -Z_C 2 pi / p exp(-mu R_AB^2) F_0(p |P - C|^2)
with p = a + b, mu = a b / p, P = (a A + b B) / p.
"""
from __future__ import annotations

import numpy as np

from . import boys, jk, normalize


def one_electron(mol):
    if np.any(mol.shell_l != 0):
        raise ValueError("s shells only")
    c = normalize(mol)
    S = np.zeros((mol.nshell, mol.nshell))
    T = np.zeros_like(S)
    V = np.zeros_like(S)
    for i in range(mol.nshell):
        A = mol.xyz[mol.shell_atom[i]]
        for j in range(mol.nshell):
            B = mol.xyz[mol.shell_atom[j]]
            for u in range(mol.shell_nprim[i]):
                a = mol.exps[mol.shell_prim_offset[i] + u]
                ca = c[mol.shell_prim_offset[i] + u]
                for v in range(mol.shell_nprim[j]):
                    b = mol.exps[mol.shell_prim_offset[j] + v]
                    cb = c[mol.shell_prim_offset[j] + v]
                    p = a + b
                    mu = a * b / p
                    R2 = float(np.dot(A - B, A - B))
                    Kab = np.exp(-mu * R2)
                    P = (a * A + b * B) / p
                    s = (np.pi / p) ** 1.5 * Kab
                    S[i, j] += ca * cb * s
                    T[i, j] += ca * cb * mu * (3.0 - 2.0 * mu * R2) * s
                    for Cn, Z in zip(mol.xyz, mol.charges):
                        PC2 = float(np.dot(P - Cn, P - Cn))
                        V[i, j] += -Z * ca * cb * 2.0 * np.pi / p * Kab * boys(0, p * PC2)[0]
    return S, T, V


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
