"""Pins for the oracle's J/K, energy and screening (the Fock two-electron
build of Sec. 2.1 and the atomic J/K reduction of Sec. 6)."""
import json
import os

import numpy as np
import pytest

import molgen
import oracle
import oracle.scf as scf

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _mol(seed, shells, natom=3, kmax=2):
    return molgen.random_molecule(seed, natom, shells, 1, kmax, 0.15, 8.0, layout="cube", box=4.0, min_spacing=1.2)


def test_all_vs_unique_bookkeeping():
    # every quartet (the definition) vs unique quartets with explicit images
    mol = _mol(21, [0, 1, 2])
    D = molgen.density(mol, 5)
    J0, K0, n0 = oracle.jk(mol, D, mode="all")
    J1, K1, n1 = oracle.jk(mol, D, mode="unique")
    S = mol.nshell
    P = S * (S + 1) // 2
    assert n0 == S ** 4 and n1 == P * (P + 1) // 2
    assert np.abs(J0 - J1).max() < 1e-12 * np.abs(J0).max()
    assert np.abs(K0 - K1).max() < 1e-12 * np.abs(K0).max()


def test_jk_against_full_tensor():
    mol = _mol(22, [0, 1, 3], natom=2)
    D = molgen.density(mol, 6)
    I = oracle.eri_full(mol)
    J, K, _ = oracle.jk(mol, D, mode="unique")
    assert np.allclose(J, np.einsum("mnls,ls->mn", I, D), rtol=0, atol=1e-12 * np.abs(J).max())
    assert np.allclose(K, np.einsum("mlns,ls->mn", I, D), rtol=0, atol=1e-12 * np.abs(K).max())


def test_invariants_config0():
    mol, D = molgen.config(0)
    J, K, _ = oracle.jk(mol, D, mode="all")
    assert np.abs(J - J.T).max() < 1e-13 * np.abs(J).max()
    assert np.abs(K - K.T).max() < 1e-13 * np.abs(K).max()
    # PSD density + positive-definite Coulomb metric
    assert np.sum(D * J) > 0 and np.sum(D * K) > 0
    # E_J >= E_K/2 for PSD D (Cauchy-Schwarz in the Coulomb metric)
    assert 0.5 * np.sum(D * J) >= 0.25 * np.sum(D * K)
    # translating the molecule leaves J and K unchanged
    Jt, Kt, _ = oracle.jk(mol.translated([0.37, -1.1, 2.3]), D, mode="unique")
    assert np.abs(J - Jt).max() < 1e-12 * np.abs(J).max()
    assert np.abs(K - Kt).max() < 1e-12 * np.abs(K).max()


def test_rows_match_full_build():
    mol = _mol(23, [0, 1, 2], natom=3)
    D = molgen.density(mol, 7)
    J, K, _ = oracle.jk(mol, D, mode="unique")
    rows = [0, 4, mol.nshell - 1]
    Jr, Kr = oracle.jk_rows(mol, D, rows)
    idx = oracle.bf_shell_rows(mol, rows)
    assert np.abs(Jr - J[idx]).max() < 1e-12 * np.abs(J).max()
    assert np.abs(Kr - K[idx]).max() < 1e-12 * np.abs(K).max()


def test_screening_bound():
    # dropping quartets with Q_ab Q_cd < thresh changes each J/K element by at
    # most (number of dropped quartet images) * thresh * max|D|
    mol = molgen.random_molecule(31, 6, [0, 1, 2], 1, 3, 0.3, 30.0, layout="lattice", spacing=3.5)
    D = molgen.density(mol, 8)
    J0, K0, n0 = oracle.jk(mol, D, mode="unique")
    thresh = 1e-6
    J1, K1, n1 = oracle.jk(mol, D, thresh=thresh, mode="unique")
    assert n1 < n0
    nbf = mol.nbf
    bound = (n0 - n1) * 8 * 100 * thresh * np.abs(D).max()
    assert np.abs(J0 - J1).max() <= bound and np.abs(K0 - K1).max() <= bound
    assert np.abs(J0 - J1).max() > 0


def test_h2_sto3g_textbook():
    g = json.load(open(os.path.join(GOLD, "h2_sto3g.json")))
    tol = 0.5 * 10 ** -g["printed_decimals"] + 1e-12
    mol = molgen.h2_sto3g(g["R_bohr"])
    S, T, V = scf.one_electron(mol)
    assert abs(S[0, 1] - g["S12"]) <= tol
    assert abs(T[0, 0] - g["T11"]) <= tol and abs(T[0, 1] - g["T12"]) <= tol
    assert abs(V[0, 0] - g["V11_total"]) <= tol and abs(V[0, 1] - g["V12_total"]) <= tol
    I = oracle.eri_full(mol)
    assert abs(I[0, 0, 0, 0] - g["eri_1111"]) <= tol
    assert abs(I[0, 0, 1, 1] - g["eri_1122"]) <= tol
    assert abs(I[1, 0, 0, 0] - g["eri_2111"]) <= tol
    assert abs(I[1, 0, 1, 0] - g["eri_2121"]) <= tol
    E, Eel, P = scf.rhf(mol, nocc=1)
    assert abs(Eel - g["E_electronic"]) <= tol
    assert abs(E - g["E_total"]) <= tol
    # the energy expression used for the workloads, E2 = tr(PJ)/2 - tr(PK)/4,
    # is the two-electron part of that SCF energy
    J, K, _ = oracle.jk(mol, P, mode="all")
    H = S * 0 + T + V
    assert abs(oracle.energy(P, J, K) + float(np.sum(P * H)) - Eel) < 1e-12


def test_extended_precision_rows():
    """The long-double J/K rows (the extended-precision reference the full-size
    FP64 parity was checked against) agree with the FP64 rows and with the
    FP64 all-quartet build to FP64 rounding on a small molecule, for s, p and
    d rows; a wrong conversion or truncated type in the templated path would
    show here."""
    mol = _mol(25, [0, 1, 2], natom=3, kmax=3)
    D = molgen.density(mol, 9)
    J, K, _ = oracle.jk(mol, D, mode="all")
    for shells in ([0], [1, 2]):
        rows = oracle.bf_shell_rows(mol, shells)
        Jd, Kd = oracle.jk_rows(mol, D, shells)
        Jl, Kl = oracle.jk_rows(mol, D, shells, extended=True)
        for X, Y in ((Jl, Jd), (Kl, Kd), (Jl, J[rows]), (Kl, K[rows])):
            assert np.abs(X - Y).max() <= 1e-13 * np.abs(Y).max()


def test_extended_precision_unique_build():
    """The long-double unique-quartet J/K (what writes the full-size golden
    values) agree with the FP64 unique and all-quartet builds to FP64
    rounding, keep the same quartets, and with the long-double rows."""
    mol = _mol(26, [0, 1, 2], natom=3, kmax=3)
    D = molgen.density(mol, 10)
    J, K, kept = oracle.jk(mol, D, 1e-12, mode="unique")
    Jl, Kl, kept_l = oracle.jk(mol, D, 1e-12, mode="unique", extended=True)
    Ja, Ka, _ = oracle.jk(mol, D, 1e-12, mode="all")
    assert kept_l == kept
    for X, Y in ((Jl, J), (Kl, K), (Jl, Ja), (Kl, Ka)):
        assert np.abs(X - Y).max() <= 1e-13 * np.abs(Y).max()
    assert np.abs(Jl - Jl.T).max() <= 1e-14 * np.abs(Jl).max()
    rows = oracle.bf_shell_rows(mol, [2])
    Jr, Kr = oracle.jk_rows(mol, D, [2], 1e-12, extended=True)
    assert np.abs(Jr - Jl[rows]).max() <= 1e-14 * np.abs(Jl).max()
    assert np.abs(Kr - Kl[rows]).max() <= 1e-14 * np.abs(Kl).max()
