"""Pins for the oracle's explicit-list J/K (``oracle.jk_quartets``), the checker
of the density-screened and mixed-precision GPU builds and of the partial
(row-range) builds: the J/K contributions of a list of unique shell quartets,
each added to its eight permutational images (Sec. 2.2, Eq. 2, contracted with
the density into the Fock two-electron terms of Sec. 2.1).

The list helper below enumerates unique quartets (a >= b, c >= d, ab >= cd) by
its own loop; the pins compare against the definition J_mn = sum_ls (mn|ls)
D_ls, K_mn = sum_ls (ml|ns) D_ls over every quartet (``oracle.jk(mode="all")``)
and against the contracted full ERI tensor, so a wrong degeneracy factor, a
dropped or doubled image, or a transposed K index fails here."""
import numpy as np

import molgen
import oracle


def _mol(seed, shells, natom=3, kmax=2):
    return molgen.random_molecule(seed, natom, shells, 1, kmax, 0.15, 8.0, layout="cube", box=4.0, min_spacing=1.2)


def _unique_quartets(S, Q=None, thresh=None):
    out = []
    for a in range(S):
        for b in range(a + 1):
            ab = a * (a + 1) // 2 + b
            for c in range(S):
                for d in range(c + 1):
                    if c * (c + 1) // 2 + d > ab:
                        continue
                    if thresh and Q[a, b] * Q[c, d] < thresh:
                        continue
                    out.append((a, b, c, d))
    return np.array(out, dtype=np.int32)


def _rel(x, ref):
    return float(np.abs(x - ref).max() / np.abs(ref).max())


def test_full_list_equals_definition_l3():
    # s, p, d, f shells on three centres: every degeneracy pattern (a == b,
    # c == d, ab == cd, all distinct) and every class up to (ff|ff)
    mol = _mol(31, [0, 1, 2, 3])
    D = molgen.density(mol, 9)
    q = _unique_quartets(mol.nshell)
    J, K = oracle.jk_quartets(mol, D, q)
    J0, K0, n0 = oracle.jk(mol, D, mode="all")
    assert n0 == mol.nshell ** 4
    assert _rel(J, J0) < 1e-12 and _rel(K, K0) < 1e-12
    # and the contracted ERI tensor itself (no recurrence shared with the list path's bookkeeping)
    I = oracle.eri_full(mol)
    assert _rel(J, np.einsum("mnls,ls->mn", I, D)) < 1e-12
    assert _rel(K, np.einsum("mlns,ls->mn", I, D)) < 1e-12


def test_random_split_sums_to_whole():
    mol = _mol(32, [0, 1, 2])
    D = molgen.density(mol, 10)
    q = _unique_quartets(mol.nshell)
    rng = np.random.Generator(np.random.PCG64(77))
    take = rng.random(len(q)) < 0.37
    J1, K1 = oracle.jk_quartets(mol, D, q[take])
    J2, K2 = oracle.jk_quartets(mol, D, q[~take])
    J, K = oracle.jk_quartets(mol, D, q)
    assert _rel(J1 + J2, J) < 1e-13 and _rel(K1 + K2, K) < 1e-13
    # a partial list is not the whole: both parts carry weight
    assert _rel(J1, J) > 1e-3 and _rel(J2, J) > 1e-3


def test_screened_list_equals_screened_build():
    mol = _mol(33, [0, 1, 2], natom=4, kmax=3)
    D = molgen.density(mol, 11)
    Q = oracle.schwarz(mol)
    thresh = float(np.quantile(np.outer(Q, Q), 0.3))  # drop about a third of the quartets
    q = _unique_quartets(mol.nshell, Q, thresh)
    J, K = oracle.jk_quartets(mol, D, q)
    Ju, Ku, kept = oracle.jk(mol, D, thresh, mode="unique")
    Ja, Ka, _ = oracle.jk(mol, D, thresh, mode="all")
    assert kept == len(q)
    assert _rel(J, Ju) < 1e-13 and _rel(K, Ku) < 1e-13
    assert _rel(J, Ja) < 1e-12 and _rel(K, Ka) < 1e-12


def test_single_quartet_images():
    # one quartet (ab|cd) with a, b, c, d all different: its eight images give
    # J_ab += 2 I D_cd (both orders), J_cd += 2 I D_ab, and the four K blocks
    mol = _mol(34, [0, 1], natom=2)
    D = molgen.density(mol, 12)
    S = mol.nshell
    a, b, c, d = 3, 2, 1, 0
    J, K = oracle.jk_quartets(mol, D, np.array([[a, b, c, d]], dtype=np.int32))
    I = oracle.eri_full(mol)
    off = mol.shell_offsets()
    nl = [(int(l) + 1) * (int(l) + 2) // 2 for l in mol.shell_l]
    sl = [slice(int(off[s]), int(off[s]) + nl[s]) for s in range(S)]
    mask = np.zeros((mol.nbf,) * 4)
    for p, q_, r, t in ((a, b, c, d), (b, a, c, d), (a, b, d, c), (b, a, d, c),
                        (c, d, a, b), (d, c, a, b), (c, d, b, a), (d, c, b, a)):
        mask[sl[p], sl[q_], sl[r], sl[t]] = 1.0
    Im = I * mask
    assert _rel(J, np.einsum("mnls,ls->mn", Im, D)) < 1e-13
    assert _rel(K, np.einsum("mlns,ls->mn", Im, D)) < 1e-13
