"""One-electron integrals over contracted Cartesian Gaussian shells, for the
oracle's SCF (test infrastructure only).

The SCF structure of Sec. 2.1 needs, besides J and K, the overlap S, the
kinetic energy T and the nuclear attraction V.  The oracle evaluates them with
the Obara-Saika recursions (the family Sec. 2.2 describes), in plain FP64
Python, one primitive pair at a time:

  1-D overlap   S_00 = sqrt(pi/p) exp(-mu X_AB^2),
                S_(i+1)j = X_PA S_ij + (i S_(i-1)j + j S_i(j-1)) / 2p,
                S_i(j+1) = X_PB S_ij + (i S_(i-1)j + j S_i(j-1)) / 2p;
  kinetic       -1/2 d^2/dx^2 acting on the ket:
                T_ij = -1/2 [ j(j-1) S_i(j-2) - 2b(2j+1) S_ij + 4b^2 S_i(j+2) ],
                T = Tx Sy Sz + Sx Ty Sz + Sx Sy Tz;
  nuclear       Theta^(m)_00 = (2 pi / p) K_AB F_m(p |P-C|^2), and on the bra
                Theta^(m)_(a+1_i) = X_PA,i Theta^(m)_a - X_PC,i Theta^(m+1)_a
                    + a_i/2p (Theta^(m)_(a-1_i) - Theta^(m+1)_(a-1_i)),
                then the horizontal transfer (a|b+1_i) = (a+1_i|b) + X_AB,i (a|b);
                V = -sum_C Z_C Theta^(0).

Normalisation and component order as the rest of the oracle (axial, lx then
ly descending).  Parity status: pinned (tests/test_oracle_one_electron.py) by
Gauss-Hermite quadrature of S, T and of V through the Gaussian transform of
1/r, the closed s-shell forms, symmetry and definiteness, and the H2 STO-3G
textbook values.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

from . import boys, normalize


def cart_components(l):
    return [(lx, l - lx - lz, lz) for lx in range(l, -1, -1) for lz in range(0, l - lx + 1)]


def _overlap_1d(la, lb, PA, PB, p, s00):
    """S[i][j] for i <= la, j <= lb (one axis)."""
    S = np.zeros((la + 1, lb + 1))
    S[0, 0] = s00
    for i in range(la + 1):
        for j in range(lb + 1):
            if i == 0 and j == 0:
                continue
            if i > 0:
                v = PA * S[i - 1, j]
                if i > 1:
                    v += (i - 1) * S[i - 2, j] / (2 * p)
                if j > 0:
                    v += j * S[i - 1, j - 1] / (2 * p)
            else:
                v = PB * S[i, j - 1]
                if j > 1:
                    v += (j - 1) * S[i, j - 2] / (2 * p)
            S[i, j] = v
    return S


def _nuclear_prim(la, lb, A, B, a, b, C):
    """Theta^(0) over all component pairs of one primitive pair and one
    nucleus at C (without the charge), array [ncart(la), ncart(lb)]."""
    p = a + b
    P = (a * A + b * B) / p
    mu = a * b / p
    AB = A - B
    K = math.exp(-mu * float(AB @ AB))
    PA, PC = P - A, P - C
    L = la + lb
    F = boys(L, p * float(PC @ PC))
    base = [2.0 * math.pi / p * K * F[m] for m in range(L + 1)]

    @lru_cache(maxsize=None)
    def vrr(e, m):
        # (e|0)^(m) on the bra, e a tuple (ex, ey, ez)
        if min(e) < 0:
            return 0.0
        if e == (0, 0, 0):
            return base[m]
        i = next(k for k in range(3) if e[k] > 0)
        em = list(e)
        em[i] -= 1
        em = tuple(em)
        v = PA[i] * vrr(em, m) - PC[i] * vrr(em, m + 1)
        if em[i] > 0:
            emm = list(em)
            emm[i] -= 1
            emm = tuple(emm)
            v += em[i] / (2 * p) * (vrr(emm, m) - vrr(emm, m + 1))
        return v

    @lru_cache(maxsize=None)
    def hrr(ea, eb):
        if min(eb) < 0:
            return 0.0
        if eb == (0, 0, 0):
            return vrr(ea, 0)
        i = next(k for k in range(3) if eb[k] > 0)
        ebm = list(eb)
        ebm[i] -= 1
        eap = list(ea)
        eap[i] += 1
        return hrr(tuple(eap), tuple(ebm)) + AB[i] * hrr(ea, tuple(ebm))

    ca, cb = cart_components(la), cart_components(lb)
    return np.array([[hrr(x, y) for y in cb] for x in ca])


def one_electron(mol):
    """S, T, V [nbf, nbf] (V needs mol.charges)."""
    c = normalize(mol)
    off = mol.shell_offsets()
    n = mol.nbf
    S = np.zeros((n, n))
    T = np.zeros((n, n))
    V = np.zeros((n, n))
    Z = None if mol.charges is None else np.asarray(mol.charges, dtype=np.float64)
    for sa in range(mol.nshell):
        la, A = int(mol.shell_l[sa]), mol.xyz[mol.shell_atom[sa]]
        ca = cart_components(la)
        for sb in range(mol.nshell):
            lb, B = int(mol.shell_l[sb]), mol.xyz[mol.shell_atom[sb]]
            cb = cart_components(lb)
            blk = np.s_[off[sa]:off[sa] + len(ca), off[sb]:off[sb] + len(cb)]
            for u in range(mol.shell_nprim[sa]):
                a = mol.exps[mol.shell_prim_offset[sa] + u]
                wa = c[mol.shell_prim_offset[sa] + u]
                for v in range(mol.shell_nprim[sb]):
                    b = mol.exps[mol.shell_prim_offset[sb] + v]
                    w = wa * c[mol.shell_prim_offset[sb] + v]
                    p = a + b
                    P = (a * A + b * B) / p
                    mu = a * b / p
                    s1 = [_overlap_1d(la, lb + 2, P[k] - A[k], P[k] - B[k], p,
                                      math.sqrt(math.pi / p) * math.exp(-mu * (A[k] - B[k]) ** 2)) for k in range(3)]
                    t1 = []
                    for k in range(3):
                        s = s1[k]
                        t = np.zeros((la + 1, lb + 1))
                        for i in range(la + 1):
                            for j in range(lb + 1):
                                t[i, j] = -0.5 * ((j * (j - 1) * s[i, j - 2] if j >= 2 else 0.0)
                                                  - 2 * b * (2 * j + 1) * s[i, j] + 4 * b * b * s[i, j + 2])
                        t1.append(t)
                    for x, ex in enumerate(ca):
                        for y, ey in enumerate(cb):
                            sx, sy, sz = (s1[k][ex[k], ey[k]] for k in range(3))
                            tx, ty, tz = (t1[k][ex[k], ey[k]] for k in range(3))
                            S[blk][x, y] += w * sx * sy * sz
                            T[blk][x, y] += w * (tx * sy * sz + sx * ty * sz + sx * sy * tz)
                    if Z is not None:
                        for Cn, z in zip(mol.xyz, Z):
                            V[blk] -= w * z * _nuclear_prim(la, lb, A, B, a, b, Cn)
    return S, T, V
