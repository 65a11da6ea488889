"""Pure (real solid-harmonic) shells for the oracle (test infrastructure only).

The paper evaluates integrals over Cartesian Gaussians (Sec. 2.2, Eq. 1).
Production basis sets use pure d and f shells: 2l+1 real solid harmonics in
place of the (l+1)(l+2)/2 Cartesian components.  The integrals over the pure
functions are fixed linear combinations of the Cartesian ones, so the oracle
defines them literally: every index of the Cartesian ERI tensor is
transformed, then J and K are contracted in the pure basis.

Construction of the solid harmonics (independent of the library's closed-form
table): for 0 <= m <= l, the associated Legendre part is the m-th derivative
of the Legendre polynomial P_l(t), P_l(t) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k,l)
t^(l-2k); written homogeneously in (x, y, z) (t^j -> z^j r^(l-m-j)) and
multiplied by Re (x+iy)^m (cosine type, m >= 0) or Im (x+iy)^|m| (sine type,
m < 0).  No Condon-Shortley phase, positive overall scale.  Each function is
normalised with the angular moments over the unit sphere,
    int x^a y^b z^c dOmega = 2 G((a+1)/2) G((b+1)/2) G((c+1)/2) / G((a+b+c+3)/2)
(all of a, b, c even; zero otherwise), to the norm of the axial component
x^l: the library normalises contracted Cartesian shells on x^l, so a pure
function then has the norm of a normalised contracted shell.  s and p shells
are not transformed (p stays x, y, z).  Pure components are ordered
m = -l, ..., l.

Parity status: pinned (tests/test_oracle_spherical.py) by harmonicity
(Laplacian zero), definite |m| (eigenfunctions of L_z^2) and reflection
parity, orthonormality under the Gaussian moment metric, and one-centre
rotational invariance of the oracle's own integrals.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def cart_components(l: int):
    """(lx, ly, lz) in the library's order: lx descending, then ly descending."""
    return [(lx, l - lx - lz, lz) for lx in range(l, -1, -1) for lz in range(0, l - lx + 1)]


def nsph(l: int) -> int:
    return 2 * l + 1 if l >= 2 else (l + 1) * (l + 2) // 2


def _poly_mul(p, q):
    r = {}
    for e1, c1 in p.items():
        for e2, c2 in q.items():
            e = (e1[0] + e2[0], e1[1] + e2[1], e1[2] + e2[2])
            r[e] = r.get(e, 0) + c1 * c2
    return {e: c for e, c in r.items() if c != 0}


def _poly_pow(p, n):
    r = {(0, 0, 0): Fraction(1)}
    for _ in range(n):
        r = _poly_mul(r, p)
    return r


def legendre(l: int):
    """Coefficients {power: c} of P_l(t) (explicit sum form)."""
    return {l - 2 * k: Fraction((-1) ** k * math.comb(l, k) * math.comb(2 * l - 2 * k, l), 2 ** l)
            for k in range(l // 2 + 1)}


def solid_harmonic(l: int, m: int):
    """Unnormalised real solid harmonic of degree l, order m, as an exact
    polynomial {(a, b, c): coefficient} in x, y, z."""
    am = abs(m)
    d = legendre(l)
    for _ in range(am):  # m-th derivative in t
        d = {p - 1: c * p for p, c in d.items() if p > 0}
    r2 = {(2, 0, 0): Fraction(1), (0, 2, 0): Fraction(1), (0, 0, 2): Fraction(1)}
    radial = {}
    for j, c in d.items():  # t^j -> z^j r^(l-m-j); l-m-j is even
        k = (l - am - j) // 2
        for e, cc in _poly_pow(r2, k).items():
            e2 = (e[0], e[1], e[2] + j)
            radial[e2] = radial.get(e2, 0) + c * cc
    # (x + iy)^|m| = sum_k C(|m|,k) x^(|m|-k) (iy)^k; i^k is real for even k, imaginary for odd k
    az = {}
    for k in range(am + 1):
        if (m >= 0) == (k % 2 == 0):
            sign = (-1) ** (k // 2)
            az[(am - k, k, 0)] = Fraction(sign * math.comb(am, k))
    return {e: c for e, c in _poly_mul(radial, az).items() if c != 0}


def sphere_moment(a: int, b: int, c: int) -> float:
    """Integral of x^a y^b z^c over the unit sphere."""
    if a % 2 or b % 2 or c % 2:
        return 0.0
    g = math.gamma
    return 2.0 * g((a + 1) / 2) * g((b + 1) / 2) * g((c + 1) / 2) / g((a + b + c + 3) / 2)


def _angular_inner(p, q) -> float:
    return sum(float(c1) * float(c2) * sphere_moment(e1[0] + e2[0], e1[1] + e2[1], e1[2] + e2[2])
               for e1, c1 in p.items() for e2, c2 in q.items())


def coefficients(l: int) -> np.ndarray:
    """T_l [ncart(l), nsph(l)]: pure function m (column, m = -l..l) as a
    combination of the library's normalised Cartesian components (rows).
    Identity for l <= 1."""
    comps = cart_components(l)
    if l <= 1:
        return np.eye(len(comps))
    ref = _angular_inner({(l, 0, 0): 1}, {(l, 0, 0): 1})  # norm^2 of the axial component
    T = np.zeros((len(comps), 2 * l + 1))
    for col, m in enumerate(range(-l, l + 1)):
        p = solid_harmonic(l, m)
        s = math.sqrt(ref / _angular_inner(p, p))
        for e, c in p.items():
            T[comps.index(e), col] = float(c) * s
    return T


def transform_matrix(mol) -> np.ndarray:
    """Block-diagonal T [nbf_cart, nbf_pure] over the shells of `mol`."""
    ls = [int(l) for l in mol.shell_l]
    nc = sum((l + 1) * (l + 2) // 2 for l in ls)
    ns = sum(nsph(l) for l in ls)
    T = np.zeros((nc, ns))
    i = j = 0
    for l in ls:
        t = coefficients(l)
        T[i:i + t.shape[0], j:j + t.shape[1]] = t
        i += t.shape[0]
        j += t.shape[1]
    return T


def eri_pure(mol) -> np.ndarray:
    """(ij|kl) over the pure basis: every index of the oracle's Cartesian
    tensor transformed (small molecules only: O(nbf^4) memory)."""
    from . import eri_full
    T = transform_matrix(mol)
    g = eri_full(mol)
    g = np.einsum("abcd,ai->ibcd", g, T, optimize=True)
    g = np.einsum("ibcd,bj->ijcd", g, T, optimize=True)
    g = np.einsum("ijcd,ck->ijkd", g, T, optimize=True)
    return np.einsum("ijkd,dl->ijkl", g, T, optimize=True)


def jk_pure(mol, D_pure):
    """J_ij = sum_kl (ij|kl) D_kl and K_ij = sum_kl (ik|jl) D_kl in the pure basis."""
    g = eri_pure(mol)
    return np.einsum("ijkl,kl->ij", g, D_pure), np.einsum("ikjl,kl->ij", g, D_pure)
