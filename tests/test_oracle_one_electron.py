"""Pins of the oracle's one-electron integrals (oracle/one_electron.py).

Each reference below is computed by a route that shares no step with the
Obara-Saika recursions: Gauss-Hermite quadrature of the separable overlap
integrand (exact for polynomial times Gaussian); the kinetic energy in its
symmetric first-derivative form 1/2 int grad(a) . grad(b) (the recursion uses
the second derivative of the ket); the nuclear attraction through the Gaussian
transform 1/r = 2/sqrt(pi) int_0^inf exp(-t^2 r^2) dt, Gauss-Hermite in space
and Gauss-Legendre in t; the closed forms for s shells; and symmetry and
definiteness."""
import math

import numpy as np
import pytest

import molgen
import oracle
from oracle import one_electron as oe

GH_X, GH_W = np.polynomial.hermite.hermgauss(24)  # exact to polynomial degree 47
GL_X, GL_W = np.polynomial.legendre.leggauss(160)


def _mol(seed, shells, natom=2, charges=True):
    m = molgen.random_molecule(900 + seed, natom, shells, 1, 3, 0.2, 8.0, layout="lattice", spacing=1.6)
    if charges:
        m.charges = np.arange(1, natom + 1, dtype=np.float64) + 0.5
    return m


def _prims(mol):
    """Per shell: centre, l, exponents, normalised coefficients."""
    c = oracle.normalize(mol)
    out = []
    for s in range(mol.nshell):
        o, k = mol.shell_prim_offset[s], mol.shell_nprim[s]
        out.append((mol.xyz[mol.shell_atom[s]], int(mol.shell_l[s]), mol.exps[o:o + k], c[o:o + k]))
    return out


def _axis_factor(ea, eb, Aa, Bb, a, b, t2=0.0, C=0.0, da=False, db=False):
    """int f_a(x) f_b(x) exp(-t2 (x - C)^2) dx for f(x) = (x - X)^e exp(-al (x - X)^2),
    or with f replaced by its first derivative (da / db), by Gauss-Hermite."""
    q = a + b + t2
    Q = (a * Aa + b * Bb + t2 * C) / q
    pref = math.exp(-(a * b * (Aa - Bb) ** 2 + a * t2 * (Aa - C) ** 2 + b * t2 * (Bb - C) ** 2) / q)
    x = Q + GH_X / math.sqrt(q)

    def poly(e, X, al, d):
        y = x - X
        if not d:
            return y ** e
        return (e * y ** (e - 1) if e > 0 else 0.0) - 2.0 * al * y ** (e + 1)

    return pref / math.sqrt(q) * float(np.sum(GH_W * poly(ea, Aa, a, da) * poly(eb, Bb, b, db)))


def _quad_S_T(mol):
    P = _prims(mol)
    off = mol.shell_offsets()
    n = mol.nbf
    S = np.zeros((n, n))
    T = np.zeros((n, n))
    for sa, (A, la, ea_, ca_) in enumerate(P):
        for sb, (B, lb, eb_, cb_) in enumerate(P):
            for x, ex in enumerate(oe.cart_components(la)):
                for y, ey in enumerate(oe.cart_components(lb)):
                    s = t = 0.0
                    for a, ca in zip(ea_, ca_):
                        for b, cb in zip(eb_, cb_):
                            f = [_axis_factor(ex[k], ey[k], A[k], B[k], a, b) for k in range(3)]
                            g = [_axis_factor(ex[k], ey[k], A[k], B[k], a, b, da=True, db=True) for k in range(3)]
                            s += ca * cb * f[0] * f[1] * f[2]
                            t += ca * cb * 0.5 * (g[0] * f[1] * f[2] + f[0] * g[1] * f[2] + f[0] * f[1] * g[2])
                    S[off[sa] + x, off[sb] + y] = s
                    T[off[sa] + x, off[sb] + y] = t
    return S, T


def _quad_V(mol):
    P = _prims(mol)
    off = mol.shell_offsets()
    n = mol.nbf
    V = np.zeros((n, n))
    # t = u / (1 - u), dt = du / (1 - u)^2, u in [0, 1)
    u = 0.5 * (GL_X + 1.0)
    wu = 0.5 * GL_W
    ts = u / (1.0 - u)
    wt = wu / (1.0 - u) ** 2
    for sa, (A, la, ea_, ca_) in enumerate(P):
        for sb, (B, lb, eb_, cb_) in enumerate(P):
            for x, ex in enumerate(oe.cart_components(la)):
                for y, ey in enumerate(oe.cart_components(lb)):
                    v = 0.0
                    for Cn, Z in zip(mol.xyz, mol.charges):
                        for a, ca in zip(ea_, ca_):
                            for b, cb in zip(eb_, cb_):
                                acc = 0.0
                                for t, w in zip(ts, wt):
                                    acc += w * math.prod(_axis_factor(ex[k], ey[k], A[k], B[k], a, b, t * t, Cn[k])
                                                         for k in range(3))
                                v -= Z * ca * cb * 2.0 / math.sqrt(math.pi) * acc
                    V[off[sa] + x, off[sb] + y] = v
    return V


@pytest.mark.parametrize("seed,shells", [(1, [0, 1]), (2, [2, 0]), (3, [3, 1]), (4, [2, 3])])
def test_overlap_and_kinetic_against_quadrature(seed, shells):
    mol = _mol(seed, shells)
    S, T, _ = oe.one_electron(mol)
    Sq, Tq = _quad_S_T(mol)
    np.testing.assert_allclose(S, Sq, rtol=0, atol=1e-12)
    np.testing.assert_allclose(T, Tq, rtol=0, atol=1e-11 * max(1.0, np.abs(Tq).max()))


@pytest.mark.parametrize("seed,shells", [(5, [0, 1]), (6, [2]), (7, [1, 3])])
def test_nuclear_attraction_against_quadrature(seed, shells):
    mol = _mol(seed, shells)
    _, _, V = oe.one_electron(mol)
    Vq = _quad_V(mol)
    np.testing.assert_allclose(V, Vq, rtol=0, atol=1e-9 * max(1.0, np.abs(Vq).max()))


def test_s_shells_closed_forms():
    """S = (pi/p)^(3/2) e^(-mu R^2), T = mu (3 - 2 mu R^2) S, V = -Z 2 pi/p e^(-mu R^2) F_0(p |P-C|^2)
    per primitive pair (textbook forms for s Gaussians)."""
    mol = _mol(8, [0, 0], natom=3)
    S, T, V = oe.one_electron(mol)
    c = oracle.normalize(mol)
    off = mol.shell_offsets()
    for i in range(mol.nshell):
        A = mol.xyz[mol.shell_atom[i]]
        for j in range(mol.nshell):
            B = mol.xyz[mol.shell_atom[j]]
            s = t = v = 0.0
            for u in range(mol.shell_nprim[i]):
                a, ca = mol.exps[mol.shell_prim_offset[i] + u], c[mol.shell_prim_offset[i] + u]
                for w in range(mol.shell_nprim[j]):
                    b, cb = mol.exps[mol.shell_prim_offset[j] + w], c[mol.shell_prim_offset[j] + w]
                    p, mu = a + b, a * b / (a + b)
                    R2 = float((A - B) @ (A - B))
                    s0 = (math.pi / p) ** 1.5 * math.exp(-mu * R2)
                    s += ca * cb * s0
                    t += ca * cb * mu * (3 - 2 * mu * R2) * s0
                    Pc = (a * A + b * B) / p
                    for Cn, Z in zip(mol.xyz, mol.charges):
                        v -= ca * cb * Z * 2 * math.pi / p * math.exp(-mu * R2) * oracle.boys(0, p * float((Pc - Cn) @ (Pc - Cn)))[0]
            assert S[off[i], off[j]] == pytest.approx(s, rel=1e-13, abs=1e-15)
            assert T[off[i], off[j]] == pytest.approx(t, rel=1e-12, abs=1e-14)
            assert V[off[i], off[j]] == pytest.approx(v, rel=1e-12, abs=1e-14)


def test_symmetry_definiteness_normalisation():
    mol = _mol(9, [0, 1, 2, 3])
    S, T, V = oe.one_electron(mol)
    for M in (S, T, V):
        np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-13 * np.abs(M).max())
    assert np.linalg.eigvalsh(S).min() > 0 and np.linalg.eigvalsh(T).min() > 0
    assert np.linalg.eigvalsh(V).max() < 0  # attraction to positive charges
    # the axial components x^l, y^l, z^l of every shell have unit norm
    off = mol.shell_offsets()
    for s, l in enumerate(mol.shell_l):
        comps = oe.cart_components(int(l))
        for ax in range(3):
            e = tuple(int(l) if k == ax else 0 for k in range(3))
            k = off[s] + comps.index(e)
            assert S[k, k] == pytest.approx(1.0, rel=1e-13)
    # translating everything (nuclei included) changes nothing
    m2 = mol.translated([0.7, -1.1, 0.4])
    m2.charges = mol.charges
    for M, M2 in zip((S, T, V), oe.one_electron(m2)):
        np.testing.assert_allclose(M, M2, rtol=0, atol=1e-12 * np.abs(M).max())
