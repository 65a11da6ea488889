"""Pins of the oracle's pure (real solid-harmonic) shells.

Each property below is fixed by the mathematics of the solid harmonics, not by
the construction in oracle/spherical.py: a wrong Legendre coefficient, a
swapped cosine/sine type, a wrong sign or a wrong normalisation each fails one
of them."""
import math
from fractions import Fraction

import numpy as np
import pytest

import molgen
import oracle
from oracle import spherical as sp


def _d(p, axis):
    """Partial derivative of an exact polynomial {(a, b, c): coef}."""
    r = {}
    for e, c in p.items():
        if e[axis] == 0:
            continue
        e2 = list(e)
        e2[axis] -= 1
        r[tuple(e2)] = r.get(tuple(e2), 0) + c * e[axis]
    return r


def _add(p, q, s=1):
    r = dict(p)
    for e, c in q.items():
        r[e] = r.get(e, 0) + s * c
    return {e: c for e, c in r.items() if c != 0}


def _mulvar(p, axis):
    r = {}
    for e, c in p.items():
        e2 = list(e)
        e2[axis] += 1
        r[tuple(e2)] = c
    return r


def _lz(p):
    """L_z p = x dp/dy - y dp/dx (without the factor -i)."""
    return _add(_mulvar(_d(p, 1), 0), _mulvar(_d(p, 0), 1), -1)


@pytest.mark.parametrize("l", range(0, 5))
def test_solid_harmonics_are_harmonic(l):
    for m in range(-l, l + 1):
        p = sp.solid_harmonic(l, m)
        assert p, (l, m)
        assert all(sum(e) == l for e in p)  # homogeneous of degree l
        lap = {}
        for axis in range(3):
            lap = _add(lap, _d(_d(p, axis), axis))
        assert lap == {}, (l, m)


@pytest.mark.parametrize("l", range(1, 5))
def test_solid_harmonics_have_definite_m_and_reflection_parity(l):
    for m in range(-l, l + 1):
        p = sp.solid_harmonic(l, m)
        assert _lz(_lz(p)) == {e: -m * m * c for e, c in p.items() if m != 0}, (l, m)
        # sine type (m < 0) is odd under y -> -y, cosine type even
        odd = {e: c for e, c in p.items() if e[1] % 2}
        assert (odd == p) if m < 0 else (odd == {}), (l, m)
        # sign convention: the x^|m| z^(l-|m|) (cosine) or x^(|m|-1) y z^(l-|m|) (sine) term is positive
        am = abs(m)
        lead = (am, 0, l - am) if m >= 0 else (am - 1, 1, l - am)
        assert p[lead] > 0, (l, m)


def _gaussian_metric(l):
    """Overlap of the axially normalised Cartesian components of one shell
    (same centre, same radial part): prod (e_i + e_i' - 1)!! / (2l - 1)!!."""
    def df(n):
        return 1 if n <= 0 else n * df(n - 2)
    comps = sp.cart_components(l)
    G = np.zeros((len(comps), len(comps)))
    for i, a in enumerate(comps):
        for j, b in enumerate(comps):
            s = [a[k] + b[k] for k in range(3)]
            if all(x % 2 == 0 for x in s):
                G[i, j] = df(s[0] - 1) * df(s[1] - 1) * df(s[2] - 1) / df(2 * l - 1)
    return G


@pytest.mark.parametrize("l", range(0, 5))
def test_pure_functions_are_orthonormal(l):
    T = sp.coefficients(l)
    assert T.shape == (molgen.ncart(l), sp.nsph(l))
    np.testing.assert_allclose(T.T @ _gaussian_metric(l) @ T, np.eye(T.shape[1]), atol=1e-14)


def test_d_coefficients_closed_form():
    """The five d functions in the axial convention: sqrt3 xy, sqrt3 yz,
    zz - (xx + yy)/2, sqrt3 xz, sqrt3/2 (xx - yy) (components xx xy xz yy yz zz)."""
    r3 = math.sqrt(3.0)
    want = np.zeros((6, 5))
    want[1, 0] = r3
    want[4, 1] = r3
    want[[0, 3, 5], 2] = [-0.5, -0.5, 1.0]
    want[2, 3] = r3
    want[[0, 3], 4] = [r3 / 2, -r3 / 2]
    np.testing.assert_allclose(sp.coefficients(2), want, atol=1e-15)


def _one_atom(ls, seed=3):
    rng = np.random.default_rng(seed)
    nprim = [2] * len(ls)
    exps = np.concatenate([np.sort(rng.uniform(0.3, 4.0, 2))[::-1] for _ in ls])
    coefs = rng.uniform(0.2, 1.0, exps.shape[0])
    return molgen.Molecule(np.array([[0.3, -0.2, 0.1]]), np.zeros(len(ls), np.int32), np.array(ls, np.int32),
                           np.array(nprim, np.int32), np.arange(0, 2 * len(ls), 2, dtype=np.int32), exps, coefs)


@pytest.mark.parametrize("l", [2, 3])
def test_one_centre_integrals_are_rotationally_invariant(l):
    """On one centre with a spherical charge (ss), (m m'|ss) and (m s|m' s) are
    proportional to delta_mm' with an m-independent constant: the pure
    functions carry one irreducible representation of the rotation group.
    The Cartesian blocks are not diagonal (xx and yy overlap), so the check
    bites on the transform."""
    mol = _one_atom([0, l])
    g = sp.eri_pure(mol)
    n = sp.nsph(l)
    d = slice(1, 1 + n)
    for block in (g[d, d, 0, 0], g[d, 0, d, 0]):
        diag = np.diag(block)
        assert np.ptp(diag) < 1e-13 * abs(diag[0])
        np.testing.assert_allclose(block, diag[0] * np.eye(n), atol=1e-13 * abs(diag[0]))
    gc = oracle.eri_full(mol)
    nc = molgen.ncart(l)
    assert np.max(np.abs(gc[1:1 + nc, 1:1 + nc, 0, 0] - np.diag(np.diag(gc[1:1 + nc, 1:1 + nc, 0, 0])))) > 1e-3


def test_pure_jk_equals_transformed_cartesian_jk():
    """J and K of the pure basis (every tensor index transformed) equal
    T^T J(T D T^T) T and T^T K(T D T^T) T from the Cartesian oracle, and the
    energy is the Cartesian energy of T D T^T."""
    mol = molgen.random_molecule(seed=77, natom=2, shells_per_atom=[0, 1, 2, 3], kmin=1, kmax=2,
                                 alpha_min=0.3, alpha_max=6.0)
    T = sp.transform_matrix(mol)
    rng = np.random.default_rng(5)
    C = rng.normal(0, 0.3, (T.shape[1], 4))
    Dp = C @ C.T
    Jp, Kp = sp.jk_pure(mol, Dp)
    Dc = T @ Dp @ T.T
    Jc, Kc, _ = oracle.jk(mol, Dc, mode="all")
    np.testing.assert_allclose(Jp, T.T @ Jc @ T, atol=1e-11 * np.abs(Jp).max())
    np.testing.assert_allclose(Kp, T.T @ Kc @ T, atol=1e-11 * np.abs(Kp).max())
    np.testing.assert_allclose(Jp, Jp.T, atol=1e-12 * np.abs(Jp).max())
    np.testing.assert_allclose(Kp, Kp.T, atol=1e-12 * np.abs(Kp).max())
    Ep = 0.5 * np.sum(Dp * Jp) - 0.25 * np.sum(Dp * Kp)
    assert Ep == pytest.approx(oracle.energy(Dc, Jc, Kc), rel=1e-12)
    assert np.sum(Dp * Jp) > 0 and np.sum(Dp * Kp) > 0


def test_transform_matrix_layout():
    mol = _one_atom([0, 1, 2, 3, 2])
    T = sp.transform_matrix(mol)
    assert T.shape == (1 + 3 + 6 + 10 + 6, 1 + 3 + 5 + 7 + 5)
    np.testing.assert_array_equal(T[:4, :4], np.eye(4))
    np.testing.assert_allclose(T[4:10, 4:9], sp.coefficients(2))
    np.testing.assert_allclose(T[10:20, 9:16], sp.coefficients(3))
    assert np.count_nonzero(T[4:10, 9:]) == 0 and np.count_nonzero(T[:4, 4:]) == 0


def test_legendre_recursion():
    """Bonnet's recursion (n+1) P_{n+1} = (2n+1) t P_n - n P_{n-1}."""
    for n in range(1, 6):
        lhs = {p: c * (n + 1) for p, c in sp.legendre(n + 1).items()}
        rhs = {p + 1: c * (2 * n + 1) for p, c in sp.legendre(n).items()}
        for p, c in sp.legendre(n - 1).items():
            rhs[p] = rhs.get(p, 0) - n * c
        assert lhs == {p: c for p, c in rhs.items() if c != 0}
    assert sp.legendre(0) == {0: Fraction(1)}


def test_pure_scf_is_variational():
    """The pure functions span a subspace of the Cartesian ones (each d or f
    shell loses its r^2 s or r^2 p combination), so the pure-basis RHF energy
    lies above the Cartesian one; for s and p shells the two are identical."""
    from oracle import scf
    mol = molgen.h2_polarised()
    e_cart, _, _ = scf.rhf(mol, 1)
    e_pure, _, P = scf.rhf(mol, 1, pure=True)
    assert e_cart < e_pure < e_cart + 1e-2
    assert P.shape == (18, 18)
    h2 = molgen.h2_sto3g(1.4)
    assert scf.rhf(h2, 1, pure=True)[0] == pytest.approx(scf.rhf(h2, 1)[0], abs=1e-13)
