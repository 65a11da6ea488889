"""Pins for the oracle's contracted ERIs (Eq. 2 "contraction", evaluated by
Obara-Saika + HRR as in Sec. 2.2).

* closed-form (ss|ss) and two special cases of it;
* brute-force quadrature: 1/r12 = 2/sqrt(pi) int_0^inf exp(-t^2 r12^2) dt makes
  the six-dimensional integrand Gaussian for every t; the remaining t
  integral is done by Gauss-Legendre, and p, d, f primitives are centre
  derivatives of s primitives (differentiated symbolically with sympy), so
  none of this shares a step with the recurrences;
* the 8-fold permutational symmetry and the Schwarz inequality.
"""
import itertools
import math

import numpy as np
import pytest
import sympy as sp

import molgen
import oracle


def comps(l):
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def test_ss_closed_form_one_primitive():
    rng = np.random.default_rng(7)
    for _ in range(20):
        R = rng.uniform(-2, 2, size=(4, 3))
        e = np.exp(rng.uniform(np.log(0.1), np.log(20), size=4))
        v = oracle.eri_quartet([(R[i], 0, [e[i]], [1.0]) for i in range(4)])[0, 0, 0, 0]
        a, b, c, d = e
        p, q = a + b, c + d
        P = (a * R[0] + b * R[1]) / p
        Q = (c * R[2] + d * R[3]) / q
        Kab = math.exp(-a * b / p * np.sum((R[0] - R[1]) ** 2))
        Kcd = math.exp(-c * d / q * np.sum((R[2] - R[3]) ** 2))
        T = p * q / (p + q) * np.sum((P - Q) ** 2)
        F0 = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T)) if T > 0 else 1.0
        ref = 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * Kab * Kcd * F0
        assert abs(v - ref) <= 1e-14 * abs(ref)


def test_ss_self_repulsion():
    # four identical normalised s functions on one centre: (ss|ss) = 2 sqrt(alpha/pi)
    for alpha in (0.3, 1.0, 7.5):
        N = (2 * alpha / math.pi) ** 0.75
        v = oracle.eri_quartet([(np.zeros(3), 0, [alpha], [N])] * 4)[0, 0, 0, 0]
        assert abs(v - 2 * math.sqrt(alpha / math.pi)) < 1e-14
    # exponent alpha on electron 1, beta on electron 2 (same centre): two unit
    # Gaussian charges of exponents 2 alpha and 2 beta repel with
    # 2/sqrt(pi) sqrt(a1 a2 / (a1 + a2)) = 2/sqrt(pi) sqrt(2 alpha beta / (alpha + beta))
    a, b = 0.8, 2.3
    Na, Nb = (2 * a / math.pi) ** 0.75, (2 * b / math.pi) ** 0.75
    v = oracle.eri_quartet([(np.zeros(3), 0, [a], [Na])] * 2 + [(np.zeros(3), 0, [b], [Nb])] * 2)[0, 0, 0, 0]
    ref = 2.0 / math.sqrt(math.pi) * math.sqrt(2 * a * b / (a + b))
    assert abs(v - ref) < 1e-14


# ---------------------------------------------------------------- quadrature
_SYM = None


def _symbols():
    global _SYM
    if _SYM is None:
        t = sp.Symbol("t", positive=True)
        e = sp.symbols("a b c d", positive=True)
        R = [sp.symbols(f"{n}x {n}y {n}z", real=True) for n in "ABCD"]
        a, b, c, d = e
        p, q = a + b, c + d
        AB2 = sum((R[0][i] - R[1][i]) ** 2 for i in range(3))
        CD2 = sum((R[2][i] - R[3][i]) ** 2 for i in range(3))
        P = [(a * R[0][i] + b * R[1][i]) / p for i in range(3)]
        Q = [(c * R[2][i] + d * R[3][i]) / q for i in range(3)]
        PQ2 = sum((P[i] - Q[i]) ** 2 for i in range(3))
        det = p * q + t ** 2 * (p + q)
        # 2/sqrt(pi) * int dr1 dr2 exp(-a rA^2 - b rB^2 - t^2 r12^2 - c rC^2 - d rD^2)
        f = 2 / sp.sqrt(sp.pi) * sp.exp(-a * b / p * AB2 - c * d / q * CD2) * sp.pi ** 3 * det ** sp.Rational(-3, 2) \
            * sp.exp(-p * q * t ** 2 * PQ2 / det)
        _SYM = (t, e, R, f)
    return _SYM


def _poly_op(expr, Rs, alpha, comp):
    """Turn an s primitive into x^lx y^ly z^lz times it by centre derivatives:
    x_A^n g = sum_k coef_k d^k g / dA_x^k with
    n=1: d/(2a);  n=2: (d^2 + 2a)/(4a^2);  n=3: (d^3 + 6a d)/(8a^3)."""
    for axis, n in enumerate(comp):
        X = Rs[axis]
        if n == 0:
            continue
        if n == 1:
            expr = sp.diff(expr, X) / (2 * alpha)
        elif n == 2:
            expr = (sp.diff(expr, X, 2) + 2 * alpha * expr) / (4 * alpha ** 2)
        elif n == 3:
            expr = (sp.diff(expr, X, 3) + 6 * alpha * sp.diff(expr, X)) / (8 * alpha ** 3)
        else:
            raise ValueError(n)
    return expr


def _quad_value(ls, cs, R, ex):
    t, e, Rs, f = _symbols()
    expr = f
    for i in range(4):
        expr = _poly_op(expr, Rs[i], e[i], cs[i])
    subs = {e[i]: ex[i] for i in range(4)}
    for i in range(4):
        for k in range(3):
            subs[Rs[i][k]] = R[i][k]
    g = sp.lambdify(t, expr.subs(subs), "numpy")
    # t = u / (1 - u), Gauss-Legendre on u in (0, 1)
    x, w = np.polynomial.legendre.leggauss(400)
    u = 0.5 * (x + 1)
    w = 0.5 * w
    tv = u / (1 - u)
    return float(np.sum(w * np.asarray(g(tv), dtype=float) / (1 - u) ** 2))


QUAD_CASES = [
    ((0, 0, 0, 0), None),
    ((1, 0, 0, 0), None), ((0, 1, 0, 0), None), ((0, 0, 1, 0), None), ((0, 0, 0, 1), None),
    ((1, 1, 0, 0), None), ((1, 0, 1, 0), None), ((1, 0, 0, 1), None),
    ((1, 1, 1, 1), [((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 0, 0)), ((0, 0, 1), (0, 0, 1), (0, 1, 0), (0, 1, 0))]),
    ((2, 0, 0, 0), None), ((0, 2, 0, 0), [((0, 0, 0), (0, 2, 0), (0, 0, 0), (0, 0, 0))]),
    ((2, 1, 0, 0), [((1, 1, 0), (0, 1, 0), (0, 0, 0), (0, 0, 0)), ((2, 0, 0), (1, 0, 0), (0, 0, 0), (0, 0, 0))]),
    ((2, 0, 2, 0), [((1, 0, 1), (0, 0, 0), (0, 1, 1), (0, 0, 0)), ((0, 2, 0), (0, 0, 0), (0, 2, 0), (0, 0, 0))]),
    ((1, 0, 2, 1), [((0, 1, 0), (0, 0, 0), (0, 1, 1), (0, 0, 1))]),
    ((3, 0, 0, 0), [((3, 0, 0), (0, 0, 0), (0, 0, 0), (0, 0, 0)), ((1, 1, 1), (0, 0, 0), (0, 0, 0), (0, 0, 0)),
                    ((0, 2, 1), (0, 0, 0), (0, 0, 0), (0, 0, 0))]),
    ((3, 0, 1, 0), [((1, 2, 0), (0, 0, 0), (0, 1, 0), (0, 0, 0))]),
    ((0, 3, 0, 3), [((0, 0, 0), (2, 0, 1), (0, 0, 0), (0, 1, 2))]),
]


@pytest.mark.parametrize("ls,which", QUAD_CASES)
def test_quadrature(ls, which):
    rng = np.random.default_rng(sum(ls) * 31 + len(QUAD_CASES))
    R = rng.uniform(-1.2, 1.2, size=(4, 3))
    ex = np.exp(rng.uniform(np.log(0.3), np.log(3.0), size=4))
    blk = oracle.eri_quartet([(R[i], ls[i], [ex[i]], [1.0]) for i in range(4)])
    if which is None:
        which = list(itertools.product(*[comps(l) for l in ls]))
    for cs in which:
        idx = tuple(comps(ls[i]).index(tuple(cs[i])) for i in range(4))
        ref = _quad_value(ls, cs, R, ex)
        assert abs(blk[idx] - ref) <= 1e-11 * max(1.0, abs(ref)), (ls, cs, blk[idx], ref)


# ---------------------------------------------------------------- symmetry
def _small_mol(seed, shells, natom=2):
    return molgen.random_molecule(seed, natom, shells, 1, 2, 0.2, 6.0, layout="cube", box=3.0, min_spacing=1.0)


@pytest.mark.parametrize("shells", [[0, 1], [2], [1, 3], [0, 2, 3]])
def test_eightfold_symmetry_and_schwarz(shells):
    mol = _small_mol(11 + len(shells), shells)
    I = oracle.eri_full(mol)
    tol = 1e-12 * np.abs(I).max()   # HRR loses a few digits to (A-B) cancellation
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.abs(I - I.transpose(perm)).max() <= tol
    n = mol.nbf
    M = I.reshape(n * n, n * n)
    diag = np.diag(M)
    assert diag.min() >= -tol                           # (ab|ab) >= 0
    assert np.all(np.abs(M) <= np.sqrt(np.outer(diag, diag)) * (1 + 1e-12) + tol)  # Schwarz
    # the Coulomb metric is positive semi-definite
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() >= -1e-10 * np.abs(M).max()


def test_schwarz_factor_bounds_blocks():
    mol = _small_mol(5, [0, 1, 2], natom=3)
    Q = oracle.schwarz(mol)
    I = oracle.eri_full(mol)
    off = mol.shell_offsets()
    n = [(int(l) + 1) * (int(l) + 2) // 2 for l in mol.shell_l]
    S = mol.nshell
    for a, b, c, d in itertools.product(range(S), repeat=4):
        blk = I[off[a]:off[a] + n[a], off[b]:off[b] + n[b], off[c]:off[c] + n[c], off[d]:off[d] + n[d]]
        assert np.abs(blk).max() <= Q[a, b] * Q[c, d] * (1 + 1e-12) + 1e-15


def test_normalisation_axial_component():
    # the contracted axial component x^l exp(-a r^2) has unit norm; 1-D quadrature per axis
    from scipy import integrate
    mol = molgen.random_molecule(3, 1, [0, 1, 2, 3], 2, 4, 0.1, 30.0)
    c = oracle.normalize(mol)
    for s in range(mol.nshell):
        l, k, o = int(mol.shell_l[s]), int(mol.shell_nprim[s]), int(mol.shell_prim_offset[s])
        e, cc = mol.exps[o:o + k], c[o:o + k]
        tot = 0.0
        for i in range(k):
            for j in range(k):
                p = e[i] + e[j]
                ix = integrate.quad(lambda x: x ** (2 * l) * np.exp(-p * x * x), -np.inf, np.inf, epsabs=0, epsrel=1e-13)[0]
                iy = integrate.quad(lambda x: np.exp(-p * x * x), -np.inf, np.inf, epsabs=0, epsrel=1e-13)[0]
                tot += cc[i] * cc[j] * ix * iy * iy
        assert abs(tot - 1.0) < 1e-10
