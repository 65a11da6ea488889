"""CPU oracle (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
import this package; the GPU library never does.  It wraps the plain FP64
Obara-Saika/HRR C++ code in ``eri_oracle.cpp`` (built with g++ and OpenMP)
through ctypes, the one-electron integrals (Obara-Saika, any l) in
``one_electron.py``, a small numpy RHF in ``scf.py`` and the pure
(solid-harmonic) d/f transform in ``spherical.py``.

Parity status per function (what pins each one, see the ``-m "not gpu"``
tests): Boys (closed forms, the incomplete-gamma identity, asymptote,
recursion), quartets (closed-form (ss|ss), Gauss-Legendre quadrature of the
1/r12 integral for s/p/d classes, 8-fold symmetry, Schwarz), J/K (all-quartet
vs unique-quartet bookkeeping, symmetry, positivity, translation), energy
(H2 STO-3G textbook value), gradient (central finite differences and
translational invariance), one-electron S, T, V (Gauss-Hermite quadrature,
the first-derivative kinetic form, the Gaussian transform of 1/r, closed s
forms, definiteness), pure shells (harmonicity, definite |m| and
reflection parity, orthonormality, one-centre rotational invariance).  No
function is left unpinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eri_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++ -O2 -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Mol(C.Structure):
    _fields_ = [("natom", C.c_int), ("xyz", C.c_void_p), ("nshell", C.c_int),
                ("atom", C.c_void_p), ("l", C.c_void_p), ("nprim", C.c_void_p),
                ("off", C.c_void_p), ("exps", C.c_void_p), ("coefs", C.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
            lib.orc_boys.argtypes = [C.c_int, C.c_double, dp]
            lib.orc_normalize.argtypes = [C.c_int, ip, ip, ip, dp, dp, dp]
            lib.orc_eri_quartet.argtypes = ([dp, C.c_int, C.c_int, dp, dp] * 4) + [dp]
            lib.orc_eri_quartet.restype = C.c_int
            lib.orc_eri_full.argtypes = [C.POINTER(_Mol), dp]
            lib.orc_schwarz.argtypes = [C.POINTER(_Mol), dp]
            lib.orc_jk.argtypes = [C.POINTER(_Mol), dp, C.c_double, C.c_int, dp, dp]
            lib.orc_jk.restype = C.c_longlong
            lib.orc_jk_ld.argtypes = [C.POINTER(_Mol), dp, C.c_double, C.c_int, dp, dp]
            lib.orc_jk_ld.restype = C.c_longlong
            lib.orc_jk_rows.argtypes = [C.POINTER(_Mol), dp, C.c_double, C.c_int, ip, dp, dp]
            lib.orc_jk_rows.restype = C.c_int
            lib.orc_jk_rows_ld.argtypes = [C.POINTER(_Mol), dp, C.c_double, C.c_int, ip, dp, dp]
            lib.orc_jk_rows_ld.restype = C.c_int
            lib.orc_jk_quartets.argtypes = [C.POINTER(_Mol), dp, C.c_longlong, ip, dp, dp]
            lib.orc_jk_quartets.restype = C.c_longlong
            lib.orc_energy.argtypes = [C.c_int, dp, dp, dp]
            lib.orc_energy.restype = C.c_double
            lib.orc_grad.argtypes = [C.POINTER(_Mol), dp, C.c_double, C.c_int, dp]
            lib.orc_grad.restype = C.c_int
            lib.orc_num_threads.restype = C.c_int
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def boys(mmax: int, T: float) -> np.ndarray:
    """F_m(T), m = 0..mmax."""
    F = np.zeros(mmax + 1)
    _load().orc_boys(int(mmax), float(T), _dp(F))
    return F


def normalize(mol) -> np.ndarray:
    """Normalised contraction coefficients (primitive norm included)."""
    out = np.zeros_like(mol.coefs)
    l, k, o = (np.ascontiguousarray(x, dtype=np.int32) for x in (mol.shell_l, mol.shell_nprim, mol.shell_prim_offset))
    _load().orc_normalize(int(mol.nshell), _ip(l), _ip(k), _ip(o), _dp(np.ascontiguousarray(mol.exps)),
                          _dp(np.ascontiguousarray(mol.coefs)), _dp(out))
    return out


class _MolView:
    """Keeps the numpy buffers alive while the C code reads them."""

    def __init__(self, mol):
        self.xyz = np.ascontiguousarray(mol.xyz, dtype=np.float64)
        self.atom = np.ascontiguousarray(mol.shell_atom, dtype=np.int32)
        self.l = np.ascontiguousarray(mol.shell_l, dtype=np.int32)
        self.nprim = np.ascontiguousarray(mol.shell_nprim, dtype=np.int32)
        self.off = np.ascontiguousarray(mol.shell_prim_offset, dtype=np.int32)
        self.exps = np.ascontiguousarray(mol.exps, dtype=np.float64)
        self.coefs = normalize(mol)
        self.s = _Mol(self.xyz.shape[0], self.xyz.ctypes.data, self.l.shape[0], self.atom.ctypes.data,
                      self.l.ctypes.data, self.nprim.ctypes.data, self.off.ctypes.data,
                      self.exps.ctypes.data, self.coefs.ctypes.data)
        self.nbf = int(mol.nbf)

    def ref(self):
        return C.byref(self.s)


def eri_quartet(shells) -> np.ndarray:
    """One contracted quartet from four explicit shells.

    ``shells`` = four tuples (centre[3], l, exps[k], normalised coefs[k]).
    Returns an array [na, nb, nc, nd]."""
    args, keep, dims = [], [], []
    for R, l, e, c in shells:
        R = np.ascontiguousarray(R, dtype=np.float64)
        e = np.ascontiguousarray(e, dtype=np.float64)
        c = np.ascontiguousarray(c, dtype=np.float64)
        keep += [R, e, c]
        args += [_dp(R), int(l), int(e.shape[0]), _dp(e), _dp(c)]
        dims.append((l + 1) * (l + 2) // 2)
    out = np.zeros(int(np.prod(dims)))
    rc = _load().orc_eri_quartet(*args, _dp(out))
    if rc != 0:
        raise ValueError("unsupported angular momentum")
    return out.reshape(dims)


def eri_full(mol) -> np.ndarray:
    """All (mn|ls) of a small molecule, shape [nbf]*4."""
    v = _MolView(mol)
    out = np.zeros(v.nbf ** 4)
    _load().orc_eri_full(v.ref(), _dp(out))
    return out.reshape((v.nbf,) * 4)


def schwarz(mol) -> np.ndarray:
    """Q[a, b] = sqrt(max_i |(ab|ab)_ii|) over shells."""
    v = _MolView(mol)
    Q = np.zeros((mol.nshell, mol.nshell))
    _load().orc_schwarz(v.ref(), _dp(Q))
    return Q


def jk(mol, D, thresh: float | None = None, mode: str = "unique", extended: bool = False):
    """J, K (and the number of shell quartets kept).  mode "all" loops over
    every quartet; "unique" over a>=b, c>=d, ab>=cd with explicit images.
    ``extended``: every integral and sum in long double (an extended-precision
    reference on x86, where long double has a 64-bit significand), rounded to
    FP64 at the end."""
    v = _MolView(mol)
    D = np.ascontiguousarray(D, dtype=np.float64)
    J = np.zeros_like(D)
    K = np.zeros_like(D)
    fn = _load().orc_jk_ld if extended else _load().orc_jk
    kept = fn(v.ref(), _dp(D), float(thresh or 0.0), 0 if mode == "all" else 1, _dp(J), _dp(K))
    return J, K, int(kept)


def jk_quartets(mol, D, quartets):
    """J/K contributions (all images) of an explicit list of unique shell
    quartets, array [n, 4] of (a, b, c, d) with a>=b, c>=d, ab>=cd."""
    v = _MolView(mol)
    D = np.ascontiguousarray(D, dtype=np.float64)
    q = np.ascontiguousarray(quartets, dtype=np.int32)
    J = np.zeros_like(D)
    K = np.zeros_like(D)
    n = _load().orc_jk_quartets(v.ref(), _dp(D), int(q.shape[0]), _ip(q), _dp(J), _dp(K))
    if n < 0:
        raise ValueError("malformed quartet list")
    return J, K


def sample_unique_quartets(mol, n, seed, thresh=None, Q=None):
    """n random unique shell quartets (a>=b, c>=d, ab>=cd) that pass the
    Schwarz test, drawn uniformly (rejection) with numpy PCG64(seed)."""
    S = mol.nshell
    if thresh and Q is None:
        Q = schwarz(mol)
    rng = np.random.Generator(np.random.PCG64(seed))
    P = S * (S + 1) // 2
    tri_a = np.floor((np.sqrt(8 * np.arange(P) + 1) - 1) / 2).astype(np.int64)
    tri_b = np.arange(P) - tri_a * (tri_a + 1) // 2
    out = []
    while sum(len(o) for o in out) < n:
        ab = rng.integers(0, P, size=4 * n)
        cd = rng.integers(0, P, size=4 * n)
        sw = cd > ab
        ab, cd = np.where(sw, cd, ab), np.where(sw, ab, cd)
        a, b, c, d = tri_a[ab], tri_b[ab], tri_a[cd], tri_b[cd]
        if thresh:
            keep = Q[a, b] * Q[c, d] >= thresh
            a, b, c, d = a[keep], b[keep], c[keep], d[keep]
        out.append(np.stack([a, b, c, d], axis=1))
    return np.concatenate(out)[:n].astype(np.int32)


def jk_rows(mol, D, shells, thresh: float | None = None, extended: bool = False):
    """Rows of J and K for every basis function of the listed shells.
    ``extended``: every integral and sum in long double (an extended-precision
    reference on x86, where long double has a 64-bit significand)."""
    v = _MolView(mol)
    D = np.ascontiguousarray(D, dtype=np.float64)
    shells = np.ascontiguousarray(shells, dtype=np.int32)
    nrow = int(sum((int(mol.shell_l[s]) + 1) * (int(mol.shell_l[s]) + 2) // 2 for s in shells))
    Jr = np.zeros((nrow, v.nbf))
    Kr = np.zeros((nrow, v.nbf))
    fn = _load().orc_jk_rows_ld if extended else _load().orc_jk_rows
    rc = fn(v.ref(), _dp(D), float(thresh or 0.0), int(shells.shape[0]), _ip(shells), _dp(Jr), _dp(Kr))
    if rc != 0:
        raise ValueError("bad row shell")
    return Jr, Kr


def energy(D, J, K) -> float:
    """E = tr(DJ)/2 - tr(DK)/4 (compensated sum)."""
    D, J, K = (np.ascontiguousarray(x, dtype=np.float64) for x in (D, J, K))
    return float(_load().orc_energy(int(D.shape[0]), _dp(D), _dp(J), _dp(K)))


def grad(mol, D, thresh: float | None = None, mode: str = "unique") -> np.ndarray:
    """dE/dR [natom, 3] for E = tr(DJ)/2 - tr(DK)/4 at fixed D."""
    v = _MolView(mol)
    D = np.ascontiguousarray(D, dtype=np.float64)
    g = np.zeros((mol.natom, 3))
    _load().orc_grad(v.ref(), _dp(D), float(thresh or 0.0), 0 if mode == "all" else 1, _dp(g))
    return g


def bf_shell_rows(mol, shells):
    """Basis-function indices covered by the listed shells (row order of jk_rows)."""
    off = mol.shell_offsets()
    out = []
    for s in shells:
        n = (int(mol.shell_l[s]) + 1) * (int(mol.shell_l[s]) + 2) // 2
        out += list(range(int(off[s]), int(off[s]) + n))
    return np.array(out, dtype=np.int64)
