"""The Cartesian <-> pure transform kernel and its generated coefficient table,
compiled as plain C++ (tests/emu/cuda_runtime.h stands in for CUDA) and run on
the CPU against the oracle's independently built transform matrix.

The kernel source is the library's own csrc/sph_transform.cuh and the table is
what codegen/sph_codegen.py emits for the build; the shell records are laid out
as the runtime lays them out.  Test infrastructure only."""
import ctypes as C
import hashlib
import os
import subprocess
import sys

import numpy as np
import pytest

import molgen
from oracle import spherical as sp

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2412_13203_gb300", "csrc")
BUILD = os.path.join(HERE, "_emu_build", "sph")

DRIVER = r"""
#include "sph_transform.cuh"
emu_dim3 blockIdx, threadIdx, blockDim, gridDim;
extern "C" int gb_sph_table(const double** coef, const int** off);
extern "C" int emu_table(const double** coef, const int** off) { return gb_sph_table(coef, off); }
// one emulated thread walks the grid-stride loop over every output element
extern "C" void emu_sph(const double* in, double* out, int n_in, int n_out, int dir, const int* owner,
                        const int* shell4, const double* coef) {
    gb::SphArgs a;
    a.in = in; a.out = out; a.n_in = n_in; a.n_out = n_out; a.dir = dir;
    a.owner = owner; a.shell = reinterpret_cast<const int4*>(shell4); a.coef = coef;
    gridDim = {1, 1, 1}; blockDim = {1, 1, 1}; blockIdx = {0, 0, 0}; threadIdx = {0, 0, 0};
    gb::k_sph_transform(a);
}
"""


@pytest.fixture(scope="module")
def lib():
    sys.path.insert(0, os.path.join(ROOT, "paper_2412_13203_gb300", "codegen"))
    try:
        import sph_codegen
    finally:
        sys.path.pop(0)
    os.makedirs(BUILD, exist_ok=True)
    table = sph_codegen.emit(BUILD)
    drv = os.path.join(BUILD, "driver.cpp")
    with open(drv, "w") as f:
        f.write(DRIVER)
    srcs = [drv, table, os.path.join(CSRC, "sph_transform.cuh"), os.path.join(HERE, "emu", "cuda_runtime.h")]
    h = hashlib.sha1()
    for s in srcs:
        h.update(open(s, "rb").read())
    so = os.path.join(BUILD, f"libsph_{h.hexdigest()[:12]}.so")
    if not os.path.exists(so):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-w", "-I", os.path.join(HERE, "emu"),
                        "-I", CSRC, drv, "-x", "c++", table, "-o", tmp], check=True)
        os.replace(tmp, so)
    L = C.CDLL(so)
    vp = C.c_void_p
    L.emu_sph.argtypes = [vp, vp, C.c_int, C.c_int, C.c_int, vp, vp, vp]
    L.emu_table.argtypes = [C.POINTER(C.POINTER(C.c_double)), C.POINTER(C.POINTER(C.c_int))]
    return L


def _layout(lib, ls):
    """Shell records, owners and the coefficient table, as the runtime builds them."""
    cp, op = C.POINTER(C.c_double)(), C.POINTER(C.c_int)()
    lmax = lib.emu_table(C.byref(cp), C.byref(op))
    assert lmax == 3
    off = [op[i] for i in range(lmax + 2)]
    coef = np.array([cp[i] for i in range(off[-1])])
    shell, own_c, own_p = [], [], []
    c = p = 0
    for s, l in enumerate(ls):
        nc, np_ = molgen.ncart(l), sp.nsph(l)
        shell.append((l, c, p, off[l]))
        own_c += [s] * nc
        own_p += [s] * np_
        c += nc
        p += np_
    return (np.array(shell, np.int32).ravel(), np.array(own_c, np.int32), np.array(own_p, np.int32), coef, c, p)


def _run(lib, ls, M, direction):
    shell, own_c, own_p, coef, nc, npure = _layout(lib, ls)
    if direction == 0:
        n_in, n_out, owner = npure, nc, own_c
    else:
        n_in, n_out, owner = nc, npure, own_p
    M = np.ascontiguousarray(M, dtype=np.float64)
    assert M.shape == (n_in, n_in)
    out = np.full((n_out, n_out), np.nan)
    lib.emu_sph(M.ctypes.data, out.ctypes.data, n_in, n_out, direction, owner.ctypes.data, shell.ctypes.data,
                coef.ctypes.data)
    return out


def _mol(ls_per_atom, natom=2, seed=11):
    return molgen.random_molecule(seed=seed, natom=natom, shells_per_atom=ls_per_atom, kmin=1, kmax=2,
                                  alpha_min=0.3, alpha_max=5.0)


@pytest.mark.parametrize("ls_per_atom", [[0, 1, 2, 3], [3, 2, 2, 0, 1], [2], [3]])
def test_transform_matches_oracle(lib, ls_per_atom):
    mol = _mol(ls_per_atom)
    ls = [int(l) for l in mol.shell_l]
    T = sp.transform_matrix(mol)
    rng = np.random.default_rng(len(ls))
    Dp = rng.normal(size=(T.shape[1],) * 2)  # not symmetric: checks the row/column orientation
    Mc = rng.normal(size=(T.shape[0],) * 2)
    np.testing.assert_allclose(_run(lib, ls, Dp, 0), T @ Dp @ T.T, rtol=0, atol=1e-14 * 16 * np.abs(Dp).max())
    np.testing.assert_allclose(_run(lib, ls, Mc, 1), T.T @ Mc @ T, rtol=0, atol=1e-14 * 25 * np.abs(Mc).max())


def test_s_and_p_pass_through_exactly(lib):
    mol = _mol([0, 1, 1, 0], natom=3)
    ls = [int(l) for l in mol.shell_l]
    M = np.random.default_rng(2).normal(size=(mol.nbf, mol.nbf))
    for d in (0, 1):
        np.testing.assert_array_equal(_run(lib, ls, M, d), M)


def test_pure_jk_through_the_kernel(lib):
    """Pure-basis J/K from the Cartesian oracle and the emulated kernel in both
    directions equal the oracle's pure-basis definition."""
    import oracle
    mol = _mol([0, 1, 2, 3], natom=2, seed=4)
    ls = [int(l) for l in mol.shell_l]
    ns = sum(sp.nsph(l) for l in ls)
    C_ = np.random.default_rng(9).normal(0, 0.3, (ns, 5))
    Dp = C_ @ C_.T
    Dc = _run(lib, ls, Dp, 0)
    Jc, Kc, _ = oracle.jk(mol, Dc, mode="all")
    Jp, Kp = _run(lib, ls, Jc, 1), _run(lib, ls, Kc, 1)
    Jw, Kw = sp.jk_pure(mol, Dp)
    np.testing.assert_allclose(Jp, Jw, rtol=0, atol=1e-11 * np.abs(Jw).max())
    np.testing.assert_allclose(Kp, Kw, rtol=0, atol=1e-11 * np.abs(Kw).max())


def test_generated_table_equals_oracle_coefficients():
    """The generator's closed form (triple sum) and the oracle's Legendre
    construction give the same T_l for every l."""
    sys.path.insert(0, os.path.join(ROOT, "paper_2412_13203_gb300", "codegen"))
    try:
        import sph_codegen
    finally:
        sys.path.pop(0)
    for l in range(4):
        np.testing.assert_allclose(np.array(sph_codegen.table(l)), sp.coefficients(l), rtol=0, atol=1e-15)
