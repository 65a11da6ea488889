"""The one-electron kernel (csrc/one_electron.cuh) compiled as plain C++ against
tests/emu/cuda_runtime.h and run on the CPU over pair data laid out as the
runtime lays them out (tests/kernel_emu.py), against the oracle's Obara-Saika
S, T and V.  Test infrastructure only."""
import ctypes as C
import hashlib
import os

import numpy as np
import pytest

import molgen
import oracle
from oracle import one_electron as oe

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2412_13203_gb300", "csrc")
BUILD = os.path.join(HERE, "_emu_build", "one")

DRIVER = r"""
#include <cstring>
#include "eri_device.cuh"
#include "one_electron.cuh"
emu_dim3 blockIdx, threadIdx, blockDim, gridDim;
// one emulated thread walks the grid-stride loop over every pair
extern "C" void emu_one(int npair, const int* info4, const double* A4, const double* B4, const double* pp4,
                        const double* pp2, const double* alpha, const int* lab2, const double* boys,
                        const double* xyz, const double* Z, int natom, int nbf, double* S, double* T, double* V) {
    gb::OneElArgs a;
    std::memset(&a, 0, sizeof(a));
    a.pairs.npair = npair;
    a.pairs.info = reinterpret_cast<const int4*>(info4);
    a.pairs.A = reinterpret_cast<const double4*>(A4);
    a.pairs.B = reinterpret_cast<const double4*>(B4);
    a.pairs.pp = reinterpret_cast<const double4*>(pp4);
    a.pairs.pp2 = reinterpret_cast<const double2*>(pp2);
    a.pairs.alpha = alpha;
    a.lab = reinterpret_cast<const int2*>(lab2);
    a.boys = boys; a.xyz = xyz; a.Z = Z; a.natom = natom; a.nbf = nbf; a.S = S; a.T = T; a.V = V;
    gridDim = {1, 1, 1}; blockDim = {1, 1, 1}; blockIdx = {0, 0, 0}; threadIdx = {0, 0, 0};
    gb::k_one_electron(a);
}
"""


@pytest.fixture(scope="module")
def lib():
    os.makedirs(BUILD, exist_ok=True)
    drv = os.path.join(BUILD, "driver.cpp")
    with open(drv, "w") as f:
        f.write(DRIVER)
    h = hashlib.sha1()
    for s in (drv, os.path.join(CSRC, "one_electron.cuh"), os.path.join(CSRC, "eri_device.cuh"),
              os.path.join(HERE, "emu", "cuda_runtime.h")):
        h.update(open(s, "rb").read())
    so = os.path.join(BUILD, f"libone_{h.hexdigest()[:12]}.so")
    if not os.path.exists(so):
        import subprocess
        tmp = so + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-w", "-I", os.path.join(HERE, "emu"),
                        "-I", CSRC, "-I", os.path.join(ROOT, "include"), drv, "-o", tmp], check=True)
        os.replace(tmp, so)
    L = C.CDLL(so)
    L.emu_one.argtypes = [C.c_int] + [C.c_void_p] * 10 + [C.c_int, C.c_int] + [C.c_void_p] * 3
    return L


def _run(lib, mol):
    import kernel_emu
    pr = kernel_emu.Problem(mol, np.zeros((mol.nbf, mol.nbf)), oracle, lmax=3)
    lab = np.array([(int(mol.shell_l[a]), int(mol.shell_l[b])) for a, b in pr.pair_shells], np.int32)
    n = mol.nbf
    S, T, V = (np.full((n, n), np.nan) for _ in range(3))
    Z = np.ascontiguousarray(mol.charges, dtype=np.float64)
    xyz = np.ascontiguousarray(mol.xyz, dtype=np.float64)
    p = lambda a: a.ctypes.data  # noqa: E731
    lib.emu_one(len(pr.pair_shells), p(pr.info), p(pr.A), p(pr.B), p(pr.pp), p(pr.pp2), p(pr.alpha), p(lab),
                p(pr.boys), p(xyz), p(Z), mol.natom, n, p(S), p(T), p(V))
    return S, T, V


@pytest.mark.parametrize("seed,shells,natom", [(1, [0, 1], 3), (2, [2, 0, 1], 2), (3, [3, 1], 2), (4, [3, 2, 0], 2),
                                               (5, [0, 1, 2, 3], 2)])
def test_kernel_matches_oracle(lib, seed, shells, natom):
    mol = molgen.random_molecule(950 + seed, natom, shells, 1, 3, 0.1, 20.0, layout="lattice", spacing=1.7)
    mol.charges = np.arange(1, natom + 1, dtype=np.float64) * 1.5
    S, T, V = _run(lib, mol)
    So, To, Vo = oe.one_electron(mol)
    assert not np.isnan(S).any()  # every element written: all pairs are kept here
    for M, Mo in ((S, So), (T, To), (V, Vo)):
        np.testing.assert_allclose(M, Mo, rtol=0, atol=1e-12 * np.abs(Mo).max())
