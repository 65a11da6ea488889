"""The mixed-precision split and density-screening kernels (csrc/split_kernels.cuh),
compiled as plain C++ against tests/emu/cuda_runtime.h and run row by row on
synthetic rows, against the classification rule they implement:

    global bound g = (Q_ab max|D|) Q_cd,  weighted bound w = Q_ab Q_cd max(D blocks)
    g <  eps               -> skipped
    g >= tau, w >= tau     -> FP64 list
    g >= tau, eps <= w < tau -> demoted (FP32 list)
    g >= tau, w <  eps     -> skipped
    eps <= g < tau         -> FP32 contiguous range

Test infrastructure only."""
import ctypes as C
import hashlib
import os

import numpy as np
import pytest

import kernel_emu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2412_13203_gb300", "csrc")
BUILD = os.path.join(HERE, "_emu_build", "split")

DRIVER = r"""
#include "eri_device.cuh"
namespace {
#include "split_kernels.cuh"
}
emu_dim3 blockIdx, threadIdx, blockDim, gridDim;
// one emulated thread per row (blockDim 1, blockIdx = row)
extern "C" void emu_split(const long long* start, const int* rbra, const int* rket0, int nrows, const double* A4,
                          double dmax, double tau, double eps, const int* info4, const int* psh2, const float* dsh,
                          int nshell, int P, long long* c64, long long* cdem, long long* c32, int* k32,
                          long long* w64, long long* wdem, long long* w32, unsigned long long* qtot) {
    blockDim = {1, 1, 1}; gridDim = {(unsigned)nrows, 1, 1}; threadIdx = {0, 0, 0};
    for (int r = 0; r < nrows; ++r) {
        blockIdx = {(unsigned)r, 0, 0};
        k_rows_split(start, rbra, rket0, nrows, reinterpret_cast<const double4*>(A4), &dmax, tau, eps,
                     reinterpret_cast<const int4*>(info4), reinterpret_cast<const int2*>(psh2), dsh, nshell, P,
                     c64, cdem, c32, k32, w64, wdem, w32, qtot);
    }
}
extern "C" void emu_fill(const int* rbra, const int* rket0, const int* k32, int nrows, const double* A4, double tau,
                         double eps, const int* psh2, const float* dsh, int nshell, const long long* l64,
                         const long long* ldem, int* list64, int* listdem, float taup, float* thr64) {
    blockDim = {1, 1, 1}; gridDim = {(unsigned)nrows, 1, 1}; threadIdx = {0, 0, 0};
    for (int r = 0; r < nrows; ++r) {
        blockIdx = {(unsigned)r, 0, 0};
        k_rows_fill(rbra, rket0, k32, nrows, reinterpret_cast<const double4*>(A4), tau, eps,
                    reinterpret_cast<const int2*>(psh2), dsh, nshell, l64, ldem, list64, listdem, taup, thr64);
    }
}
"""


def build_split_lib():
    """Compile (cached by source hash) and load the split-kernel emulation library."""
    os.makedirs(BUILD, exist_ok=True)
    drv = os.path.join(BUILD, "driver.cpp")
    with open(drv, "w") as f:
        f.write(DRIVER)
    h = hashlib.sha1()
    for s in (drv, os.path.join(CSRC, "split_kernels.cuh"), os.path.join(CSRC, "eri_device.cuh"),
              os.path.join(HERE, "emu", "cuda_runtime.h")):
        h.update(open(s, "rb").read())
    so = os.path.join(BUILD, f"libsplit_{h.hexdigest()[:12]}.so")
    if not os.path.exists(so):
        import subprocess
        tmp = so + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-w", "-I", os.path.join(HERE, "emu"),
                        "-I", CSRC, "-I", os.path.join(ROOT, "include"), drv, "-o", tmp], check=True)
        os.replace(tmp, so)
    L = C.CDLL(so)
    vp = C.c_void_p
    L.emu_split.argtypes = ([vp, vp, vp, C.c_int, vp, C.c_double, C.c_double, C.c_double, vp, vp, vp, C.c_int, C.c_int]
                            + [vp] * 8)
    L.emu_fill.argtypes = [vp, vp, vp, C.c_int, vp, C.c_double, C.c_double, vp, vp, C.c_int, vp, vp, vp, vp,
                           C.c_float, vp]
    return L


@pytest.fixture(scope="module")
def lib():
    return build_split_lib()


def _rows(seed, nshell=12, npair=40, nrows=25):
    """Pairs with Q sorted descending (as the pair build leaves them), shells
    per pair, shell-block maxima of D, and rows (bra pair, ket range)."""
    rng = np.random.default_rng(seed)
    Q = np.sort(10.0 ** rng.uniform(-7, 0.5, npair))[::-1]
    A = np.zeros((npair, 4))
    A[:, 3] = Q
    info = np.zeros((npair, 4), np.int32)
    info[:, 2] = rng.integers(1, 10, npair)  # primitive pairs
    psh = np.sort(rng.integers(0, nshell, (npair, 2)), axis=1)[:, ::-1].astype(np.int32).copy()
    dsh = (10.0 ** rng.uniform(-6, 0, (nshell, nshell))).astype(np.float32)
    dsh = np.maximum(dsh, dsh.T).copy()
    rbra = rng.integers(0, npair, nrows).astype(np.int32)
    rket0 = rng.integers(0, npair, nrows).astype(np.int32)
    cnt = np.array([rng.integers(0, npair - k + 1) for k in rket0], np.int64)
    cnt[0] = 0  # an empty row
    start = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    return A, info, psh, dsh, rbra, rket0, start, float(dsh.max())


def _classify(A, psh, dsh, i, j, dmax, tau, eps):
    qi, qj = A[i, 3], A[j, 3]
    g = (qi * dmax) * qj
    if g < eps:
        return "skip"
    if g < tau:
        return "fp32"
    (a, b), (c, d) = psh[i], psh[j]
    w = qi * qj * float(max(dsh[a, b], dsh[c, d], dsh[a, c], dsh[a, d], dsh[b, c], dsh[b, d]))
    return "fp64" if w >= tau else ("dem" if w >= eps else "skip")


@pytest.mark.parametrize("seed,tau,eps", [(1, 1e-2, 0.0), (2, 1e-2, 1e-6), (3, 1e-4, 1e-3), (4, 0.0, 1e-5),
                                          (5, 1e-3, 1e-9)])
def test_split_and_fill_follow_the_rule(lib, seed, tau, eps):
    A, info, psh, dsh, rbra, rket0, start, dmax = _rows(seed)
    n = len(rbra)
    P = 4
    out = {k: np.zeros(n + 1, np.int64) for k in ("c64", "cdem", "c32", "w64", "wdem", "w32")}
    k32 = np.zeros(n, np.int32)
    qtot = np.zeros(8, np.uint64)
    lib.emu_split(start.ctypes.data, rbra.ctypes.data, rket0.ctypes.data, n, A.ctypes.data, dmax, tau, eps,
                  info.ctypes.data, psh.ctypes.data, dsh.ctypes.data, dsh.shape[0], P,
                  *[out[k].ctypes.data for k in ("c64", "cdem", "c32")], k32.ctypes.data,
                  *[out[k].ctypes.data for k in ("w64", "wdem", "w32")], qtot.ctypes.data)
    l64 = np.concatenate([[0], np.cumsum(out["c64"][:n])]).astype(np.int64)
    ldem = np.concatenate([[0], np.cumsum(out["cdem"][:n])]).astype(np.int64)
    list64 = np.full(max(1, l64[-1]), -1, np.int32)
    listdem = np.full(max(1, ldem[-1]), -1, np.int32)
    thr64 = np.full(max(1, l64[-1]), -1.0, np.float32)
    taup = np.float32(tau / 10)
    lib.emu_fill(rbra.ctypes.data, rket0.ctypes.data, k32.ctypes.data, n, A.ctypes.data, tau, eps,
                 psh.ctypes.data, dsh.ctypes.data, dsh.shape[0], l64.ctypes.data, ldem.ctypes.data,
                 list64.ctypes.data, listdem.ctypes.data, taup, thr64.ctypes.data)
    tot = {"fp64": 0, "dem": 0, "fp32": 0, "skip": 0}
    for r in range(n):
        i, s, c = int(rbra[r]), int(rket0[r]), int(start[r + 1] - start[r])
        cls = [_classify(A, psh, dsh, i, j, dmax, tau, eps) for j in range(s, s + c)]
        for k in cls:
            tot[k] += 1
        m = kernel_emu.mg.item_split(P, int(info[i, 2]))
        want64 = [j for j, k in zip(range(s, s + c), cls) if k == "fp64"]
        wantdem = [j for j, k in zip(range(s, s + c), cls) if k == "dem"]
        want32 = [j for j, k in zip(range(s, s + c), cls) if k == "fp32"]
        assert (out["c64"][r], out["cdem"][r], out["c32"][r]) == (len(want64), len(wantdem), len(want32)), r
        assert (out["w64"][r], out["wdem"][r], out["w32"][r]) == (m * len(want64), m * len(wantdem), m * len(want32))
        # the FP32 kets are the contiguous range starting at k32
        assert want32 == list(range(int(k32[r]), int(k32[r]) + len(want32)))
        assert list(list64[l64[r]:l64[r + 1]]) == want64
        assert list(listdem[ldem[r]:ldem[r + 1]]) == wantdem
        # primitive cut of every FP64 entry: taup over the largest |D| of the quartet's six blocks, in FP32
        (a, b) = psh[i]
        for e, j in zip(range(l64[r], l64[r + 1]), want64):
            (c, d) = psh[j]
            dq = np.float32(max(dsh[a, b], dsh[c, d], dsh[a, c], dsh[a, d], dsh[b, c], dsh[b, d]))
            assert thr64[e] == np.float32(taup / dq), (thr64[e], taup / dq)
    assert int(qtot[0]) == tot["fp32"] + tot["dem"] and int(qtot[1]) == tot["fp64"] and int(qtot[7]) == tot["dem"]
    if eps == 0.0:
        assert tot["skip"] == 0
    else:
        assert tot["skip"] > 0


def test_split_with_zero_density_demotes_everything(lib):
    A, info, psh, dsh, rbra, rket0, start, _ = _rows(7)
    n = len(rbra)
    z = np.zeros_like(dsh)
    bufs = [np.zeros(n + 1, np.int64) for _ in range(6)]
    k32 = np.zeros(n, np.int32)
    qtot = np.zeros(8, np.uint64)
    lib.emu_split(start.ctypes.data, rbra.ctypes.data, rket0.ctypes.data, n, A.ctypes.data, 0.0, 1e-2, 0.0,
                  info.ctypes.data, psh.ctypes.data, z.ctypes.data, z.shape[0], 4,
                  *[b.ctypes.data for b in bufs[:3]], k32.ctypes.data, *[b.ctypes.data for b in bufs[3:]],
                  qtot.ctypes.data)
    assert int(qtot[1]) == 0 and int(qtot[0]) == int(start[-1])
    np.testing.assert_array_equal(k32, rket0)
