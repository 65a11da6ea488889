"""A mixed build end to end on the CPU, as the runtime runs it: the split and
list kernels (csrc/split_kernels.cuh) place every quartet of a row in the
FP64 list, the FP32 range, the demoted FP32 list or, under density screening,
nowhere; the generated class kernels then run the three parts (the FP64 list
kernel with explicit ket lists, the FP32 kernel over the contiguous range from
k32, the FP32 kernel over the demoted list), each from its own work-item
prefix.  J and K are compared with the oracle over exactly the kept quartets.
Pairs are ordered by Schwarz factor inside each class, as the runtime orders
them.  Test infrastructure only."""
import numpy as np
import pytest

import kernel_emu
import molgen
import oracle
from test_split_emulation import _classify, build_split_lib

mg = kernel_emu.mg


def _excl(x):
    return np.concatenate([[0], np.cumsum(x)]).astype(np.int64)


def _mixed_build(pr, tau, eps, taup=0.0):
    """A mixed build as the runtime runs it: split counts, list fill, then the
    FP64 list, the FP32 suffix and the demoted list through the class kernels;
    with taup > 0 (a primitive-sorted problem) the FP64 list runs its large
    primitive quartets in FP64 (primitive mode 1) and the rest in FP32 over the
    same list (mode 2)."""
    lib = kernel_emu.load(pr.lmax, pr.only)
    split = build_split_lib()
    mol, D, n = pr.mol, pr.D, pr.nbf
    off = np.concatenate([mol.shell_offsets(), [n]])
    S = mol.nshell
    dsh = np.array([[np.abs(D[off[a]:off[a + 1], off[b]:off[b + 1]]).max() for b in range(S)] for a in range(S)],
                   dtype=np.float32)
    dmax = float(np.abs(D).max())
    psh = np.ascontiguousarray(np.array(pr.pair_shells, np.int32))
    J = np.zeros((n, n))
    K = np.zeros((n, n))
    kept, want = [], 0
    parts = {"fp64": 0, "fp32": 0, "dem": 0}
    p = pr._p
    common = lambda: (len(pr.info), p(pr.info), p(pr.A), p(pr.B), p(pr.pp), p(pr.pp2), p(pr.ppf), p(pr.ppf2),  # noqa
                      p(pr.alpha))
    tail = lambda: (p(pr.boys), p(pr.boysf), kernel_emu.C.c_float(1.0), p(pr.D), p(pr.Df), p(J), p(K), n)  # noqa
    for X in range(len(pr.pcs)):
        for Y in range(X + 1):
            r = pr.rows(X, Y, items=False)
            if r is None:
                continue
            bra, ket0, start = r
            nr = len(bra)
            P = mg.split_of(pr.pcs[X], pr.pcs[Y])
            cnt = {k: np.zeros(nr + 1, np.int64) for k in ("c64", "cdem", "c32", "w64", "wdem", "w32")}
            k32 = np.zeros(nr, np.int32)
            qtot = np.zeros(8, np.uint64)
            split.emu_split(start.ctypes.data, bra.ctypes.data, ket0.ctypes.data, nr, pr.A.ctypes.data, dmax, tau,
                            eps, pr.info.ctypes.data, psh.ctypes.data, dsh.ctypes.data, S, P,
                            *[cnt[k].ctypes.data for k in ("c64", "cdem", "c32")], k32.ctypes.data,
                            *[cnt[k].ctypes.data for k in ("w64", "wdem", "w32")], qtot.ctypes.data)
            s64, s32, sdem = (_excl(cnt[k][:nr]) for k in ("w64", "w32", "wdem"))
            l64, ldem = _excl(cnt["c64"][:nr]), _excl(cnt["cdem"][:nr])
            list64 = np.zeros(max(1, l64[-1]), np.int32)
            listdem = np.zeros(max(1, ldem[-1]), np.int32)
            thr64 = np.zeros(max(1, l64[-1]), np.float32)
            split.emu_fill(bra.ctypes.data, ket0.ctypes.data, k32.ctypes.data, nr, pr.A.ctypes.data, tau, eps,
                           psh.ctypes.data, dsh.ctypes.data, S, l64.ctypes.data, ldem.ctypes.data,
                           list64.ctypes.data, listdem.ctypes.data, taup, thr64.ctypes.data if taup > 0 else None)
            launches = [(0, s64, None, l64, list64, 1 if taup > 0 else 0), (1, s32, k32, None, None, 0),
                        (1, sdem, None, ldem, listdem, 0)]
            if taup > 0:
                launches.append((1, s64, None, l64, list64, 2))
            for prec, st, k0, ko, kl, pmode in launches:
                if st[-1] == 0:
                    continue
                lib.emu_set_prim(None if pr.pq is None else p(pr.pq), p(thr64) if pmode else None, pmode)
                rc = lib.emu_jk(X, Y, prec, *common(), nr, p(st), p(bra), None if k0 is None else p(k0),
                                None if ko is None else p(ko), None if kl is None else p(kl), *tail())
                assert rc == 0
            parts["fp64"] += int(l64[-1])
            parts["dem"] += int(ldem[-1])
            parts["fp32"] += int(cnt["c32"][:nr].sum())
            for row in range(nr):
                i = int(bra[row])
                kets = list(list64[l64[row]:l64[row + 1]]) + list(range(int(k32[row]), int(k32[row]) + int(cnt["c32"][row]))) \
                    + list(listdem[ldem[row]:ldem[row + 1]])
                kept += [(i, int(j)) for j in kets]
                c = int(start[row + 1] - start[row])
                want += sum(_classify(pr.A, psh, dsh, i, j, dmax, tau, eps) != "skip"
                            for j in range(int(ket0[row]), int(ket0[row]) + c))
    assert len(kept) == want
    quartets = []
    for i, j in kept:
        a, b = sorted(pr.pair_shells[i], reverse=True)
        c, d = sorted(pr.pair_shells[j], reverse=True)
        if a * (a + 1) // 2 + b < c * (c + 1) // 2 + d:
            a, b, c, d = c, d, a, b
        quartets.append((a, b, c, d))
    return J + J.T, K + K.T, np.array(quartets, np.int32), parts


@pytest.mark.parametrize("seed,shells,scale,tau,eps,taup", [(81, [0, 1, 2], 1.0, 1e-2, 0.0, 0.0),
                                                            (82, [0, 1, 2], 1e-2, 1e-2, 1e-7, 0.0),
                                                            (83, [2, 0, 1], 1e-3, 0.0, 1e-8, 0.0),
                                                            (84, [0, 1, 3], 1e-2, 1e-3, 1e-7, 0.0),
                                                            (81, [0, 1, 2], 1.0, 1e-2, 0.0, 1e-3),
                                                            (84, [0, 1, 3], 1e-2, 1e-3, 1e-7, 1e-5)])
def test_mixed_build_with_screening_matches_oracle(seed, shells, scale, tau, eps, taup):
    mol = molgen.random_molecule(1000 + seed, 3, shells, 1, 3, 0.1, 50.0, layout="lattice", spacing=2.2)
    D = molgen.density(mol, 1100 + seed) * scale
    lmax = max(shells)
    pr = kernel_emu.Problem(mol, D, oracle, lmax=lmax, own_classes=True, q_order=True, prim_sort=taup > 0)
    J, K, q, parts = _mixed_build(pr, tau, eps, taup)
    if tau == 0.0:  # FP64 build with screening: every kept quartet in the FP64 list
        assert parts["fp32"] == parts["dem"] == 0 and parts["fp64"] == len(q)
    elif seed in (81, 84):  # all three launch forms run
        assert min(parts.values()) > 0
    nq_all = len(pr.pair_shells) * (len(pr.pair_shells) + 1) // 2
    if eps == 0.0:
        assert len(q) == nq_all
    else:
        assert 0 < len(q) < nq_all
    Jo, Ko = oracle.jk_quartets(mol, D, q)
    s = max(np.abs(Jo).max(), 1e-300)
    assert np.abs(J - Jo).max() <= 2e-6 * s, np.abs(J - Jo).max() / s
    assert np.abs(K - Ko).max() <= 2e-6 * s, np.abs(K - Ko).max() / s
