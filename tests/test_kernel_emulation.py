"""The generated CUDA kernels, compiled as plain C++ and run thread by thread
on the CPU (tests/kernel_emu.py), against the oracle: J and K of every l <= 2
class in FP64 and in FP32 (all quartets in the FP32 kernels), and the nuclear
gradient.  This exercises the kernels' own work-item decoding, splitting over
bra primitive pairs, degeneracy factors, digestion and Boys evaluation, not
only the generated algebra."""
import numpy as np
import pytest

import molgen
import oracle

kernel_emu = pytest.importorskip("kernel_emu")


def _mol(seed, shells, natom, kmax):
    mol = molgen.random_molecule(seed, natom, shells, 1, kmax, 0.1, 60.0, layout="lattice", spacing=1.9)
    return mol, molgen.density(mol, seed + 50)


@pytest.mark.parametrize("seed,shells,natom,kmax", [(61, [0, 1, 2], 2, 3), (62, [2, 1], 2, 2), (63, [0, 2, 2], 2, 2)])
def test_emulated_jk_fp64_and_fp32(seed, shells, natom, kmax):
    mol, D = _mol(seed, shells, natom, kmax)
    pr = kernel_emu.Problem(mol, D, oracle)
    Jo, Ko, _ = oracle.jk(mol, D, mode="unique")
    J, K = pr.jk(0)
    assert np.abs(J - Jo).max() <= 1e-10 * max(1.0, np.abs(Jo).max())
    assert np.abs(K - Ko).max() <= 1e-10 * max(1.0, np.abs(Ko).max())
    J, K = pr.jk(1)
    assert np.abs(J - Jo).max() <= 2e-6 * np.abs(Jo).max()
    assert np.abs(K - Ko).max() <= 2e-6 * np.abs(Ko).max()
    # the explicit-ket-list form of the rows (mixed builds' FP64 and demoted lists)
    J, K = pr.jk(0, lists=True)
    assert np.abs(J - Jo).max() <= 1e-10 * max(1.0, np.abs(Jo).max())
    assert np.abs(K - Ko).max() <= 1e-10 * max(1.0, np.abs(Ko).max())


def test_emulated_gradient():
    mol, D = _mol(64, [0, 1, 2], 2, 2)
    pr = kernel_emu.Problem(mol, D, oracle)
    g = pr.grad()
    go = oracle.grad(mol, D, mode="unique")
    assert np.abs(g - go).max() <= 1e-10 * max(1.0, np.abs(go).max())


@pytest.mark.parametrize("seed,shells,lmax", [(64, [0, 1, 2], 2), (74, [1, 3], 3)])
def test_emulated_gradient_fp32(seed, shells, lmax):
    """The FP32 derivative kernels (every quartet in FP32, real FP32 arithmetic;
    the mixed gradient runs them for its small-bound quartets) against the
    oracle's analytic gradient, and translational invariance."""
    mol, D = _mol(seed, shells, 2, 2)
    pr = kernel_emu.Problem(mol, D, oracle, lmax=lmax)
    g = pr.grad(prec=1)
    go = oracle.grad(mol, D, mode="unique")
    scale = max(1.0, np.abs(go).max())
    assert np.abs(g - go).max() <= 2e-6 * scale, np.abs(g - go).max() / scale
    assert np.abs(g.sum(axis=0)).max() <= 2e-6 * scale


@pytest.mark.parametrize("seed,shells", [(69, [0, 3]), (70, [3, 1]), (71, [2, 3])])
def test_emulated_gradient_f_classes(seed, shells):
    """Derivative kernels of classes with an f shell (one thread per work item
    and ket component, rolled R) against the oracle's analytic gradient."""
    mol, D = _mol(seed, shells, 2, 2)
    pr = kernel_emu.Problem(mol, D, oracle, lmax=3)
    g = pr.grad()
    go = oracle.grad(mol, D, mode="unique")
    scale = max(1.0, np.abs(go).max())
    assert np.abs(g - go).max() <= 1e-10 * scale, np.abs(g - go).max()
    assert np.abs(g.sum(axis=0)).max() <= 1e-10 * scale


@pytest.mark.parametrize("seed,shells", [(65, [0, 3]), (66, [1, 3]), (72, [0, 1, 2, 3])])
def test_emulated_f_classes(seed, shells):
    """Classes with an f shell (one thread per ket component, rolled R)."""
    mol, D = _mol(seed, shells, 2, 2)
    pr = kernel_emu.Problem(mol, D, oracle, lmax=3)
    Jo, Ko, _ = oracle.jk(mol, D, mode="unique")
    for prec, tol in ((0, 1e-10), (1, 2e-6)):
        J, K = pr.jk(prec)
        assert np.abs(J - Jo).max() <= tol * max(1.0, np.abs(Jo).max()), (prec, np.abs(J - Jo).max())
        assert np.abs(K - Ko).max() <= tol * max(1.0, np.abs(Ko).max()), (prec, np.abs(K - Ko).max())


@pytest.mark.parametrize("seed,shells,lmax", [(67, [0, 1, 2], 2), (68, [2, 3], 3)])
def test_emulated_schwarz_factors(seed, shells, lmax):
    """Q_ab = sqrt(max_i |(ab|ab)_ii|) from the generated Schwarz kernels
    (single-thread and per-component forms) against the oracle's."""
    mol, D = _mol(seed, shells, 2, 2)
    pr = kernel_emu.Problem(mol, D, oracle, lmax=lmax)
    Q = pr.schwarz()
    Qo = oracle.schwarz(mol)
    want = np.array([Qo[a, b] for a, b in pr.pair_shells])
    assert np.abs(Q - want).max() <= 1e-11 * max(1.0, want.max()), np.abs(Q - want).max()


def test_emulated_path_searched_r(monkeypatch):
    """The kernels emitted with Algorithm 1's recursion order (off in the
    built library) give the same J and K."""
    import md_codegen
    monkeypatch.setattr(md_codegen, "R_PATH_LAMBDA", 1.0)
    mol, D = _mol(69, [0, 1, 2], 2, 2)
    pr = kernel_emu.Problem(mol, D, oracle, own_classes=True)
    Jo, Ko, _ = oracle.jk(mol, D, mode="unique")
    for prec, tol in ((0, 1e-10), (1, 2e-6)):
        J, K = pr.jk(prec)
        assert np.abs(J - Jo).max() <= tol * max(1.0, np.abs(Jo).max()), prec
        assert np.abs(K - Ko).max() <= tol * max(1.0, np.abs(Ko).max()), prec


@pytest.mark.parametrize("seed,shells,natom,kmax", [(61, [0, 1, 2], 2, 3), (63, [0, 2, 2], 2, 2)])
def test_emulated_double_float(seed, shells, natom, kmax):
    """The double-float kernels (hi + lo float pairs, FP32 arithmetic only; the
    mixed build runs its largest-bound quartets in them) against the oracle,
    and far more accurate than the FP32 kernels."""
    mol, D = _mol(seed, shells, natom, kmax)
    pr = kernel_emu.Problem(mol, D, oracle)
    Jo, Ko, _ = oracle.jk(mol, D, mode="unique")
    J, K = pr.jk(3)
    sJ, sK = max(1.0, np.abs(Jo).max()), max(1.0, np.abs(Ko).max())
    assert np.abs(J - Jo).max() <= 1e-11 * sJ, np.abs(J - Jo).max() / sJ
    assert np.abs(K - Ko).max() <= 1e-11 * sK, np.abs(K - Ko).max() / sK


def test_emulated_rpath_variants_of_the_library():
    """The FP32 range kernels the library also carries in Algorithm 1's
    recursion order ((dd|dd), (dd|dp), (dp|dp); launched under the R-path
    option) give the oracle's J and K like the fixed-order ones."""
    mol, D = _mol(73, [1, 2], 2, 2)
    pr = kernel_emu.Problem(mol, D, oracle)
    Jo, Ko, _ = oracle.jk(mol, D, mode="unique")
    J1, K1 = pr.jk(1)
    J2, K2 = pr.jk(2)
    for J, K in ((J1, K1), (J2, K2)):
        assert np.abs(J - Jo).max() <= 2e-6 * max(1.0, np.abs(Jo).max())
        assert np.abs(K - Ko).max() <= 2e-6 * max(1.0, np.abs(Ko).max())
    # a different evaluation order, so not bit-identical, but the same integrals
    assert np.abs(J2 - J1).max() > 0.0


def test_emulated_batched_mode():
    """The kernels' batched mode (rows of several molecules in one launch,
    per-row molecule lookup) gives each molecule's J and K."""
    mols = [_mol(70 + i, sh, 2, 2) for i, sh in enumerate([[0, 1, 2], [1, 2], [0, 0, 2]])]
    prs = [kernel_emu.Problem(m, D, oracle) for m, D in mols]
    for prec, tol in ((0, 1e-10), (1, 2e-6)):
        Js, Ks = kernel_emu.jk_batched(prs, prec)
        for (mol, D), J, K in zip(mols, Js, Ks):
            Jo, Ko, _ = oracle.jk(mol, D, mode="unique")
            assert np.abs(J - Jo).max() <= tol * max(1.0, np.abs(Jo).max()), prec
            assert np.abs(K - Ko).max() <= tol * max(1.0, np.abs(Ko).max()), prec


@pytest.mark.parametrize("seed,shells,natom,kmax", [(81, [0, 1, 2], 2, 4), (82, [2, 1], 3, 3)])
def test_emulated_primitive_split(seed, shells, natom, kmax):
    """The primitive split of a mixed build's FP64 list: with each pair's
    primitive pairs sorted by their Schwarz factor, the kernels' primitive
    mode 1 (quartets at or above the cut) and mode 2 (below it) together
    evaluate every primitive quartet exactly once -- FP64 mode 1 + FP64 mode 2
    equals the unsplit FP64 build -- and mode 2 in FP32 beside mode 1 in FP64
    or double-float stays within FP32 rounding of the cut part."""
    mol, D = _mol(seed, shells, natom, kmax)
    pr = kernel_emu.Problem(mol, D, oracle, prim_sort=True)
    Jo, Ko, _ = oracle.jk(mol, D, mode="unique")
    J0, K0 = pr.jk(0, lists=True)
    assert np.abs(J0 - Jo).max() <= 1e-10 * max(1.0, np.abs(Jo).max())
    taup = 1e-3
    J1, K1 = pr.jk(0, lists=True, pmode=1, taup=taup)
    J2, K2 = pr.jk(0, lists=True, pmode=2, taup=taup)
    scale = max(1.0, np.abs(J0).max(), np.abs(K0).max())
    # a real split: both modes carry work
    assert np.abs(J1).max() > 1e-3 * scale and np.abs(J2).max() > 0.0
    assert np.abs(J1 + J2 - J0).max() <= 1e-12 * scale and np.abs(K1 + K2 - K0).max() <= 1e-12 * scale
    # the cut part in FP32: its error is FP32 rounding of that part alone
    J2f, K2f = pr.jk(1, lists=True, pmode=2, taup=taup)
    part = max(np.abs(J2).max(), np.abs(K2).max())
    assert np.abs(J2f - J2).max() <= 2e-6 * part and np.abs(K2f - K2).max() <= 2e-6 * part
    J1d, K1d = pr.jk(3, lists=True, pmode=1, taup=taup)
    assert np.abs(J1d + J2f - Jo).max() <= 2e-6 * part + 1e-10 * scale
    assert np.abs(K1d + K2f - Ko).max() <= 2e-6 * part + 1e-10 * scale
    # a cut of zero keeps everything in mode 1 (and nothing in mode 2)
    Jz, Kz = pr.jk(0, lists=True, pmode=2, taup=0.0)
    assert np.abs(Jz).max() == 0.0 and np.abs(Kz).max() == 0.0


@pytest.mark.parametrize("seed,shells,natom,kmax", [(83, [0, 1, 2], 2, 3), (84, [1, 3], 2, 2)])
def test_emulated_gradient_primitive_split(seed, shells, natom, kmax):
    """The derivative kernels' primitive modes (the mixed gradient's FP64 list
    split at a primitive cut): FP64 mode 1 + FP64 mode 2 equals the unsplit
    FP64 gradient, and FP64 mode 1 + FP32 mode 2 stays within FP32 rounding of
    the part below the cut."""
    mol, D = _mol(seed, shells, natom, kmax)
    pr = kernel_emu.Problem(mol, D, oracle, lmax=max(shells), prim_sort=True)
    go = oracle.grad(mol, D, mode="unique")
    g0 = pr.grad(0, lists=True)
    scale = max(1.0, np.abs(go).max())
    assert np.abs(g0 - go).max() <= 1e-10 * scale
    taup = 1e-4
    g1 = pr.grad(0, lists=True, pmode=1, taup=taup)
    g2 = pr.grad(0, lists=True, pmode=2, taup=taup)
    assert np.abs(g1).max() > 1e-3 * scale and np.abs(g2).max() > 0.0
    assert np.abs(g1 + g2 - g0).max() <= 1e-12 * scale
    g2f = pr.grad(1, lists=True, pmode=2, taup=taup)
    assert np.abs(g2f - g2).max() <= 2e-6 * max(np.abs(g2).max(), 1e-300)
