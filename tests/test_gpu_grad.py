"""GPU parity of the nuclear-gradient adjoint kernel: against the oracle's
analytic FP64 gradient (small molecules, every class up to d), central finite
differences of the GPU energy (24-atom workload, h = 1e-4 bohr), and the
torch.autograd.Function wrapper."""
import numpy as np
import pytest

import molgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_13203_gb300 as g
    g.load()
    return g


@pytest.mark.parametrize("seed,shells,natom,kmax", [(1, [0, 1], 3, 2), (2, [2, 0], 3, 3), (3, [1, 2], 2, 3),
                                                    (4, [0, 1, 2], 3, 2)])
def test_gradient_matches_oracle(g, seed, shells, natom, kmax):
    mol = molgen.random_molecule(300 + seed, natom, shells, 1, kmax, 0.1, 50.0, layout="lattice", spacing=1.8)
    D = molgen.density(mol, 400 + seed)
    pairs = g.ShellPairs(mol)
    gg = g.jk_grad(pairs, torch.from_numpy(D).cuda(), "fp64").cpu().numpy()
    go = oracle.grad(mol, D, mode="unique")
    scale = max(1.0, np.abs(go).max())
    assert np.abs(gg - go).max() <= 1e-10 * scale, (gg, go)
    assert np.abs(gg.sum(axis=0)).max() <= 1e-10 * scale


def test_gradient_fd_24_atoms(g):
    mol, D = molgen.config(3)
    thresh = molgen.CONFIG_THRESH[3]
    Dt = torch.from_numpy(D).cuda()
    pairs = g.ShellPairs(mol, thresh)
    grad = g.jk_grad(pairs, Dt, "fp64").cpu().numpy()
    pairs.free()
    assert grad.shape == (24, 3)
    assert np.abs(grad.sum(axis=0)).max() <= 1e-8 * np.abs(grad).max()
    h = 1e-4

    def energy(xyz):
        p = g.ShellPairs(mol.with_xyz(xyz), thresh)
        J, K = g.jk_build(p, Dt, "fp64")
        e = g.jk_energy(Dt, J, K)
        p.free()
        return e
    for a, x in [(0, 0), (13, 2)]:
        xp, xm = mol.xyz.copy(), mol.xyz.copy()
        xp[a, x] += h
        xm[a, x] -= h
        fd = (energy(xp) - energy(xm)) / (2 * h)
        assert abs(fd - grad[a, x]) <= 1e-5 * max(1.0, abs(grad[a, x])), (a, x, fd, grad[a, x])


def test_autograd_function(g):
    mol = molgen.random_molecule(77, 3, [0, 1, 2], 1, 2, 0.2, 20.0, layout="lattice", spacing=2.0)
    D = molgen.density(mol, 78)
    xyz = torch.tensor(mol.xyz, dtype=torch.float64, device="cuda", requires_grad=True)
    Dt = torch.tensor(D, dtype=torch.float64, device="cuda", requires_grad=True)
    E = g.jk_energy_fn(xyz, Dt, mol)
    E.backward()
    go = oracle.grad(mol, D, mode="unique")
    assert np.abs(xyz.grad.cpu().numpy() - go).max() <= 1e-10 * max(1.0, np.abs(go).max())
    Jo, Ko, _ = oracle.jk(mol, D, mode="unique")
    e = float(E.detach())
    assert abs(e - oracle.energy(D, Jo, Ko)) <= 1e-10 * max(1.0, abs(e))
    assert np.abs(Dt.grad.cpu().numpy() - (Jo - 0.5 * Ko)).max() <= 1e-10 * max(1.0, np.abs(Jo).max())


@pytest.mark.parametrize("seed,shells,natom,kmax", [(4, [0, 1, 2], 3, 2), (5, [0, 0, 1, 2], 4, 4)])
def test_mixed_gradient_matches_oracle(g, seed, shells, natom, kmax):
    """Mixed-precision gradient: the derivative integrals of the quartets
    whose density-weighted bound is below grad_tau in FP32 (added to dE/dR in
    FP64), the others FP64 -- within 1e-6 of the oracle's analytic gradient.
    With grad_tau above every bound (all FP32) the FP32 kernels alone are
    held to the same relative accuracy as the FP32 J/K kernels."""
    mol = molgen.random_molecule(300 + seed, natom, shells, 1, kmax, 0.1, 50.0, layout="lattice", spacing=1.8)
    D = molgen.density(mol, 400 + seed)
    pairs = g.ShellPairs(mol)
    Dt = torch.from_numpy(D).cuda()
    go = oracle.grad(mol, D, mode="unique")
    scale = max(1.0, np.abs(go).max())
    tau = g.get_option("grad_tau")
    both = False
    try:
        for t in (tau, 1e-2):
            g.set_option("grad_tau", t)
            gm = g.jk_grad(pairs, Dt, "mixed").cpu().numpy()
            n32, n64 = g.last_split(pairs)
            assert n32 + n64 == pairs.nquartets
            both = both or (n32 > 0 and n64 > 0)
            assert np.abs(gm - go).max() <= 1e-6, (t, np.abs(gm - go).max())
            assert np.abs(gm.sum(axis=0)).max() <= 1e-8 * scale
        assert both  # some setting ran both precisions
        g.set_option("grad_tau", 1e30)
        ga = g.jk_grad(pairs, Dt, "mixed").cpu().numpy()
        assert g.last_split(pairs)[1] == 0
        assert np.abs(ga - go).max() <= 2e-6 * scale
    finally:
        g.set_option("grad_tau", tau)
    pairs.free()


def test_mixed_gradient_24_atoms(g):
    """The 24-atom workload: mixed gradient within 1e-6 of the FP64 one (itself
    pinned to the oracle above), and its parts sum to it."""
    mol, D = molgen.config(3)
    pairs = g.ShellPairs(mol, molgen.CONFIG_THRESH[3])
    Dt = torch.from_numpy(D).cuda()
    g64 = g.jk_grad(pairs, Dt, "fp64")
    gm = g.jk_grad(pairs, Dt, "mixed")
    assert float((gm - g64).abs().max()) <= 1e-6, float((gm - g64).abs().max())
    gs = sum(g.jk_grad_part(pairs, Dt, p, 2, "mixed") for p in range(2))
    assert float((gs - gm).abs().max()) <= 1e-9 * float(gm.abs().max())
    pairs.free()


@pytest.mark.parametrize("seed,shells,natom,kmax", [(6, [0, 1, 2], 3, 4), (7, [1, 3], 2, 2)])
def test_gradient_primitive_split(g, seed, shells, natom, kmax):
    """The primitive split of the mixed gradient's FP64 list (JK_OPT_GRAD_PRIM_TAU)
    with every quartet FP64-selected (grad_tau 0): a vanishing cut gives the
    unsplit FP64 gradient, an unreachable one the FP32 derivative kernels
    alone (FP32 rounding of the oracle), the default cut the oracle to 1e-6."""
    mol = molgen.random_molecule(300 + seed, natom, shells, 1, kmax, 0.1, 50.0, layout="lattice", spacing=1.8)
    D = molgen.density(mol, 400 + seed)
    pairs = g.ShellPairs(mol)
    Dt = torch.from_numpy(D).cuda()
    go = oracle.grad(mol, D, mode="unique")
    scale = max(1.0, np.abs(go).max())
    old = {k: g.get_option(k) for k in ("grad_tau", "grad_prim_tau")}
    out = {}
    try:
        g.set_option("grad_tau", 0.0)
        for pt in (0.0, 1e-300, 1e300, old["grad_prim_tau"]):
            g.set_option("grad_prim_tau", pt)
            out[pt] = g.jk_grad(pairs, Dt, "mixed").cpu().numpy()
            assert g.last_split(pairs)[1] == pairs.nquartets
    finally:
        for k, v in old.items():
            g.set_option(k, v)
    assert np.abs(out[0.0] - go).max() <= 1e-10 * scale
    assert np.abs(out[1e-300] - out[0.0]).max() <= 1e-12 * scale
    assert np.abs(out[1e300] - go).max() <= 2e-6 * scale
    assert np.abs(out[old["grad_prim_tau"]] - go).max() <= 1e-6
    pairs.free()
