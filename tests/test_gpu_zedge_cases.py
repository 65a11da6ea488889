"""GPU edge cases of the J/K path (through the C ABI): a one-function basis,
a basis whose every pair is screened out, a zero density in the mixed path,
and a batch that mixes such molecules with an ordinary one."""
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


def _one_s_shell(nprim=1):
    exps = np.array([1.3, 0.4, 0.1][:nprim])
    coefs = np.array([0.7, 0.4, 0.2][:nprim])
    return molgen.Molecule(np.array([[0.1, -0.2, 0.3]]), np.array([0], np.int32), np.array([0], np.int32),
                           np.array([nprim], np.int32), np.array([0], np.int32), exps, coefs)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nprim", [1, 3])
def test_one_basis_function(g, prec, nprim):
    """nbf = 1: one pair, one quartet, J = K = (ss|ss) D (a mixed build runs
    the quartet's small primitive quartets in FP32: the mixed target, 1e-6 Eh)."""
    mol = _one_s_shell(nprim)
    pairs = g.ShellPairs(mol)
    assert (pairs.nbf, pairs.npairs, pairs.nquartets) == (1, 1, 1)
    D = np.array([[0.8]])
    Dt = torch.from_numpy(D).cuda()
    J, K = g.jk_build(pairs, Dt, prec)
    E = g.jk_energy(Dt, J, K)
    Jo, Ko, _ = oracle.jk(mol, D, mode="all")
    tol = 1e-10 * Jo[0, 0] if prec == "fp64" else 1e-6
    assert abs(float(J[0, 0]) - Jo[0, 0]) <= tol
    assert abs(float(K[0, 0]) - Ko[0, 0]) <= tol
    assert abs(E - oracle.energy(D, Jo, Ko)) <= (1e-10 * abs(E) if prec == "fp64" else 1e-6)
    gr = g.jk_grad(pairs, Dt, "fp64").cpu().numpy()
    assert np.abs(gr).max() <= 1e-12 * abs(E)  # one centre: no geometry dependence


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_everything_screened_out(g, prec):
    """A threshold above every Schwarz product keeps no pair: J = K = 0
    exactly, E = 0, zero gradient."""
    mol, D = molgen.config(0)
    pairs = g.ShellPairs(mol, 1e3)
    assert pairs.npairs == 0 and pairs.nquartets == 0 and pairs.nbf == 20
    Dt = torch.from_numpy(D).cuda()
    J = torch.full_like(Dt, 7.0)
    K = torch.full_like(Dt, 7.0)
    g.jk_build(pairs, Dt, prec, J, K)
    assert int(torch.count_nonzero(J)) == 0 and int(torch.count_nonzero(K)) == 0
    assert g.jk_energy(Dt, J, K) == 0.0
    if prec == "mixed":
        assert g.last_split(pairs) == (0, 0)
    assert int(torch.count_nonzero(g.jk_grad(pairs, Dt, "fp64"))) == 0


def test_zero_density_mixed(g):
    """D = 0: every density-weighted bound is 0 < tau, so every quartet takes
    the FP32 path, and J = K = 0 exactly."""
    mol, _ = molgen.config(0)
    pairs = g.ShellPairs(mol)
    Dt = torch.zeros((pairs.nbf, pairs.nbf), dtype=torch.float64, device="cuda")
    J, K = g.jk_build(pairs, Dt, "mixed")
    n32, n64 = g.last_split(pairs)
    assert (n32, n64) == (pairs.nquartets, 0)
    assert int(torch.count_nonzero(J)) == 0 and int(torch.count_nonzero(K)) == 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_with_degenerate_molecules(g, prec):
    """One launch sequence over an ordinary molecule, a one-function molecule
    and a molecule with no surviving pair: each result equals its own
    single-molecule build (a mixed build's FP32 sums are grouped over other
    warp lanes in a batch: FP32 rounding)."""
    mol0, D0 = molgen.config(0)
    mol1 = _one_s_shell(3)
    D1 = np.array([[0.6]])
    plist = [g.ShellPairs(mol0), g.ShellPairs(mol1), g.ShellPairs(mol0, 1e3)]
    Ds = [torch.from_numpy(D).cuda() for D in (D0, D1, D0)]
    Js, Ks = g.jk_build_batched(plist, Ds, precision=prec)
    for p, D, Jb, Kb in zip(plist, Ds, Js, Ks):
        J, K = g.jk_build(p, D, prec)
        scale = max(1.0, float(J.abs().max())) * (1e-10 if prec == "fp64" else 1e-6)
        assert float((Jb - J).abs().max()) <= scale
        assert float((Kb - K).abs().max()) <= scale
    assert int(torch.count_nonzero(Js[2])) == 0 and int(torch.count_nonzero(Ks[2])) == 0


def test_batch_plan_does_not_outlive_its_handles(g):
    """A batch plan is cached by its handles and matrices; a handle freed and
    replaced (whose host address may come back) must not reuse the old plan:
    the batched result of the new molecule equals its own build."""
    mol, D = molgen.config(0)
    Dt = torch.from_numpy(D).cuda()
    J = torch.empty_like(Dt)
    K = torch.empty_like(Dt)
    p = g.ShellPairs(mol)
    g.jk_build_batched([p], [Dt], [J], [K], "fp64")
    p.free()
    moved = mol.with_xyz(mol.xyz * 1.1)  # same basis size, other integrals
    q = g.ShellPairs(moved)
    g.jk_build_batched([q], [Dt], [J], [K], "fp64")
    J1, K1 = g.jk_build(q, Dt, "fp64")
    assert float((J - J1).abs().max()) <= 1e-12 * float(J1.abs().max())
    assert float((K - K1).abs().max()) <= 1e-12 * float(K1.abs().max())
