"""Parity at the benchmark's full size (32-atom lattice, 480 Cartesian basis
functions, Schwarz 1e-10) in the configuration bench.py times: one sampled
row of J and K (an s shell, all 480 columns) from the oracle, which sums the
definition over every (not only unique) screened shell quartet, against the
GPU FP64 and mixed builds."""
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


def test_bench_workload_sampled_row(g):
    mol, D = molgen.config(1)
    thresh = molgen.CONFIG_THRESH[1]
    pairs = g.ShellPairs(mol, thresh)
    Dt = torch.from_numpy(D).cuda()
    J64, K64 = g.jk_build(pairs, Dt, "fp64")
    J64, K64 = J64.cpu().numpy(), K64.cpu().numpy()
    Jm, Km = g.jk_build(pairs, Dt, "mixed")
    Jm, Km = Jm.cpu().numpy(), Km.cpu().numpy()
    shell = int(np.where(np.asarray(mol.shell_l) == 0)[0][5])
    row = int(sum((int(l) + 1) * (int(l) + 2) // 2 for l in mol.shell_l[:shell]))
    Jr, Kr = oracle.jk_rows(mol, D, [shell], thresh)
    # quartets whose Schwarz product lies within the last bits of the threshold
    # may be kept on one side and dropped on the other; each moves an element
    # by at most thresh * max|D|
    Q = oracle.schwarz(mol)
    qa = Q[shell]
    amb = np.abs(np.outer(qa, Q.ravel()) - thresh) <= 1e-8 * thresh
    flips = 2 * thresh * np.abs(D).max() * int(amb.sum())
    # FP64 tolerance 1e-10 relative to the largest element (as in the other FP64
    # parity tests: an element here sums ~1e6 quartet contributions of size ~1)
    tolJ = 1e-10 * max(1.0, np.abs(Jr).max()) + flips
    tolK = 1e-10 * max(1.0, np.abs(Kr).max()) + flips
    assert np.abs(J64[row] - Jr[0]).max() <= tolJ, np.abs(J64[row] - Jr[0]).max()
    assert np.abs(K64[row] - Kr[0]).max() <= tolK, np.abs(K64[row] - Kr[0]).max()
    assert np.abs(Jm[row] - Jr[0]).max() <= 1e-6
    assert np.abs(Km[row] - Kr[0]).max() <= 1e-6
    # and the whole matrices: symmetric, mixed within the target of FP64
    assert np.abs(J64 - J64.T).max() == 0.0 and np.abs(K64 - K64.T).max() == 0.0
    assert np.abs(Jm - J64).max() <= 1e-6 and np.abs(Km - K64).max() <= 1e-6
    pairs.free()
