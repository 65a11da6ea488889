"""The allocation-free energy entry point (jk_energy_noalloc) against the
regular one (jk_energy), through the C ABI, on two calls in a row.

jk_energy_noalloc serves callers that cannot allocate device memory (their
own allocator owns the whole budget, or cudaMalloc's synchronisation is not
acceptable in their loop); it reduces through a fixed library-owned scratch
array instead.  This file is collected last on purpose."""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_13203_gb300 as g
    g.load()
    return g


def _sym(n, seed):
    gen = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn((n, n), generator=gen, device="cuda", dtype=torch.float64)
    return (x + x.T).contiguous()


def test_noalloc_energy_matches_regular_entry_point(g):
    # two calls in a row with different sizes: the shared scratch keeps the
    # previous call's partials, which must not leak into the next result
    for seed, n in ((11, 517), (12, 130)):
        D, J, K = _sym(n, seed), _sym(n, seed + 1), _sym(n, seed + 2)
        e_ref = g.jk_energy(D, J, K)
        e_na = g.jk_energy_noalloc(D, J, K)
        assert abs(e_na - e_ref) <= 1e-10 * max(1.0, abs(e_ref)), (n, e_na, e_ref)


def test_noalloc_energy_of_a_jk_build(g):
    import molgen
    mol, D = molgen.config(0)
    pairs = g.ShellPairs(mol)
    Dt = torch.from_numpy(D).cuda()
    J, K = g.jk_build(pairs, Dt, "fp64")
    for _ in range(2):
        assert abs(g.jk_energy_noalloc(Dt, J, K) - g.jk_energy(Dt, J, K)) <= 1e-10
    pairs.free()


def test_noalloc_rejects_oversize(g):
    # rejected on the host before any device work
    lib = g.load()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    E = ctypes.c_double()
    p = ctypes.c_void_p(x.data_ptr())
    rc = lib.jk_energy_noalloc(16384, p, p, p, ctypes.byref(E), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1 and b"exceeds" in lib.jk_last_error()
