"""Host-side argument checks of the C ABI (no GPU needed).

Every entry point validates its arguments (and shellpairs_build the whole
basis) on the host before the first CUDA call, so a bad call returns a
negative status with a message and never reaches the device.  These tests exercise exactly those paths through the exported
symbols; nothing here launches a kernel or touches a CUDA context."""
import ctypes as C
import math

import numpy as np
import pytest

JK_OK, JK_ERR_INVALID = 0, -1
JK_FP64, JK_MIXED = 0, 1
OPT_TAU, OPT_TSMALL = 0, 1


@pytest.fixture(scope="module")
def lib():
    import paper_2412_13203_gb300 as g
    return g.load()


def err(lib):
    return lib.jk_last_error().decode()


def molecule_arrays(natom=2):
    """A valid two-atom, two-shell (s, p) input; tests corrupt one field."""
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.4]][:natom], dtype=np.float64)
    atom = np.array([0, natom - 1], dtype=np.int32)
    l = np.array([0, 1], dtype=np.int32)
    nprim = np.array([2, 1], dtype=np.int32)
    off = np.array([0, 2], dtype=np.int32)
    exps = np.array([3.4, 0.62, 0.8], dtype=np.float64)
    coefs = np.array([0.15, 0.53, 1.0], dtype=np.float64)
    return dict(xyz=xyz, atom=atom, l=l, nprim=nprim, off=off, exps=exps, coefs=coefs)


def structs(a, natom=None, nshell=None, drop=None):
    import paper_2412_13203_gb300 as g
    ptr = {k: (None if k == drop else v.ctypes.data) for k, v in a.items()}
    atoms = g._Atoms(a["xyz"].shape[0] if natom is None else natom, ptr["xyz"])
    shells = g._Shells(a["atom"].shape[0] if nshell is None else nshell, ptr["atom"], ptr["l"], ptr["nprim"],
                       ptr["off"], ptr["exps"], ptr["coefs"])
    return atoms, shells


def build(lib, atoms, shells, thresh=1e-12):
    h = C.c_void_p(1234)  # must be reset to NULL on failure
    rc = lib.shellpairs_build(C.byref(atoms), C.byref(shells), thresh, C.byref(h), None)
    return rc, h


def test_shellpairs_build_null_arguments(lib):
    a = molecule_arrays()
    atoms, shells = structs(a)
    h = C.c_void_p()
    assert lib.shellpairs_build(None, C.byref(shells), 1e-12, C.byref(h), None) == JK_ERR_INVALID
    assert "null" in err(lib)
    assert lib.shellpairs_build(C.byref(atoms), None, 1e-12, C.byref(h), None) == JK_ERR_INVALID
    assert lib.shellpairs_build(C.byref(atoms), C.byref(shells), 1e-12, None, None) == JK_ERR_INVALID


@pytest.mark.parametrize("natom", [0, -3])
def test_shellpairs_build_rejects_empty_molecule(lib, natom):
    atoms, shells = structs(molecule_arrays(), natom=natom)
    rc, h = build(lib, atoms, shells)
    assert rc == JK_ERR_INVALID and h.value is None
    assert "no atoms" in err(lib)


@pytest.mark.parametrize("nshell", [0, -1])
def test_shellpairs_build_rejects_empty_basis(lib, nshell):
    atoms, shells = structs(molecule_arrays(), nshell=nshell)
    rc, h = build(lib, atoms, shells)
    assert rc == JK_ERR_INVALID and h.value is None
    assert "no shells" in err(lib)


@pytest.mark.parametrize("field", ["xyz", "atom", "l", "nprim", "off", "exps", "coefs"])
def test_shellpairs_build_rejects_missing_array(lib, field):
    atoms, shells = structs(molecule_arrays(), drop=field)
    rc, h = build(lib, atoms, shells)
    assert rc == JK_ERR_INVALID and h.value is None


@pytest.mark.parametrize("thresh", [math.nan, math.inf, -math.inf])
def test_shellpairs_build_rejects_non_finite_threshold(lib, thresh):
    atoms, shells = structs(molecule_arrays())
    rc, h = build(lib, atoms, shells, thresh)
    assert rc == JK_ERR_INVALID and h.value is None
    assert "threshold" in err(lib)


def test_builds_reject_null_handle(lib):
    buf = (C.c_double * 4)()
    p = C.cast(buf, C.c_void_p)
    assert lib.jk_build(None, p, p, p, JK_FP64, None) == JK_ERR_INVALID
    assert "null" in err(lib)
    assert lib.jk_grad(None, p, p, JK_FP64, None) == JK_ERR_INVALID
    assert lib.jk_autotune(None, p, p, p, JK_MIXED, None) == JK_ERR_INVALID


def test_batched_argument_checks(lib):
    arr = C.c_void_p * 1
    null1 = arr(None)
    # no molecules: nothing to do, and no device work
    assert lib.jk_build_batched(0, None, None, None, None, JK_FP64, None) == JK_OK
    assert lib.jk_build_batched(-1, None, None, None, None, JK_FP64, None) == JK_ERR_INVALID
    assert lib.jk_build_batched(1, None, null1, null1, null1, JK_FP64, None) == JK_ERR_INVALID
    assert lib.jk_build_batched(1, null1, null1, null1, null1, 7, None) == JK_ERR_INVALID
    assert "precision" in err(lib)
    assert lib.jk_build_batched(1, null1, null1, null1, null1, JK_MIXED, None) == JK_ERR_INVALID
    assert "null molecule entry" in err(lib)


def test_energy_argument_checks(lib):
    buf = (C.c_double * 4)()
    p = C.cast(buf, C.c_void_p)
    E = C.c_double(5.0)
    for n in (0, -2):
        assert lib.jk_energy(n, p, p, p, C.byref(E), None) == JK_ERR_INVALID
        assert lib.jk_energy_noalloc(n, p, p, p, C.byref(E), None) == JK_ERR_INVALID
    assert lib.jk_energy(2, p, p, p, None, None) == JK_ERR_INVALID
    # the allocation-free reduction has a fixed scratch of 16383 rows
    assert lib.jk_energy_noalloc(16384, p, p, p, C.byref(E), None) == JK_ERR_INVALID
    assert "16383" in err(lib) and "jk_energy" in err(lib)
    assert E.value == 5.0


@pytest.mark.parametrize("L,n", [(-1, 4), (14, 4), (0, -1)])
def test_boys_argument_checks(lib, L, n):
    buf = (C.c_double * 4)()
    p = C.cast(buf, C.c_void_p)
    assert lib.jk_boys(L, n, p, p, JK_FP64, None) == JK_ERR_INVALID


def test_boys_rejects_null_buffers(lib):
    assert lib.jk_boys(2, 3, None, None, JK_FP64, None) == JK_ERR_INVALID


def test_options_round_trip_and_validation(lib):
    v = C.c_double()
    assert lib.jk_get_option(OPT_TAU, C.byref(v)) == JK_OK
    tau0 = v.value
    assert tau0 == pytest.approx(5e-3)
    assert lib.jk_get_option(10, C.byref(v)) == JK_OK and v.value == pytest.approx(1e-4)  # JK_OPT_PRIM_TAU
    assert lib.jk_get_option(11, C.byref(v)) == JK_OK and v.value == pytest.approx(1e-6)  # JK_OPT_GRAD_PRIM_TAU
    for bad in (-1e-3, math.nan, math.inf):
        assert lib.jk_set_option(10, bad) == JK_ERR_INVALID
        assert lib.jk_set_option(11, bad) == JK_ERR_INVALID
    try:
        assert lib.jk_set_option(OPT_TAU, 3e-3) == JK_OK
        assert lib.jk_get_option(OPT_TAU, C.byref(v)) == JK_OK and v.value == 3e-3
        for bad in (-1e-3, math.nan):
            assert lib.jk_set_option(OPT_TAU, bad) == JK_ERR_INVALID
            assert lib.jk_get_option(OPT_TAU, C.byref(v)) == JK_OK and v.value == 3e-3
        assert lib.jk_set_option(OPT_TSMALL, -0.5) == JK_ERR_INVALID
    finally:
        assert lib.jk_set_option(OPT_TAU, tau0) == JK_OK
    assert lib.jk_set_option(99, 1.0) == JK_ERR_INVALID and "unknown option" in err(lib)
    assert lib.jk_get_option(99, C.byref(v)) == JK_ERR_INVALID
    assert lib.jk_get_option(OPT_TAU, None) == JK_ERR_INVALID


def test_handle_queries_reject_null(lib):
    i64 = C.c_int64()
    i32 = C.c_int()
    assert lib.jk_last_split(None, C.byref(i64), C.byref(i64)) == JK_ERR_INVALID
    assert lib.jk_last_launches(None, C.byref(i64)) == JK_ERR_INVALID
    assert lib.jk_tuning(None, 0, None, C.byref(i32)) == JK_ERR_INVALID
    assert lib.jk_set_tuning(None, 0, None) == JK_ERR_INVALID
    assert lib.jk_class_stats(None, 0, None, C.byref(i32)) == JK_ERR_INVALID
    assert lib.jk_split_stats(None, 0, None, C.byref(i32)) == JK_ERR_INVALID
    assert lib.jk_profile(None, 0, None, C.byref(i32)) == JK_ERR_INVALID
    lib.shellpairs_free(None)  # freeing NULL is a no-op


def test_fma_peak_argument_checks(lib):
    f = C.c_double()
    assert lib.jk_fma_peak(JK_FP64, 0, C.byref(f), None) == JK_ERR_INVALID
    assert lib.jk_fma_peak(JK_FP64, 100, None, None) == JK_ERR_INVALID


def corrupt(a, field, idx, value):
    b = {k: v.copy() for k, v in a.items()}
    b[field][idx] = value
    return b


@pytest.mark.parametrize("field,idx,value,code,word", [
    ("l", 1, -1, JK_ERR_INVALID, "negative angular momentum"),
    ("l", 1, 4, -5, "angular momentum"),
    ("nprim", 0, 0, JK_ERR_INVALID, "without primitives"),
    ("atom", 1, 2, JK_ERR_INVALID, "atom out of range"),
    ("atom", 0, -1, JK_ERR_INVALID, "atom out of range"),
    ("off", 1, -2, JK_ERR_INVALID, "negative primitive offset"),
    ("exps", 1, 0.0, JK_ERR_INVALID, "exponent"),
    ("exps", 2, -0.3, JK_ERR_INVALID, "exponent"),
    ("exps", 0, math.nan, JK_ERR_INVALID, "exponent"),
    ("coefs", 2, math.inf, JK_ERR_INVALID, "coefficient"),
    ("xyz", (1, 2), math.nan, JK_ERR_INVALID, "coordinate"),
])
def test_shellpairs_build_rejects_malformed_basis(lib, field, idx, value, code, word):
    """The basis checks run on the host before the first CUDA call, so they
    report the same status whether or not a device is present."""
    a = corrupt(molecule_arrays(), field, idx, value)  # keeps the arrays alive during the call
    atoms, shells = structs(a)
    rc, h = build(lib, atoms, shells)
    assert rc == code and h.value is None
    assert word in err(lib)


def test_density_screen_option(lib):
    OPT_SCREEN = 5
    v = C.c_double(-1.0)
    assert lib.jk_get_option(OPT_SCREEN, C.byref(v)) == JK_OK and v.value == 0.0  # off by default
    try:
        assert lib.jk_set_option(OPT_SCREEN, 1e-9) == JK_OK
        assert lib.jk_get_option(OPT_SCREEN, C.byref(v)) == JK_OK and v.value == 1e-9
        for bad in (-1e-12, math.nan, math.inf):
            assert lib.jk_set_option(OPT_SCREEN, bad) == JK_ERR_INVALID
            assert "density screening" in err(lib)
        assert lib.jk_get_option(OPT_SCREEN, C.byref(v)) == JK_OK and v.value == 1e-9
    finally:
        assert lib.jk_set_option(OPT_SCREEN, 0.0) == JK_OK


def test_new_entry_points_reject_null_arguments(lib):
    buf = (C.c_double * 4)()
    p = C.cast(buf, C.c_void_p)
    n = C.c_int(-7)
    assert lib.jk_sph_nbf(None, C.byref(n)) == JK_ERR_INVALID and n.value == -7
    assert lib.jk_sph_transform(None, 0, p, p, None) == JK_ERR_INVALID
    assert "null" in err(lib)
    assert lib.jk_one_electron(None, p, p, p, p, None) == JK_ERR_INVALID
    assert "null" in err(lib)


def test_limits(lib):
    import paper_2412_13203_gb300 as g
    assert g.limits() == {"lmax": 3, "grad_lmax": 3}
    assert lib.jk_limits(None, None) == JK_ERR_INVALID
