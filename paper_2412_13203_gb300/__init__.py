"""Python binding of the GB300 screened-ERI / J-K / gradient library.

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in ``include/gb300_eri.h``.  PyTorch
provides device memory and streams.  There is no CPU fallback: if the shared
library has not been built (``paper_2412_13203_gb300.build.build()``) or no
CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgb300eri.so")

JK_OPT = {"mixed_tau": 0, "mixed_tsmall": 1, "check_symmetry": 2, "graph": 3, "profile": 4, "density_screen": 5,
          "rpath": 6, "fail_alloc_after": 7, "grad_tau": 8, "df_tier": 9, "prim_tau": 10, "grad_prim_tau": 11}
_PREC = {"fp64": 0, "mixed": 1}

_lib = None
_lock = threading.Lock()


class JKError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class _Atoms(C.Structure):
    _fields_ = [("natom", C.c_int), ("xyz", C.c_void_p)]


class _Shells(C.Structure):
    _fields_ = [("nshell", C.c_int), ("atom", C.c_void_p), ("l", C.c_void_p), ("nprim", C.c_void_p),
                ("prim_offset", C.c_void_p), ("exps", C.c_void_p), ("coefs", C.c_void_p)]


EXPORTS = ["shellpairs_build", "shellpairs_info", "jk_build", "jk_grad", "jk_build_batched", "jk_energy", "jk_boys",
           "jk_energy_noalloc",
           "jk_set_option", "jk_get_option", "jk_last_split", "shellpairs_free", "jk_last_error",
           "jk_class_stats", "jk_profile", "jk_fma_peak", "jk_last_launches", "jk_autotune", "jk_tuning",
           "jk_set_tuning", "jk_split_stats", "jk_sph_nbf", "jk_sph_transform",
           "jk_one_electron", "jk_limits", "jk_build_part", "jk_grad_part", "jk_partition", "jk_part_rows"]


def load():
    """Load the compiled library (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing; run paper_2412_13203_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        vp, i64p = C.c_void_p, C.POINTER(C.c_int64)
        lib.shellpairs_build.argtypes = [C.POINTER(_Atoms), C.POINTER(_Shells), C.c_double, C.POINTER(vp), vp]
        lib.shellpairs_info.argtypes = [vp, C.POINTER(C.c_int), i64p, i64p, i64p]
        lib.jk_build.argtypes = [vp, vp, vp, vp, C.c_int, vp]
        lib.jk_grad.argtypes = [vp, vp, vp, C.c_int, vp]
        lib.jk_build_batched.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.c_int, vp]
        lib.jk_energy.argtypes = [C.c_int, vp, vp, vp, C.POINTER(C.c_double), vp]
        lib.jk_energy_noalloc.argtypes = [C.c_int, vp, vp, vp, C.POINTER(C.c_double), vp]
        lib.jk_boys.argtypes = [C.c_int, C.c_int, vp, vp, C.c_int, vp]
        lib.jk_set_option.argtypes = [C.c_int, C.c_double]
        lib.jk_get_option.argtypes = [C.c_int, C.POINTER(C.c_double)]
        lib.jk_last_split.argtypes = [vp, i64p, i64p]
        lib.jk_last_launches.argtypes = [vp, i64p]
        lib.jk_autotune.argtypes = [vp, vp, vp, vp, C.c_int, vp]
        lib.jk_tuning.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        lib.jk_set_tuning.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
        lib.jk_class_stats.argtypes = [vp, C.c_int, i64p, C.POINTER(C.c_int)]
        lib.jk_split_stats.argtypes = [vp, C.c_int, i64p, C.POINTER(C.c_int)]
        lib.jk_profile.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)]
        lib.jk_fma_peak.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double), vp]
        lib.jk_one_electron.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.jk_limits.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int)]
        lib.jk_build_part.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp, C.c_int, vp]
        lib.jk_grad_part.argtypes = [vp, C.c_int, C.c_int, vp, vp, C.c_int, vp]
        lib.jk_partition.argtypes = [C.c_int64, C.POINTER(C.c_double), C.c_int, i64p]
        lib.jk_part_rows.argtypes = [vp, C.c_int, C.c_int, i64p, C.POINTER(C.c_int)]
        lib.jk_sph_nbf.argtypes = [vp, C.POINTER(C.c_int)]
        lib.jk_sph_transform.argtypes = [vp, C.c_int, vp, vp, vp]
        lib.shellpairs_free.argtypes = [vp]
        lib.shellpairs_free.restype = None
        lib.jk_last_error.restype = C.c_char_p
        _lib = lib
    return _lib


def _check(rc):
    if rc != 0:
        raise JKError(rc, load().jk_last_error().decode())


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype_name="float64"):
    import torch
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.dtype != getattr(torch, dtype_name) or not t.is_contiguous():
        raise ValueError(f"expected a contiguous {dtype_name} tensor")
    return C.c_void_p(t.data_ptr())


class ShellPairs:
    """Library-owned shell pairs, Schwarz factors and quartet work lists of one
    molecule (``shellpairs_build``).  ``mol`` provides xyz, shell_atom,
    shell_l, shell_nprim, shell_prim_offset, exps and raw coefs arrays."""

    def __init__(self, mol, thresh: float | None = None, stream=None):
        lib = load()
        self._keep = [np.ascontiguousarray(mol.xyz, dtype=np.float64)]
        ints = [np.ascontiguousarray(getattr(mol, n), dtype=np.int32)
                for n in ("shell_atom", "shell_l", "shell_nprim", "shell_prim_offset")]
        dbls = [np.ascontiguousarray(mol.exps, dtype=np.float64), np.ascontiguousarray(mol.coefs, dtype=np.float64)]
        self._keep += ints + dbls
        atoms = _Atoms(self._keep[0].shape[0], self._keep[0].ctypes.data)
        shells = _Shells(ints[0].shape[0], ints[0].ctypes.data, ints[1].ctypes.data, ints[2].ctypes.data,
                         ints[3].ctypes.data, dbls[0].ctypes.data, dbls[1].ctypes.data)
        h = C.c_void_p()
        _check(lib.shellpairs_build(C.byref(atoms), C.byref(shells), float(thresh or 0.0), C.byref(h),
                                    _stream_ptr(stream)))
        self.handle = h
        self.natom = int(self._keep[0].shape[0])
        nbf = C.c_int()
        npair, nq, npq = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib.shellpairs_info(h, C.byref(nbf), C.byref(npair), C.byref(nq), C.byref(npq)))
        self.nbf, self.npairs, self.nquartets, self.nprimquartets = nbf.value, npair.value, nq.value, npq.value
        ns = C.c_int()
        _check(lib.jk_sph_nbf(h, C.byref(ns)))
        self.nsph = ns.value  # basis size with pure d and f shells
        self._keep = None

    def free(self):
        if getattr(self, "handle", None):
            load().shellpairs_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def jk_build(pairs: ShellPairs, D, precision: str = "fp64", J=None, K=None, stream=None):
    """J and K (new or given float64 CUDA tensors, nbf x nbf) for density D."""
    import torch
    n = pairs.nbf
    if tuple(D.shape) != (n, n):
        raise ValueError("D must be nbf x nbf")
    if J is None:
        J = torch.empty((n, n), dtype=torch.float64, device=D.device)
    if K is None:
        K = torch.empty((n, n), dtype=torch.float64, device=D.device)
    _check(load().jk_build(pairs.handle, _dev_ptr(D), _dev_ptr(J), _dev_ptr(K), _PREC[precision], _stream_ptr(stream)))
    return J, K


def jk_energy(D, J, K, stream=None) -> float:
    """E = tr(DJ)/2 - tr(DK)/4 (compensated device reduction)."""
    E = C.c_double()
    _check(load().jk_energy(int(D.shape[0]), _dev_ptr(D), _dev_ptr(J), _dev_ptr(K), C.byref(E), _stream_ptr(stream)))
    return E.value


def jk_energy_noalloc(D, J, K, stream=None) -> float:
    """Same value as jk_energy, computed without any device allocation (a fixed
    library-owned scratch array; nbf <= 16383).  For callers whose device
    memory is entirely owned by their own allocator, or that cannot afford
    cudaMalloc's synchronisation; concurrent calls on different streams race
    on the shared scratch and must be serialised."""
    E = C.c_double()
    _check(load().jk_energy_noalloc(int(D.shape[0]), _dev_ptr(D), _dev_ptr(J), _dev_ptr(K), C.byref(E),
                                    _stream_ptr(stream)))
    return E.value


def jk_grad(pairs: ShellPairs, D, precision: str = "fp64", out=None, stream=None):
    """dE/dR [natom, 3] (float64 CUDA tensor) of E = tr(DJ)/2 - tr(DK)/4 at fixed D."""
    import torch
    if out is None:
        out = torch.empty((pairs.natom, 3), dtype=torch.float64, device=D.device)
    _check(load().jk_grad(pairs.handle, _dev_ptr(D), _dev_ptr(out), _PREC[precision], _stream_ptr(stream)))
    return out


def jk_build_part(pairs: ShellPairs, D, part: int, nparts: int, precision: str = "fp64", J=None, K=None,
                  stream=None):
    """J and K from the quartet rows of part ``part`` of ``nparts`` (every
    class cut into cost-balanced row ranges); the parts sum to jk_build."""
    import torch
    n = pairs.nbf
    if tuple(D.shape) != (n, n):
        raise ValueError("D must be nbf x nbf")
    if J is None:
        J = torch.empty((n, n), dtype=torch.float64, device=D.device)
    if K is None:
        K = torch.empty((n, n), dtype=torch.float64, device=D.device)
    _check(load().jk_build_part(pairs.handle, int(part), int(nparts), _dev_ptr(D), _dev_ptr(J), _dev_ptr(K),
                                _PREC[precision], _stream_ptr(stream)))
    return J, K


def jk_grad_part(pairs: ShellPairs, D, part: int, nparts: int, precision: str = "fp64", out=None, stream=None):
    """dE/dR [natom, 3] from the quartet rows of part ``part`` of ``nparts``."""
    import torch
    if out is None:
        out = torch.empty((pairs.natom, 3), dtype=torch.float64, device=D.device)
    _check(load().jk_grad_part(pairs.handle, int(part), int(nparts), _dev_ptr(D), _dev_ptr(out), _PREC[precision],
                               _stream_ptr(stream)))
    return out


def partition(cost, nparts: int) -> np.ndarray:
    """The library's partition rule on the host (no device work): bounds
    [nparts + 1] of contiguous ranges of equal cost, within one unit's cost."""
    c = np.ascontiguousarray(cost, dtype=np.float64)
    b = np.zeros(int(nparts) + 1, dtype=np.int64)
    _check(load().jk_partition(int(c.shape[0]), c.ctypes.data_as(C.POINTER(C.c_double)), int(nparts),
                               b.ctypes.data_as(C.POINTER(C.c_int64))))
    return b


def prepare_partition(pairs: ShellPairs, nparts: int) -> int:
    """Compute and cache the handle's row partition for nparts parts (one
    synchronisation); returns the number of (class, part) entries."""
    n = C.c_int()
    _check(load().jk_part_rows(pairs.handle, int(nparts), 0, None, C.byref(n)))
    return n.value


def part_rows(pairs: ShellPairs, nparts: int):
    """Row partition of a handle: per class and part, (first row, end row,
    work items, cost, largest row cost of the class)."""
    cap = 64 * int(nparts)
    buf = (C.c_int64 * (8 * cap))()
    n = C.c_int()
    _check(load().jk_part_rows(pairs.handle, int(nparts), cap, buf, C.byref(n)))
    out = []
    for k in range(min(n.value, cap)):
        r = buf[8 * k:8 * k + 8]
        out.append(dict(cls=PAIR_CLASS_NAMES[r[0]] + "|" + PAIR_CLASS_NAMES[r[1]], part=r[2], r0=r[3], r1=r[4],
                        items=r[5], cost=r[6], max_row_cost=r[7]))
    return out


def allreduce_jk(J, K, group=None):
    """Sum partial J and K over the ranks of ``group`` (torch.distributed,
    NCCL for CUDA tensors, gloo for CPU ones) in one collective: the two
    matrices are reduced as one stacked buffer when they are views of it."""
    import torch
    import torch.distributed as dist
    base = J._base if J._base is not None and J._base is K._base else None
    if base is not None and base.is_contiguous() and base.numel() == J.numel() + K.numel():
        dist.all_reduce(base, op=dist.ReduceOp.SUM, group=group)
    else:
        JK = torch.stack([J, K])
        dist.all_reduce(JK, op=dist.ReduceOp.SUM, group=group)
        J.copy_(JK[0])
        K.copy_(JK[1])
    return J, K


def jk_build_distributed(pairs: ShellPairs, D, precision: str = "fp64", group=None, stream=None):
    """One molecule's J and K over the ranks of a torch.distributed group:
    rank r builds part r of world (cost-balanced quartet rows of every
    class), then one all-reduce sums the parts.  Without an initialised
    group of more than one rank this is jk_build."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return jk_build(pairs, D, precision, stream=stream)
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    n = pairs.nbf
    JK = torch.empty((2, n, n), dtype=torch.float64, device=D.device)
    J, K = JK[0], JK[1]
    jk_build_part(pairs, D, rank, world, precision, J=J, K=K, stream=stream)
    allreduce_jk(J, K, group)
    return J, K


def jk_grad_distributed(pairs: ShellPairs, D, precision: str = "fp64", group=None, stream=None):
    """dE/dR of one molecule over the ranks of a group: a part per rank, one
    all-reduce (sum) of the [natom, 3] gradient."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return jk_grad(pairs, D, precision, stream=stream)
    g = jk_grad_part(pairs, D, dist.get_rank(group), dist.get_world_size(group), precision, stream=stream)
    dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return g


def limits() -> dict:
    """Compiled limits: {"lmax": highest shell l, "grad_lmax": highest l of jk_grad}."""
    a, b = C.c_int(), C.c_int()
    _check(load().jk_limits(C.byref(a), C.byref(b)))
    return {"lmax": a.value, "grad_lmax": b.value}


def one_electron(pairs: ShellPairs, charges, stream=None, device=None):
    """Overlap S, kinetic T and nuclear attraction V (float64 CUDA tensors,
    nbf x nbf) with nuclear charges[natom] at the handle's atoms."""
    import torch
    z = np.ascontiguousarray(charges, dtype=np.float64)
    if z.shape != (pairs.natom,):
        raise ValueError(f"expected {pairs.natom} charges")
    n = pairs.nbf
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    S, T, V = (torch.empty((n, n), dtype=torch.float64, device=dev) for _ in range(3))
    _check(load().jk_one_electron(pairs.handle, C.c_void_p(z.ctypes.data), _dev_ptr(S), _dev_ptr(T), _dev_ptr(V),
                                  _stream_ptr(stream)))
    return S, T, V


_SPH_DIR = {"to_cartesian": 0, "to_pure": 1}


def sph_transform(pairs: ShellPairs, M, direction: str, out=None, stream=None):
    """``to_cartesian``: T M T^T (M nsph x nsph, e.g. a pure-basis density);
    ``to_pure``: T^T M T (M nbf x nbf, e.g. Cartesian J or K).  T is the
    block-diagonal Cartesian-to-pure matrix of the handle's shells."""
    import torch
    n_in, n_out = (pairs.nsph, pairs.nbf) if direction == "to_cartesian" else (pairs.nbf, pairs.nsph)
    if tuple(M.shape) != (n_in, n_in):
        raise ValueError(f"expected a {n_in} x {n_in} matrix")
    if out is None:
        out = torch.empty((n_out, n_out), dtype=torch.float64, device=M.device)
    elif tuple(out.shape) != (n_out, n_out):
        raise ValueError(f"out must be {n_out} x {n_out}")
    _check(load().jk_sph_transform(pairs.handle, _SPH_DIR[direction], _dev_ptr(M), _dev_ptr(out),
                                   _stream_ptr(stream)))
    return out


def jk_build_pure(pairs: ShellPairs, D_pure, precision: str = "fp64", stream=None):
    """J and K over pure d/f shells for a pure-basis density (nsph x nsph):
    D is taken to the Cartesian basis, built, and J, K taken back."""
    Dc = sph_transform(pairs, D_pure, "to_cartesian", stream=stream)
    J, K = jk_build(pairs, Dc, precision, stream=stream)
    return sph_transform(pairs, J, "to_pure", stream=stream), sph_transform(pairs, K, "to_pure", stream=stream)


def jk_grad_pure(pairs: ShellPairs, D_pure, precision: str = "fp64", out=None, stream=None):
    """dE/dR at fixed pure-basis density: the Cartesian gradient at T D T^T."""
    return jk_grad(pairs, sph_transform(pairs, D_pure, "to_cartesian", stream=stream), precision, out, stream)


def jk_build_batched(pairs_list, Ds, Js=None, Ks=None, precision: str = "fp64", stream=None):
    import torch
    n = len(pairs_list)
    if Js is None:
        Js = [torch.empty_like(D) for D in Ds]
    if Ks is None:
        Ks = [torch.empty_like(D) for D in Ds]
    arr = C.c_void_p * n
    hp = arr(*[p.handle.value for p in pairs_list])
    dp = arr(*[_dev_ptr(D).value for D in Ds])
    jp = arr(*[_dev_ptr(J).value for J in Js])
    kp = arr(*[_dev_ptr(K).value for K in Ks])
    _check(load().jk_build_batched(n, hp, dp, jp, kp, _PREC[precision], _stream_ptr(stream)))
    return Js, Ks


def boys(L: int, T, precision: str = "fp64", stream=None):
    """F_m(T), m = 0..L, for a float64 CUDA tensor of arguments (diagnostic)."""
    import torch
    T = T.contiguous()
    F = torch.empty((T.numel(), L + 1), dtype=torch.float64, device=T.device)
    _check(load().jk_boys(int(L), int(T.numel()), _dev_ptr(T), _dev_ptr(F), _PREC[precision], _stream_ptr(stream)))
    return F


def set_option(name: str, value: float):
    _check(load().jk_set_option(JK_OPT[name], float(value)))


def get_option(name: str) -> float:
    v = C.c_double()
    _check(load().jk_get_option(JK_OPT[name], C.byref(v)))
    return v.value


def autotune(pairs: ShellPairs, D, precision: str = "fp64", stream=None):
    """Per-class work-per-thread tuning (the paper's Algorithm 2); returns the
    chosen configuration (see tuning())."""
    import torch
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    _check(load().jk_autotune(pairs.handle, _dev_ptr(D), _dev_ptr(J), _dev_ptr(K), _PREC[precision],
                              _stream_ptr(stream)))
    return tuning(pairs)


def tuning(pairs: ShellPairs):
    """{class: (fp64 block, fp64 quartets/thread, fp32 block, fp32 quartets/thread)}."""
    buf = (C.c_int * (6 * 64))()
    n = C.c_int()
    _check(load().jk_tuning(pairs.handle, 64, buf, C.byref(n)))
    out = {}
    for k in range(n.value):
        r = buf[6 * k:6 * k + 6]
        out[PAIR_CLASS_NAMES[r[0]] + "|" + PAIR_CLASS_NAMES[r[1]]] = tuple(r[2:])
    return out


def set_tuning(pairs: ShellPairs, cfg: dict):
    """Restore a configuration returned by tuning() (a tuner cache)."""
    rows = []
    for k, v in cfg.items():
        a, b = k.split("|")
        rows += [PAIR_CLASS_NAMES.index(a), PAIR_CLASS_NAMES.index(b)] + [int(x) for x in v]
    arr = (C.c_int * max(1, len(rows)))(*rows)
    _check(load().jk_set_tuning(pairs.handle, len(rows) // 6, arr))


def last_launches(pairs: ShellPairs) -> int:
    """Kernels launched by the last jk_build / jk_grad on this handle."""
    n = C.c_int64()
    _check(load().jk_last_launches(pairs.handle, C.byref(n)))
    return n.value


def last_split(pairs: ShellPairs):
    """(shell quartets run in FP32, in FP64) by the last jk_build on this handle."""
    a, b = C.c_int64(), C.c_int64()
    _check(load().jk_last_split(pairs.handle, C.byref(a), C.byref(b)))
    return a.value, b.value


PAIR_CLASS_NAMES = ["ss", "ps", "pp", "ds", "dp", "dd", "fs", "fp", "fd", "ff"]


def class_stats(pairs: ShellPairs):
    """Per (bra class, ket class): shell quartets, primitive quartets, bra
    primitive-pair work units and algorithmic FP operation count."""
    buf = (C.c_int64 * (6 * 64))()
    n = C.c_int()
    _check(load().jk_class_stats(pairs.handle, 64, buf, C.byref(n)))
    out = []
    for k in range(n.value):
        r = buf[6 * k:6 * k + 6]
        out.append(dict(cls=PAIR_CLASS_NAMES[r[0]] + "|" + PAIR_CLASS_NAMES[r[1]], bra=r[0], ket=r[1],
                        nquartets=r[2], nprimq=r[3], nbrap=r[4], flops=r[5]))
    return out


def split_stats(pairs: ShellPairs):
    """Per class of the last mixed build: FP32 and FP64 shell quartets,
    primitive quartets and algorithmic operation counts."""
    buf = (C.c_int64 * (8 * 64))()
    n = C.c_int()
    _check(load().jk_split_stats(pairs.handle, 64, buf, C.byref(n)))
    out = []
    for k in range(n.value):
        r = buf[8 * k:8 * k + 8]
        out.append(dict(cls=PAIR_CLASS_NAMES[r[0]] + "|" + PAIR_CLASS_NAMES[r[1]], bra=r[0], ket=r[1],
                        fp32=dict(nquartets=r[2], nprimq=r[3], flops=r[4]),
                        fp64=dict(nquartets=r[5], nprimq=r[6], flops=r[7])))
    return out


def profile(pairs: ShellPairs):
    """Per-launch event timings of the last jk_build (profile option set)."""
    buf = (C.c_double * (5 * 256))()
    n = C.c_int()
    _check(load().jk_profile(pairs.handle, 256, buf, C.byref(n)))
    out = []
    for k in range(min(n.value, 256)):
        r = buf[5 * k:5 * k + 5]
        out.append(dict(cls=PAIR_CLASS_NAMES[int(r[0])] + "|" + PAIR_CLASS_NAMES[int(r[1])], bra=int(r[0]),
                        ket=int(r[1]), prec={0: "fp64", 3: "df", 4: "fp32c"}.get(int(r[2]), "fp32"), nquartets=int(r[3]),
                        ms=r[4]))
    return out


def fma_peak(precision: str = "fp64", iters: int = 20000, stream=None) -> float:
    """Measured SIMT FMA throughput in FLOP/s (diagnostic microbenchmark)."""
    v = C.c_double()
    _check(load().jk_fma_peak(_PREC[precision], int(iters), C.byref(v), _stream_ptr(stream)))
    return v.value


def _autograd():
    import torch

    class JKEnergy(torch.autograd.Function):
        """E(xyz, D) = tr(D J[D])/2 - tr(D K[D])/4 for the molecule's shells
        placed at the atom positions ``xyz`` (a [natom, 3] float64 tensor).

        Forward: shellpairs_build at xyz + jk_build + jk_energy.  Backward:
        dE/dxyz from jk_grad (the adjoint kernel, run only when xyz requires
        a gradient; the handle is kept until then), dE/dD = J - K/2.  With
        ``pure`` D is a density over pure d/f shells: the build runs on
        T D T^T and J, K are taken back to the pure basis (T does not depend
        on the geometry, so dE/dxyz is the Cartesian gradient at T D T^T)."""

        @staticmethod
        def forward(ctx, xyz, D, mol, thresh=None, precision="fp64", pure=False):
            import copy
            m = copy.copy(mol)
            m.xyz = xyz.detach().cpu().numpy().astype(np.float64)
            pairs = ShellPairs(m, thresh)
            Dc = D.detach().contiguous()
            if pure:
                Dx = sph_transform(pairs, Dc, "to_cartesian")
                Jx, Kx = jk_build(pairs, Dx, precision)
                J, K = sph_transform(pairs, Jx, "to_pure"), sph_transform(pairs, Kx, "to_pure")
            else:
                Dx = Dc
                J, K = jk_build(pairs, Dc, precision)
            E = jk_energy(Dc, J, K)
            # the adjoint kernel runs in backward, and only if xyz needs a gradient
            if ctx.needs_input_grad[0]:
                ctx.pairs, ctx.Dx, ctx.precision = pairs, Dx, precision
            else:
                pairs.free()
                ctx.pairs = None
            ctx.save_for_backward(J, K)
            return torch.tensor(E, dtype=torch.float64, device=xyz.device)

        @staticmethod
        def backward(ctx, gout):
            J, K = ctx.saved_tensors
            gx = None
            if ctx.pairs is not None:
                g = jk_grad(ctx.pairs, ctx.Dx, ctx.precision)
                ctx.pairs.free()
                ctx.pairs, ctx.Dx = None, None
                gx = (gout * g).to(g.device)
            gD = gout * (J - 0.5 * K) if ctx.needs_input_grad[1] else None
            return gx, gD, None, None, None, None

    return JKEnergy


_JKE = None


def jk_energy_fn(xyz, D, mol, thresh=None, precision="fp64", pure=False):
    """Differentiable E = tr(DJ)/2 - tr(DK)/4 (torch.autograd.Function); D
    over pure d/f shells if ``pure``."""
    global _JKE
    if _JKE is None:
        _JKE = _autograd()
    return _JKE.apply(xyz, D, mol, thresh, precision, pure)
