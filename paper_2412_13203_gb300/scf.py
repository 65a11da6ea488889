"""Closed-shell Hartree-Fock on the GPU around the J/K build.

The SCF structure of Sec. 2.1: from the current density D build the Fock
matrix F = H + J(D) - K(D)/2 (H = T + V), diagonalise it in the orthogonalised
basis, take the occupied orbitals' density, evaluate the energy, repeat until
the density is stable.  The integrals come from the library's kernels
(jk_one_electron, jk_build); the dense linear algebra of each iteration (the
symmetric orthogonaliser S^(-1/2), one eigen-decomposition and a few n x n
products) is delegated to PyTorch's CUDA linear algebra (cuSOLVER, cuBLAS)
on the same device, and the nuclear repulsion is summed on the host.

Roothaan iterations from the core guess (D = 0) with DIIS extrapolation
(Pulay's commutator error FDS - SDF on the last `diis` Fock matrices, from
the second iteration on); `diis=0` gives plain Roothaan iterations.

Incremental Fock builds (`incremental_eps`): J and K are linear in D, so
J(D_n) = J(D_m) + J(D_n - D_m); the difference density shrinks as the SCF
converges, and with density screening (JK_OPT_DENSITY_SCREEN = eps) the build
of J(D_n - D_m) runs only the quartets whose density-weighted bound reaches
eps.  Every `rebuild` iterations, and for the final energy, J and K are built
from the full density again.  Density screening acts in the mixed build;
an FP64 incremental build uses it with tau = 0 (every kept quartet in FP64).

Pure d and f shells (`pure=True`): S and H are taken to the pure basis once
(T^T S T, T^T H T), the SCF runs there, and every Fock build transforms the
density to the Cartesian basis and J, K back (jk_sph_transform).
"""
from __future__ import annotations

from contextlib import contextmanager
from dataclasses import dataclass, field

import numpy as np

from . import ShellPairs, get_option, jk_build, last_split, one_electron, set_option, sph_transform


@dataclass
class SCFResult:
    energy: float             # total energy (electronic + nuclear repulsion), Eh
    electronic: float
    nuclear_repulsion: float
    iterations: int
    converged: bool
    D: object                 # total density (CUDA tensor, nbf x nbf)
    orbital_energies: object  # CUDA tensor
    C: object                 # orbital coefficients (CUDA tensor, nbf x nbf)
    quartets: list = field(default_factory=list)  # shell quartets evaluated per iteration


@contextmanager
def _screened(eps, precision):
    """Density screening at eps for the builds inside (restores the options)."""
    old_eps, old_tau = get_option("density_screen"), get_option("mixed_tau")
    set_option("density_screen", eps)
    if precision == "fp64":
        set_option("mixed_tau", 0.0)
    try:
        yield
    finally:
        set_option("density_screen", old_eps)
        set_option("mixed_tau", old_tau)


def nuclear_repulsion(xyz, charges) -> float:
    xyz = np.asarray(xyz, dtype=np.float64)
    z = np.asarray(charges, dtype=np.float64)
    e = 0.0
    for i in range(len(z)):
        for j in range(i):
            e += z[i] * z[j] / float(np.linalg.norm(xyz[i] - xyz[j]))
    return e


def rhf(mol, charges, nocc: int, thresh: float | None = None, precision: str = "fp64", maxiter: int = 100,
        e_tol: float = 1e-10, d_tol: float = 1e-8, diis: int = 6, pairs: ShellPairs | None = None,
        incremental_eps: float | None = None, rebuild: int = 8, pure: bool = False) -> SCFResult:
    """Restricted Hartree-Fock for `nocc` doubly occupied orbitals.  `mol`
    carries the geometry and shells as for ShellPairs; `charges[natom]` are
    the nuclear charges; `thresh` the Schwarz threshold of the pair build
    (None: no screening, so that S, T and V are complete); `incremental_eps`
    switches on incremental, density-screened Fock builds; `pure` runs the
    SCF over pure d and f shells (D, C and the orbital count are then those of
    the pure basis)."""
    import torch
    if pairs is None:
        pairs = ShellPairs(mol, thresh)
    S, T, V = one_electron(pairs, charges)
    H = T + V
    if pure:
        S = sph_transform(pairs, S, "to_pure")
        H = sph_transform(pairs, H, "to_pure")

    def build(Dm, prec, Jo, Ko):
        """J and K of density Dm (in the SCF's basis) into Jo, Ko."""
        if not pure:
            jk_build(pairs, Dm, prec, Jo, Ko)
            return
        Jc, Kc = jk_build(pairs, sph_transform(pairs, Dm, "to_cartesian"), prec)
        sph_transform(pairs, Jc, "to_pure", out=Jo)
        sph_transform(pairs, Kc, "to_pure", out=Ko)
    w, U = torch.linalg.eigh(S)
    X = (U * w.rsqrt()) @ U.T
    n = pairs.nsph if pure else pairs.nbf
    D = torch.zeros((n, n), dtype=torch.float64, device=S.device)
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    Jd = torch.empty_like(D)
    Kd = torch.empty_like(D)
    D_built = None  # density J and K currently belong to
    quartets = []
    e_old = None
    focks, errs = [], []
    converged = False
    eps = Cmo = None
    it = 0
    for it in range(1, maxiter + 1):
        if incremental_eps and D_built is not None and (it - 1) % rebuild != 0:
            with _screened(incremental_eps, precision):
                build(D - D_built, "mixed", Jd, Kd)
                n32, n64 = last_split(pairs)
            J += Jd
            K += Kd
            quartets.append(n32 + n64)
        else:
            build(D, precision, J, K)
            quartets.append(pairs.nquartets)
        D_built = D
        F = H + J - 0.5 * K
        e_el = 0.5 * float(torch.sum(D * (H + F)))
        if diis and it > 1:  # D = 0 of the first iteration commutes trivially: no DIIS vector
            err = F @ D @ S - S @ D @ F
            focks.append(F)
            errs.append(err)
            focks, errs = focks[-diis:], errs[-diis:]
            m = len(focks)
            if m >= 2:
                B = torch.empty((m + 1, m + 1), dtype=torch.float64, device=D.device)
                for i in range(m):
                    for j in range(m):
                        B[i, j] = torch.sum(errs[i] * errs[j])
                B[m, :m] = -1.0
                B[:m, m] = -1.0
                B[m, m] = 0.0
                rhs = torch.zeros(m + 1, dtype=torch.float64, device=D.device)
                rhs[m] = -1.0
                c = torch.linalg.lstsq(B.cpu(), rhs.cpu().unsqueeze(1)).solution.squeeze(1).to(D.device)
                F = sum(c[i] * focks[i] for i in range(m))
        eps, Cp = torch.linalg.eigh(X.T @ F @ X)
        Cmo = X @ Cp
        Cocc = Cmo[:, :nocc]
        Dn = 2.0 * Cocc @ Cocc.T
        dmax = float((Dn - D).abs().max())
        D = Dn
        if e_old is not None and abs(e_el - e_old) < e_tol and dmax < d_tol:
            converged = True
            break
        e_old = e_el
    # energy of the final density
    build(D, precision, J, K)
    e_el = 0.5 * float(torch.sum(D * (2.0 * H + J - 0.5 * K)))
    enuc = nuclear_repulsion(mol.xyz, charges)
    return SCFResult(e_el + enuc, e_el, enuc, it, converged, D, eps, Cmo, quartets)
