"""Seeded synthetic molecules and density matrices.

This module is the only code shared by the CPU oracle and the GPU library. It
draws geometries, shell recipes (angular momentum, exponents, raw contraction
coefficients) and density matrices from numpy's PCG64 generator and holds none
of the integral arithmetic: normalisation, Gaussian products, Boys functions,
recurrences and J/K contraction all live on either side of the boundary.

Recipes (the synthetic stand-ins for the paper's STO-3G benchmark molecules of
its Table "benchmarks", which are not available):

* ``config0``: 4 atoms uniform in a 6-bohr cube, min spacing 1.8 bohr;
  per atom 2 s + 1 p shell, 3 primitives each, exponents log-uniform in
  [0.1, 50].  nbf = 20.  No screening.
* ``config1``: 32 atoms on a jittered lattice (spacing 2.5 bohr); per atom
  3 s, 2 p, 1 d; primitives uniform in 1..6; exponents log-uniform in
  [0.05, 5e3].  nbf = 480.  Schwarz threshold 1e-10.
* ``config2``: 64 molecules of 8..48 atoms, each as ``config1``.
* ``config3``: 24 atoms as ``config1``.  nbf = 360.
* ``config4``: 200 atoms (spacing 2.6); per atom 4 s, 3 p, 2 d, 1 f;
  primitives 1..8; exponents log-uniform in [0.03, 1e4].  nbf = 7000.
  Density with exponential decay exp(-0.3 r_ij) between basis-function atoms.

Raw contraction coefficients are uniform in [0.1, 1.0]; both sides normalise
them with the same documented convention (axial Cartesian normalisation).
The density is D = C C^T with C ~ N(0, 0.1) of shape nbf x (nbf // 2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Molecule", "ncart", "lattice_sites", "random_molecule", "density", "density_n",
    "config", "config2_batch", "CONFIG_THRESH", "h2_sto3g",
]


def ncart(l: int) -> int:
    """Number of Cartesian components of a shell of angular momentum l."""
    return (l + 1) * (l + 2) // 2


@dataclass
class Molecule:
    """Atoms plus contracted Cartesian shells, as flat arrays.

    Basis functions are ordered shell by shell (shells are listed atom by
    atom), and inside a shell by Cartesian component with lx descending, then
    ly descending (xx, xy, xz, yy, yz, zz for d).
    """
    xyz: np.ndarray            # [natom, 3] float64, bohr
    shell_atom: np.ndarray     # [nshell] int32
    shell_l: np.ndarray        # [nshell] int32
    shell_nprim: np.ndarray    # [nshell] int32
    shell_prim_offset: np.ndarray  # [nshell] int32
    exps: np.ndarray           # [nprim_total] float64
    coefs: np.ndarray          # [nprim_total] float64, raw (un-normalised)
    charges: np.ndarray = field(default=None)  # [natom] float64 (only for SCF use)

    @property
    def natom(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def nshell(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def nbf(self) -> int:
        return int(sum(ncart(int(l)) for l in self.shell_l))

    def shell_offsets(self) -> np.ndarray:
        """First basis-function index of every shell."""
        n = np.array([ncart(int(l)) for l in self.shell_l], dtype=np.int64)
        return np.concatenate([[0], np.cumsum(n)[:-1]]).astype(np.int64)

    def bf_atom(self) -> np.ndarray:
        """Atom index of every basis function."""
        out = []
        for a, l in zip(self.shell_atom, self.shell_l):
            out += [int(a)] * ncart(int(l))
        return np.array(out, dtype=np.int64)

    def translated(self, shift) -> "Molecule":
        m = Molecule(self.xyz + np.asarray(shift, dtype=np.float64)[None, :],
                     self.shell_atom.copy(), self.shell_l.copy(), self.shell_nprim.copy(),
                     self.shell_prim_offset.copy(), self.exps.copy(), self.coefs.copy(),
                     None if self.charges is None else self.charges.copy())
        return m

    def with_xyz(self, xyz) -> "Molecule":
        return Molecule(np.ascontiguousarray(xyz, dtype=np.float64),
                        self.shell_atom.copy(), self.shell_l.copy(), self.shell_nprim.copy(),
                        self.shell_prim_offset.copy(), self.exps.copy(), self.coefs.copy(),
                        None if self.charges is None else self.charges.copy())


def lattice_sites(natom: int, spacing: float) -> np.ndarray:
    """First ``natom`` sites of an n^3 cubic lattice, n = ceil(natom^(1/3)),
    in lexicographic (x, y, z) order, z fastest."""
    n = 1
    while n ** 3 < natom:
        n += 1
    sites = [(i, j, k) for i in range(n) for j in range(n) for k in range(n)]
    return np.array(sites[:natom], dtype=np.float64) * spacing


def _uniform_cube(rng, natom, box, min_spacing):
    pts = []
    tries = 0
    while len(pts) < natom:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place atoms with the requested spacing")
        p = rng.uniform(0.0, box, size=3)
        if all(np.linalg.norm(p - q) >= min_spacing for q in pts):
            pts.append(p)
    return np.array(pts, dtype=np.float64)


def random_molecule(seed: int, natom: int, shells_per_atom, kmin: int, kmax: int,
                    alpha_min: float, alpha_max: float, *, layout: str = "lattice",
                    spacing: float = 2.5, box: float = 6.0, min_spacing: float = 1.8,
                    jitter: float = 0.2) -> Molecule:
    """Seeded molecule.

    ``shells_per_atom`` is a list of angular momenta, one entry per shell of
    every atom (e.g. ``[0, 0, 0, 1, 1, 2]``).  ``layout`` is ``"lattice"``
    (jittered cubic lattice, jitter uniform in +-jitter*spacing per coordinate)
    or ``"cube"`` (rejection-sampled uniform positions in [0, box]^3).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if layout == "lattice":
        xyz = lattice_sites(natom, spacing)
        xyz = xyz + rng.uniform(-jitter * spacing, jitter * spacing, size=xyz.shape)
    elif layout == "cube":
        xyz = _uniform_cube(rng, natom, box, min_spacing)
    else:
        raise ValueError(layout)
    atom, ls, nprim, off, exps, coefs = [], [], [], [], [], []
    cursor = 0
    for a in range(natom):
        for l in shells_per_atom:
            k = int(rng.integers(kmin, kmax + 1))
            e = np.exp(rng.uniform(math.log(alpha_min), math.log(alpha_max), size=k))
            e = np.sort(e)[::-1]
            c = rng.uniform(0.1, 1.0, size=k)
            atom.append(a); ls.append(int(l)); nprim.append(k); off.append(cursor)
            exps.extend(e.tolist()); coefs.extend(c.tolist())
            cursor += k
    return Molecule(np.ascontiguousarray(xyz, dtype=np.float64),
                    np.array(atom, dtype=np.int32), np.array(ls, dtype=np.int32),
                    np.array(nprim, dtype=np.int32), np.array(off, dtype=np.int32),
                    np.array(exps, dtype=np.float64), np.array(coefs, dtype=np.float64))


def density(mol: Molecule, seed: int, decay: float | None = None) -> np.ndarray:
    """Random symmetric positive semi-definite density D = C C^T,
    C ~ N(0, 0.1) of shape nbf x max(1, nbf // 2).  With ``decay`` the
    result is multiplied elementwise by exp(-decay * r_ij), r_ij the distance
    between the atoms of basis functions i and j (still PSD by the Schur
    product theorem)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nbf = mol.nbf
    C = rng.normal(0.0, 0.1, size=(nbf, max(1, nbf // 2)))
    D = C @ C.T
    if decay is not None:
        ba = mol.bf_atom()
        r = np.linalg.norm(mol.xyz[ba][:, None, :] - mol.xyz[ba][None, :, :], axis=-1)
        D = D * np.exp(-decay * r)
    D = 0.5 * (D + D.T)
    return np.ascontiguousarray(D)


def density_n(n: int, seed: int) -> np.ndarray:
    """The same recipe for a basis of n functions given by its size alone
    (e.g. the pure d/f basis of a molecule): D = C C^T, C ~ N(0, 0.1) of
    shape n x max(1, n // 2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    C = rng.normal(0.0, 0.1, size=(n, max(1, n // 2)))
    D = C @ C.T
    return np.ascontiguousarray(0.5 * (D + D.T))


#: Schwarz threshold per configuration (None = no screening).
CONFIG_THRESH = {0: None, 1: 1e-10, 2: 1e-10, 3: 1e-10, 4: 1e-11}

_C1_SHELLS = [0, 0, 0, 1, 1, 2]
_C4_SHELLS = [0, 0, 0, 0, 1, 1, 1, 2, 2, 3]


def config(idx: int, *, natom: int | None = None) -> tuple[Molecule, np.ndarray]:
    """Molecule and density of the named workload (PCG64 seed 1000 + idx for
    the geometry/shells, seed 1000 + idx + 500 for the density).  ``natom``
    overrides the atom count (used for reduced test cases of the same
    recipe)."""
    seed = 1000 + idx
    if idx == 0:
        mol = random_molecule(seed, natom or 4, [0, 0, 1], 3, 3, 0.1, 50.0, layout="cube",
                              box=6.0, min_spacing=1.8)
        return mol, density(mol, seed + 500)
    if idx in (1, 3):
        mol = random_molecule(seed, natom or (32 if idx == 1 else 24), _C1_SHELLS, 1, 6,
                              0.05, 5e3, layout="lattice", spacing=2.5)
        return mol, density(mol, seed + 500)
    if idx == 4:
        mol = random_molecule(seed, natom or 200, _C4_SHELLS, 1, 8, 0.03, 1e4,
                              layout="lattice", spacing=2.6)
        return mol, density(mol, seed + 500, decay=0.3)
    if idx == 2:
        return config2_batch(1)[0]
    raise ValueError(idx)


def config2_batch(nmol: int = 64, natom_range=(8, 48)) -> list[tuple[Molecule, np.ndarray]]:
    """The batched workload: molecule i draws its atom count from seed
    2000 + i, its geometry and shells from seed 12000 + i, and its density
    from seed 2500 + i."""
    out = []
    for i in range(nmol):
        rng = np.random.Generator(np.random.PCG64(2000 + i))
        natom = int(rng.integers(natom_range[0], natom_range[1] + 1))
        mol = random_molecule(2000 + i + 10000, natom, _C1_SHELLS, 1, 6, 0.05, 5e3,
                              layout="lattice", spacing=2.5)
        out.append((mol, density(mol, 2000 + i + 500)))
    return out


def h2_sto3g(R: float = 1.4) -> Molecule:
    """H2 at bond length R (bohr) in the STO-3G basis (zeta = 1.24): the
    three-Gaussian fit of a Slater 1s function (Hehre, Stewart and Pople,
    J. Chem. Phys. 51, 2657 (1969)), exponents already scaled by zeta^2.
    The coefficients are those of normalised primitives (raw here; both sides
    normalise)."""
    e = np.array([3.42525091, 0.62391373, 0.16885540])
    c = np.array([0.15432897, 0.53532814, 0.44463454])
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, R]])
    return Molecule(xyz, np.array([0, 1], np.int32), np.array([0, 0], np.int32),
                    np.array([3, 3], np.int32), np.array([0, 3], np.int32),
                    np.concatenate([e, e]), np.concatenate([c, c]),
                    charges=np.array([1.0, 1.0]))


def h2_polarised(R: float = 1.4) -> Molecule:
    """H2 / STO-3G (h2_sto3g) plus one p shell (exponent 1.1) and one d shell
    (exponent 0.8) per atom, shells listed atom by atom."""
    m = h2_sto3g(R)
    ls, atom, npr, off = list(m.shell_l), list(m.shell_atom), list(m.shell_nprim), list(m.shell_prim_offset)
    exps, coefs = list(m.exps), list(m.coefs)
    for a in range(2):
        for l, e in ((1, 1.1), (2, 0.8)):
            ls.append(l)
            atom.append(a)
            npr.append(1)
            off.append(len(exps))
            exps.append(e)
            coefs.append(1.0)
    o = np.argsort(atom, kind="stable")
    ls, atom, npr, off = (np.array(x, np.int32)[o] for x in (ls, atom, npr, off))
    return Molecule(m.xyz.copy(), atom, ls, npr, off, np.array(exps), np.array(coefs), np.array([1.0, 1.0]))


def h_chain(n: int, spacing: float) -> Molecule:
    """n hydrogens on the z axis, `spacing` bohr apart: STO-3G s (h2_sto3g)
    plus one p shell (exponent 1.0) per atom."""
    b = h2_sto3g(1.4)
    e, c = b.exps[:3], b.coefs[:3]
    ls, atom, npr, off, exps, coefs = [], [], [], [], [], []
    for a in range(n):
        for l, ee, cc in ((0, e, c), (1, np.array([1.0]), np.array([1.0]))):
            ls.append(l)
            atom.append(a)
            npr.append(len(ee))
            off.append(len(exps))
            exps += list(ee)
            coefs += list(cc)
    return Molecule(np.array([[0.0, 0.0, spacing * i] for i in range(n)]), np.array(atom, np.int32),
                    np.array(ls, np.int32), np.array(npr, np.int32), np.array(off, np.int32),
                    np.array(exps), np.array(coefs), np.ones(n))
