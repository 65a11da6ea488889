"""Writes the oracle's J, K and E of the 32-atom benchmark workload
(32 atoms on a jittered 2.5-bohr lattice, 3s 2p 1d per atom, 480 Cartesian
basis functions, Schwarz threshold 1e-10, seeded density) to jk_32atom.npz.

Only the CPU oracle runs here: Obara-Saika/HRR integrals over every unique
shell quartet that passes Schwarz, each added to its eight permutational
images with Neumaier-compensated sums (J_mn = sum_ls (mn|ls) D_ls,
K_mn = sum_ls (ml|ns) D_ls, E = tr(DJ)/2 - tr(DK)/4), every integral and sum
in long double (64-bit significand on x86) and rounded to FP64 at the end.
The FP64 oracle's elements carry errors of a few 1e-11 (the FP64 rounding of
the recursions), which add up to several 1e-10 in E, too close to the 1e-10
target to judge an FP64 build by; the extended values are good to about
1e-14.  The GPU parity test of the full-size build compares every element of
its J and K and its E with these values.  About 2.5 hours on 8 x86 cores.

Run:  python tests/golden/make_jk_32atom.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import molgen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(HERE, "jk_32atom.npz")


def main():
    mol, D = molgen.config(1)
    thresh = molgen.CONFIG_THRESH[1]
    t = time.time()
    J, K, kept = oracle.jk(mol, D, thresh, mode="unique", extended=True)
    E = oracle.energy(D, J, K)
    dt = time.time() - t
    iu = np.triu_indices(mol.nbf)
    # J and K are symmetric: the upper triangles hold every value
    np.savez_compressed(OUT, J_upper=J[iu], K_upper=K[iu], E=np.float64(E), kept=np.int64(kept),
                        nbf=np.int64(mol.nbf), thresh=np.float64(thresh),
                        asymJ=np.float64(np.abs(J - J.T).max()), asymK=np.float64(np.abs(K - K.T).max()),
                        arith=np.str_("long double"), seconds=np.float64(dt))
    print(f"nbf={mol.nbf} kept={kept} E={E!r} |J|max={np.abs(J).max():.3f} |K|max={np.abs(K).max():.3f} "
          f"threads={oracle.num_threads()} {dt:.0f}s -> {OUT}")


if __name__ == "__main__":
    main()
