"""Command-line driver: one seeded workload (a reduced atom count of any of
the synthetic recipes), J/K, gradient, pure-shell or one-electron builds on
the GPU with their wall times -- a quick check of an installation, and the
small cases the kernel profiles are captured on.

    python -m paper_2412_13203_gb300.run_jk --config 1 --prec fp64 [--natom 8] [--repeat 2]
        [--grad | --pure | --one-electron] [--screen EPS]

--pure builds J/K of the workload with its d shells pure (the density taken
to the pure basis first); --one-electron times jk_one_electron (unit
nuclear charges); --screen sets density screening for mixed builds.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--natom", type=int, default=None)
    ap.add_argument("--prec", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--grad", action="store_true")
    ap.add_argument("--pure", action="store_true")
    ap.add_argument("--one-electron", action="store_true")
    ap.add_argument("--screen", type=float, default=0.0)
    a = ap.parse_args(argv)
    import numpy as np
    import torch
    import molgen
    import paper_2412_13203_gb300 as g
    mol, D = molgen.config(a.config, natom=a.natom)
    thr = molgen.CONFIG_THRESH[a.config]
    t = time.perf_counter()
    pairs = g.ShellPairs(mol, thr)
    torch.cuda.synchronize()
    print(f"pairs {time.perf_counter() - t:.3f}s nbf {pairs.nbf} npairs {pairs.npairs} quartets {pairs.nquartets} "
          f"primitive quartets {pairs.nprimquartets}", flush=True)
    Dt = torch.from_numpy(D).cuda()
    g.set_option("density_screen", a.screen)
    if a.pure:
        Dt = g.sph_transform(pairs, Dt, "to_pure")
    for r in range(a.repeat):
        torch.cuda.synchronize()
        t = time.perf_counter()
        if a.one_electron:
            S, T, V = g.one_electron(pairs, np.ones(pairs.natom))
            torch.cuda.synchronize()
            print(f"one-electron {r} {time.perf_counter() - t:.4f}s tr S {float(S.trace()):.6f}", flush=True)
        elif a.pure:
            J, K = g.jk_build_pure(pairs, Dt, a.prec)
            torch.cuda.synchronize()
            print(f"jk pure {a.prec} {r} {time.perf_counter() - t:.4f}s E {g.jk_energy(Dt, J, K)!r}", flush=True)
        elif a.grad:
            gr = g.jk_grad(pairs, Dt, a.prec)
            torch.cuda.synchronize()
            print(f"grad {r} {time.perf_counter() - t:.4f}s |g|max {float(gr.abs().max()):.6e}", flush=True)
        else:
            J, K = g.jk_build(pairs, Dt, a.prec)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            print(f"jk {a.prec} {r} {dt:.4f}s E {g.jk_energy(Dt, J, K)!r} split {g.last_split(pairs)}", flush=True)
    pairs.free()


if __name__ == "__main__":
    main()
