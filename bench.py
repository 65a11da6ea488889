"""Benchmark: screened shell quartets/s and J/K build time, mixed vs FP64, on
the 32-atom l<=2 workload (480 Cartesian basis functions, Schwarz 1e-10),
with the other workloads as side legs.

One step = one J/K build (jk_build) of the whole workload: every screened
shell quartet evaluated, contracted into J and K and symmetrised.  The shell
pairs (a per-geometry object) are built once before timing; their build time
is reported separately.  ``value`` is the mixed-precision build's screened
quartets/s; the FP64 build is timed the same way and reported beside it, and
both are compared element by element with the CPU oracle's J, K and E
(tests/golden/jk_32atom.npz).

Side legs (N = 1; each guarded, an error is reported in the line):
  batch  64 molecules of 8..48 atoms in one batched launch sequence (mixed,
         CUDA graph on and off, the Algorithm 2 autotuner on the largest molecule),
         per-molecule errors against the oracle (smallest molecules) and
         against single FP64 builds;
  grad   nuclear gradient of the 24-atom workload (jk_grad);
  large  the 200-atom l<=3 workload: a seeded sample of cost-balanced parts
         of its quartet rows, timed, and the extrapolated full build;
  rpath  the classes emitted with Algorithm 1's recursion order, timed
         against the fixed order;
  pure   the 32-atom workload over pure d shells.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--legs a,b,...]

Under torchrun (N > 1) one molecule is split across the ranks: rank r builds
the cost-balanced part r of N of every class's quartet rows and one NCCL
all-reduce sums J and K (strong scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import molgen  # noqa: E402

CONFIG = 1
WORKLOAD = "32-atom jittered lattice (spacing 2.5 bohr), 3s2p1d per atom, K 1..6, exponents 0.05..5e3, 480 Cartesian bf, Schwarz 1e-10"
METRIC = "screened shell quartets/s (mixed FP32/FP64 J/K build)"
GOLDEN = os.path.join(ROOT, "tests", "golden", "jk_32atom.npz")
TRAFFIC = os.path.join(ROOT, "profiles", "dram_traffic.json")
LEGS = "fp64,batch,grad,large,rpath,pure"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--legs", default=LEGS, help="comma-separated side legs (N = 1): " + LEGS)
    ap.add_argument("--batch-mols", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=1)
    ap.add_argument("--large-parts", type=int, default=262144, help="parts of the 200-atom rows")
    ap.add_argument("--large-samples", type=int, default=3, help="parts timed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cpu-single-seconds", type=float, default=4.0)
    return ap.parse_args()


# ---------------------------------------------------------------- CPU oracle
def oracle_sample_rate(mol, D, thresh, seconds, seed=77):
    """The CPU oracle (as it stands) on a bounded random sample of the
    workload's screened unique quartets; returns (quartets/s, n, seconds, threads)."""
    import oracle
    Q = oracle.schwarz(mol)
    q = oracle.sample_unique_quartets(mol, 4000, seed, thresh, Q)
    t = time.perf_counter()
    oracle.jk_quartets(mol, D, q)
    dt = time.perf_counter() - t
    rate = len(q) / dt
    n = int(max(4000, min(5_000_000, rate * seconds)))
    q = oracle.sample_unique_quartets(mol, n, seed + 1, thresh, Q)
    t = time.perf_counter()
    oracle.jk_quartets(mol, D, q)
    dt = time.perf_counter() - t
    return n / dt, n, dt, oracle.num_threads()


def oracle_single_thread_rate(seconds):
    """The same bounded oracle sample on one host thread, in a child process
    started with OMP_NUM_THREADS=1 (this process's OpenMP pool is already
    sized); None if the child fails."""
    code = ("import json, bench, molgen; mol, D = molgen.config(bench.CONFIG); "
            f"print(json.dumps(bench.oracle_sample_rate(mol, D, molgen.CONFIG_THRESH[bench.CONFIG], {seconds!r})))")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=300)
        rate, n, dt, thr = json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError, OSError):
        return None
    return {"value": rate, "unit": "quartets/s", "cores": thr,
            "sample": f"{n} random screened unique shell quartets of the same workload ({dt:.1f} s)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    mol, D = molgen.config(CONFIG)
    thresh = molgen.CONFIG_THRESH[CONFIG]
    Q = oracle.schwarz(mol)
    rate0 = oracle_sample_rate(mol, D, thresh, 1.0)[0]
    n = int(max(2000, rate0 * 3.0))  # ~3 s of CPU work per step
    for w in range(args.warmup):
        oracle.jk_quartets(mol, D, oracle.sample_unique_quartets(mol, min(n, 2000), 900 + w, thresh, Q))
    times = []
    for k in range(args.steps):
        q = oracle.sample_unique_quartets(mol, n, 1000 + k, thresh, Q)
        t = time.perf_counter()
        oracle.jk_quartets(mol, D, q)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    value = n * args.steps / tot
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "quartets/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{n} random screened unique shell quartets per step"},
        "cpu_baseline": {"value": value, "unit": "quartets/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{n} random screened unique shell quartets per step, {args.steps} steps"},
        "e2e": {"value": value, "unit": "quartets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- helpers
def golden():
    """The oracle's J, K, E of the 32-atom workload (None if the file is absent)."""
    if not os.path.exists(GOLDEN):
        return None
    z = np.load(GOLDEN)
    n = int(z["nbf"])
    iu = np.triu_indices(n)
    J = np.zeros((n, n))
    K = np.zeros((n, n))
    J[iu] = z["J_upper"]
    K[iu] = z["K_upper"]
    return J + np.triu(J, 1).T, K + np.triu(K, 1).T, float(z["E"])


def errors_vs(J, K, E, Jo, Ko, Eo):
    """Max-abs and relative (to the largest element) errors of J, K and E."""
    dJ, dK = float(np.abs(J - Jo).max()), float(np.abs(K - Ko).max())
    return {"max_abs_dJ": dJ, "max_abs_dK": dK, "abs_dE": abs(E - Eo),
            "rel_dJ": dJ / float(np.abs(Jo).max()), "rel_dK": dK / float(np.abs(Ko).max()),
            "rel_dE": abs(E - Eo) / abs(Eo)}


def class_totals(records):
    """Per (class, precision): summed launch milliseconds of one build's
    profile records (a class's FP32 part has a suffix and a demoted-list
    launch, each covering all of its range kernels)."""
    tot = {}
    for r in records:
        # the FP32 complement of a primitively split FP64 list runs the FP32 kernels
        key = (r["cls"], "fp32" if r["prec"] == "fp32c" else r["prec"])
        tot[key] = tot.get(key, 0.0) + r["ms"]
    return tot


def kernel_sha(cls_name):
    """Hash of the generated source of a class's kernels plus the device
    header they include: a traffic figure measured for another hash is stale."""
    sys.path.insert(0, os.path.join(ROOT, "paper_2412_13203_gb300", "codegen"))
    try:
        import md_codegen as mg
    finally:
        sys.path.pop(0)
    names = ["ss", "ps", "pp", "ds", "dp", "dd", "fs", "fp", "fd", "ff"]
    bra, ket = cls_name.split("|")
    pc = mg.PAIR_CLASSES
    src = mg.gen_class_kernels(pc[names.index(bra)], pc[names.index(ket)])[0]
    with open(os.path.join(ROOT, "paper_2412_13203_gb300", "csrc", "eri_device.cuh"), "rb") as f:
        hdr = f.read()
    return hashlib.sha1(src.encode() + hdr).hexdigest()[:16]


def traffic_of(kernel_key):
    """DRAM bytes per launch of a kernel from the committed ncu summary table,
    or None if there is none for the current source of that kernel."""
    if not os.path.exists(TRAFFIC):
        return None
    try:
        tab = json.load(open(TRAFFIC))
        ent = tab.get(kernel_key)
        if not ent:
            return None
        cls = kernel_key.split()[0]
        if ent.get("kernel_sha") != kernel_sha(cls):
            return None
        return ent
    except (OSError, ValueError, KeyError, ImportError):
        return None


def cartesian_integrals(class_stats):
    """Cartesian integrals of the screened unique quartets: sum over classes of
    quartets x n_a n_b n_c n_d (classes named like "dp|ps")."""
    lval = {"s": 0, "p": 1, "d": 2, "f": 3}
    nc = lambda ch: (lval[ch] + 1) * (lval[ch] + 2) // 2
    total = 0
    for name, st in class_stats.items():
        bra, ket = name.split("|")
        total += st["nquartets"] * nc(bra[0]) * nc(bra[1]) * nc(ket[0]) * nc(ket[1])
    return total


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def timed(stream, fn, flush=None):
    """CUDA-event milliseconds of fn() on `stream` (L2 flushed first, outside the events)."""
    import torch
    if flush is not None:
        flush.fill_(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), r


# ---------------------------------------------------------------- side legs
def batch_leg(g, stream, flush, nmol, steps):
    """64 independent molecules in one batched launch sequence (mixed)."""
    import torch
    import oracle
    batch = molgen.config2_batch(nmol)
    t0 = time.perf_counter()
    hs = [g.ShellPairs(m, molgen.CONFIG_THRESH[2]) for m, _ in batch]
    torch.cuda.synchronize()
    pair_s = time.perf_counter() - t0
    nq = sum(h.nquartets for h in hs)
    Ds = [torch.from_numpy(D).cuda() for _, D in batch]
    Js = [torch.empty_like(D) for D in Ds]
    Ks = [torch.empty_like(D) for D in Ds]
    run = lambda: g.jk_build_batched(hs, Ds, Js, Ks, "mixed")
    out = {"workload": f"{nmol} molecules of 8..48 atoms (config-1 recipe each, own D), Schwarz 1e-10",
           "molecules": nmol, "atoms": [int(m.natom) for m, _ in batch], "screened_quartets": nq,
           "pair_build_s": round(pair_s, 3)}
    g.set_option("graph", 1)
    first, _ = timed(stream, run)
    ms = [timed(stream, run, flush)[0] for _ in range(steps)]
    out["graph"] = {"first_call_ms": first, "ms_per_step": float(np.mean(ms)), "steps": steps,
                    "value": nq / (np.mean(ms) * 1e-3), "unit": "quartets/s"}
    g.set_option("graph", 0)
    ms_ng, _ = timed(stream, run, flush)
    g.set_option("graph", 1)
    out["no_graph"] = {"ms_per_step": ms_ng, "steps": 1, "value": nq / (ms_ng * 1e-3), "unit": "quartets/s"}
    # per-molecule errors: the smallest molecules against the oracle, a few others against FP64 builds
    order = np.argsort([m.nbf for m, _ in batch])
    errs = []
    for i in order[:3]:
        m, D = batch[i]
        Jo, Ko, _ = oracle.jk(m, D, molgen.CONFIG_THRESH[2], mode="unique")
        J, K = Js[i].cpu().numpy(), Ks[i].cpu().numpy()
        e = errors_vs(J, K, g.jk_energy(Ds[i], Js[i], Ks[i]), Jo, Ko, oracle.energy(D, Jo, Ko))
        errs.append(dict(molecule=int(i), nbf=int(m.nbf), against="oracle", **e))
    for i in order[len(order) // 2: len(order) // 2 + 3]:
        J64, K64 = g.jk_build(hs[i], Ds[i], "fp64")
        e = errors_vs(Js[i].cpu().numpy(), Ks[i].cpu().numpy(), g.jk_energy(Ds[i], Js[i], Ks[i]),
                      J64.cpu().numpy(), K64.cpu().numpy(), g.jk_energy(Ds[i], J64, K64))
        errs.append(dict(molecule=int(i), nbf=int(m.nbf), against="gpu fp64", **e))
    out["errors"] = errs
    out["max_abs_error_Eh"] = max(max(e["max_abs_dJ"], e["max_abs_dK"], e["abs_dE"]) for e in errs)
    # Algorithm 2 on the largest molecule: its mixed build before and after tuning
    big = int(order[-1])
    one = lambda: g.jk_build(hs[big], Ds[big], "mixed", Js[big], Ks[big])
    timed(stream, one)
    before = min(timed(stream, one, flush)[0] for _ in range(2))
    t0 = time.perf_counter()
    cfg = g.autotune(hs[big], Ds[big], "mixed")
    tune_s = time.perf_counter() - t0
    timed(stream, one)
    after = min(timed(stream, one, flush)[0] for _ in range(2))
    out["autotune_largest_molecule"] = {
        "molecule": big, "nbf": int(batch[big][0].nbf), "before_ms": before, "after_ms": after,
        "speedup": before / after, "tune_s": round(tune_s, 2),
        "changed_classes": {k: v for k, v in cfg.items() if v[1] != 1 or v[3] != 1}}
    for h in hs:
        h.free()
    return out


def grad_leg(g, stream, flush, steps=2):
    """jk_grad of the 24-atom workload, FP64 and mixed (FP32 derivative
    integrals below the gradient cutoff, FP64 accumulation)."""
    import torch
    mol, D = molgen.config(3)
    pairs = g.ShellPairs(mol, molgen.CONFIG_THRESH[3])
    Dt = torch.from_numpy(D).cuda()
    out = {"workload": "24-atom lattice (config-1 recipe), 360 Cartesian bf, Schwarz 1e-10, 72 gradient components",
           "screened_quartets": pairs.nquartets}
    grads = {}
    for prec, n in (("fp64", 1), ("mixed", steps)):
        # the FP64 gradient takes tens of seconds: one call, timed without a warm-up
        first = timed(stream, lambda: g.jk_grad(pairs, Dt, prec))[0] if prec == "mixed" else None
        ms = []
        for _ in range(n):
            t, G = timed(stream, lambda: g.jk_grad(pairs, Dt, prec), flush)
            ms.append(t)
        grads[prec] = G.cpu().numpy()
        out[prec] = {"ms_per_call": float(np.mean(ms)), "first_call_ms": first, "steps": n,
                     "value": pairs.nquartets / (np.mean(ms) * 1e-3), "unit": "quartets/s",
                     "max_abs_sum_over_atoms": float(np.abs(grads[prec].sum(0)).max())}
        if prec == "mixed":
            n32, n64 = g.last_split(pairs)
            out[prec].update(fp32_quartets=n32, fp64_quartets=n64, grad_tau=g.get_option("grad_tau"))
    out["mixed"]["max_abs_vs_fp64"] = float(np.abs(grads["mixed"] - grads["fp64"]).max())
    out["max_abs_gradient"] = float(np.abs(grads["fp64"]).max())
    pairs.free()
    return out


def large_leg(g, stream, nparts, nsamples):
    """The 200-atom l<=3 workload: seeded cost-balanced parts, timed, and the
    extrapolated full mixed build (every part holds 1/nparts of every class's
    algorithmic cost within one row's cost)."""
    import torch
    mol, D = molgen.config(4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pairs = g.ShellPairs(mol, molgen.CONFIG_THRESH[4])
    torch.cuda.synchronize()
    pair_s = time.perf_counter() - t0
    Dt = torch.from_numpy(D).cuda()
    J = torch.empty_like(Dt)
    K = torch.empty_like(Dt)
    t0 = time.perf_counter()
    g.prepare_partition(pairs, nparts)  # computes and caches the partition
    part_s = time.perf_counter() - t0
    rng = np.random.Generator(np.random.PCG64(4242))
    parts = sorted(int(x) for x in rng.choice(nparts, size=nsamples, replace=False))
    timed(stream, lambda: g.jk_build_part(pairs, Dt, parts[0], nparts, "mixed", J, K))  # warm-up
    g.set_option("profile", 1)
    samples = []
    for p in parts:
        ms, _ = timed(stream, lambda: g.jk_build_part(pairs, Dt, p, nparts, "mixed", J, K))
        recs = g.profile(pairs)
        tot = class_totals(recs)
        split = {s["cls"]: s for s in g.split_stats(pairs)}
        kern = sum(tot.values())
        fcls = {}
        for (cls, prec), t in tot.items():
            if "f" in cls and t > 0:
                fl = split[cls]["fp32" if prec == "fp32" else "fp64"]["flops"]
                fcls[f"{cls} {prec}"] = {"ms": t, "tflops": fl / (t * 1e-3) / 1e12}
        samples.append({"part": p, "ms": ms, "kernel_ms": kern, "fp32_quartets": g.last_split(pairs)[0],
                        "fp64_quartets": g.last_split(pairs)[1], "f_classes": fcls})
    g.set_option("profile", 0)
    kern = float(np.mean([s["kernel_ms"] for s in samples]))
    wall = float(np.mean([s["ms"] for s in samples]))
    out = {"workload": "200-atom lattice (spacing 2.6 bohr), 4s3p2d1f per atom, K 1..8, exponents 0.03..1e4, "
                       "7000 Cartesian bf, Schwarz 1e-11, D with exp(-0.3 r) decay",
           "pair_build_s": round(pair_s, 2), "partition_s": round(part_s, 2), "nbf": pairs.nbf,
           "screened_quartets": pairs.nquartets, "primitive_quartets": pairs.nprimquartets,
           "parts": nparts, "sampled_parts": samples,
           "extrapolated_build_s": kernel_extrap(kern, nparts),
           "extrapolated_quartets_per_s": pairs.nquartets / (kern * nparts * 1e-3),
           "label": "extrapolation: mean kernel time of the sampled parts x number of parts",
           "part_wall_ms_mean": wall}
    pairs.free()
    return out


def kernel_extrap(kernel_ms, nparts):
    return kernel_ms * nparts * 1e-3


def rpath_leg(g, pairs, Dt, J, K):
    """Per-class FP32 times of a mixed build with the fixed R recursion order
    and with Algorithm 1's searched order (classes emitted both ways)."""
    res = {}
    for on in (0, 1):
        g.set_option("rpath", on)
        g.set_option("profile", 1)
        best = None
        for _ in range(3):
            g.jk_build(pairs, Dt, "mixed", J, K)
            tot = class_totals(g.profile(pairs))
            best = tot if best is None else {k: min(v, best[k]) for k, v in tot.items()}
        g.set_option("profile", 0)
        res[on] = best
    g.set_option("rpath", 0)
    out = {}
    for cls in ("dd|dd", "dd|dp", "dp|dp"):
        a, b = res[0].get((cls, "fp32")), res[1].get((cls, "fp32"))
        if a and b:
            out[cls] = {"fixed_ms": a, "searched_ms": b, "speedup": a / b}
    return out


def pure_leg(g, pairs, stream, flush, steps):
    """Event-timed pure-basis steps: T D T^T, the mixed build, T^T J T and
    T^T K T, with the pure density drawn by the workload's recipe (C C^T,
    C ~ N(0, 0.1) of shape nsph x nsph/2)."""
    import torch
    Dp = torch.from_numpy(molgen.density_n(pairs.nsph, 1000 + CONFIG + 700)).cuda()
    Dc = torch.empty((pairs.nbf, pairs.nbf), dtype=torch.float64, device=Dp.device)
    J = torch.empty_like(Dc)
    K = torch.empty_like(Dc)
    Jp = torch.empty_like(Dp)
    Kp = torch.empty_like(Dp)
    tr, tot = [], []
    for k in range(1 + steps):
        flush.fill_(1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        g.sph_transform(pairs, Dp, "to_cartesian", out=Dc)
        ev[1].record(stream)
        g.jk_build(pairs, Dc, "mixed", J, K)
        ev[2].record(stream)
        g.sph_transform(pairs, J, "to_pure", out=Jp)
        g.sph_transform(pairs, K, "to_pure", out=Kp)
        ev[3].record(stream)
        ev[3].synchronize()
        if k >= 1:
            tr.append(ev[0].elapsed_time(ev[1]) + ev[2].elapsed_time(ev[3]))
            tot.append(ev[0].elapsed_time(ev[3]))
    t = sum(tot) / len(tot)
    return {"nsph": pairs.nsph, "nbf": pairs.nbf, "ms_per_step": t, "transform_ms": sum(tr) / len(tr),
            "value": pairs.nquartets / (t * 1e-3), "unit": "quartets/s",
            "energy_Eh": g.jk_energy(Dp, Jp, Kp), "steps": steps,
            "density": "pure-basis recipe C C^T, C ~ N(0, 0.1) of shape nsph x nsph/2"}


def guarded(fn, *a, **k):
    try:
        return fn(*a, **k)
    except Exception as e:  # noqa: BLE001 -- reported in the line, never fatal to it
        return {"error": f"{type(e).__name__}: {e}"}


# ---------------------------------------------------------------- GPU
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import paper_2412_13203_gb300 as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    legs = set(x for x in args.legs.split(",") if x) if world == 1 else set()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    mol, D = molgen.config(CONFIG)
    thresh = molgen.CONFIG_THRESH[CONFIG]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pairs = g.ShellPairs(mol, thresh)
    torch.cuda.synchronize()
    pair_ms = 1e3 * (time.perf_counter() - t0)
    Dt = torch.from_numpy(D).to(dev)
    JK = torch.empty((2,) + Dt.shape, dtype=torch.float64, device=dev)
    J, K = JK[0], JK[1]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def build(prec, Din=None):
        """One step: the whole build (N = 1) or this rank's part plus one all-reduce of J and K."""
        Din = Dt if Din is None else Din
        if world == 1:
            g.jk_build(pairs, Din, prec, J, K)
        else:
            g.jk_build_part(pairs, Din, rank, world, prec, J, K)
            g.allreduce_jk(J, K)

    def timed_steps(prec, steps, warmup, profile=False):
        for _ in range(warmup):
            build(prec)
        barrier()
        evs, recs = [], []
        launches = 0
        for _ in range(steps):
            flush.fill_(1)  # L2 flush between timed iterations, outside the events
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            build(prec)
            e1.record(stream)
            evs.append((e0, e1))
            launches += g.last_launches(pairs)
            if profile:
                recs.append(g.profile(pairs))
        barrier()
        return [a.elapsed_time(b) for a, b in evs], recs, launches

    # FMA peaks of this GPU (own microbenchmark)
    peak64 = g.fma_peak("fp64", 4000)
    peak32 = g.fma_peak("mixed", 20000)

    clocks = ClockSampler(local)
    clocks.start()
    # the headline: the mixed build (W warm-up + K timed steps)
    ms_mx, _, lmx = timed_steps("mixed", args.steps, args.warmup)
    clk = clocks.stop()
    E_mx = g.jk_energy(Dt, J, K)
    J_mx, K_mx = J.cpu().numpy(), K.cpu().numpy()
    n32, n64 = g.last_split(pairs)
    # per-kernel event timings and per-precision work of one more mixed build
    g.set_option("profile", 1)
    _, recs_mx, _ = timed_steps("mixed", 1, 0, profile=True)
    g.set_option("profile", 0)
    split = {s["cls"]: s for s in g.split_stats(pairs)}
    tot_mx = class_totals(recs_mx[0])

    # end to end through the public API: pinned host D -> device, build, J and K back to pinned host
    Dh = torch.from_numpy(D).pin_memory()
    JKh = torch.empty(JK.shape, dtype=torch.float64).pin_memory()
    Dd = torch.empty_like(Dt)
    e2e = []
    for k in range(1 + args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Dd.copy_(Dh, non_blocking=True)
        build("mixed", Dd)
        JKh.copy_(JK, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if k >= 1:
            e2e.append(e0.elapsed_time(e1))

    # the plain FP64 form beside it (fewer steps: it is several times slower)
    ms64, recs64 = [float("nan")], None
    E64 = None
    if world > 1 or "fp64" in legs:
        g.set_option("profile", 1 if world == 1 else 0)
        ms64, recs64, _ = timed_steps("fp64", min(args.steps, 2), 1, profile=world == 1)
        g.set_option("profile", 0)
        E64 = g.jk_energy(Dt, J, K)
        J64, K64 = J.cpu().numpy(), K.cpu().numpy()

    nq = pairs.nquartets
    t_mx = float(np.mean(ms_mx))
    t_64 = float(np.mean(ms64))
    t_e2e = float(np.mean(e2e))
    from paper_2412_13203_gb300 import shard
    t_mx, t_64, t_e2e = shard.max_over_ranks([t_mx, t_64, t_e2e], device=dev)

    out = None
    if rank == 0:
        stats = {s["cls"]: s for s in g.class_stats(pairs)}
        tot_flops = sum(s["flops"] for s in stats.values())
        try:
            n_cart = cartesian_integrals(stats)
        except (KeyError, ValueError, IndexError):
            n_cart = None
        # roofline of the dominant kernel of the mixed build: the class and
        # precision with the largest summed launch time; algorithmic
        # operations of the generated code for the quartets it processed /
        # that time, against the measured FMA peak of its precision
        (dom_cls, dom_prec), dom_ms = max(tot_mx.items(), key=lambda kv: kv[1])
        # FP32 kernels against the FFMA peak; FP64 kernels against the DFMA peak;
        # double-float kernels (FP64-selected quartets on the FP32 pipe) count
        # the FP64 algorithmic operations they replace, against the DFMA peak
        dom_flops = split[dom_cls]["fp32" if dom_prec == "fp32" else "fp64"]["flops"]
        dom_peak = peak32 if dom_prec == "fp32" else peak64
        achieved = dom_flops / (dom_ms * 1e-3)
        dom_key = f"{dom_cls} {dom_prec}"
        traf = traffic_of(dom_key)
        gold = golden()
        err_mx = err_64 = None
        if gold is not None:
            err_mx = errors_vs(J_mx, K_mx, E_mx, *gold)
            if E64 is not None:
                err_64 = errors_vs(J64, K64, E64, *gold)
        roof_fp32 = {}
        for (cls, prec), ms in sorted(tot_mx.items(), key=lambda kv: -kv[1])[:6]:
            if prec == "fp32":
                roof_fp32[cls] = {"ms": ms, "tflops": split[cls]["fp32"]["flops"] / (ms * 1e-3) / 1e12,
                                  "frac": split[cls]["fp32"]["flops"] / (ms * 1e-3) / peak32}
        fp64_part = sum(v for (c, p), v in tot_mx.items() if p in ("fp64", "df"))
        fp32_part = sum(v for (c, p), v in tot_mx.items() if p == "fp32")
        df_kernels = {}
        for (cls, prec), ms in sorted(tot_mx.items(), key=lambda kv: -kv[1])[:12]:
            if prec == "df":
                fl = split[cls]["fp64"]["flops"]
                df_kernels[cls] = {"ms": ms, "fp64_equiv_tflops": fl / (ms * 1e-3) / 1e12,
                                   "vs_dfma_peak": fl / (ms * 1e-3) / peak64}
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            rate, n, dt, thr = oracle_sample_rate(mol, D, thresh, args.cpu_seconds)
            cpu = {"value": rate, "unit": "quartets/s", "cores": thr, "kind": "oracle",
                   "sample": f"{n} random screened unique shell quartets of the same workload ({dt:.1f} s)",
                   "single_thread": oracle_single_thread_rate(args.cpu_single_seconds)}
        fp64 = None
        if recs64 is not None or world > 1:
            fp64 = {"value": nq / (t_64 * 1e-3), "unit": "quartets/s", "ms_per_step": t_64,
                    "steps": min(args.steps, 2), "energy_Eh": E64, "flops_per_s": tot_flops / (t_64 * 1e-3),
                    "errors_vs_oracle": err_64}
            if recs64:
                tot64 = {k[0]: v for k, v in class_totals(recs64[0]).items()}
                d64 = max(tot64, key=tot64.get)
                ach64 = stats[d64]["flops"] / (tot64[d64] * 1e-3)
                fp64["roofline"] = {"bound": "alu", "kernel": f"eri_jk_{d64} fp64", "achieved": ach64 / 1e12,
                                    "peak": peak64 / 1e12, "unit": "TFLOP/s", "frac": ach64 / peak64,
                                    "traffic": (traffic_of(f"{d64} fp64") or {}).get("bytes_per_launch")}
                fp64["class_ms"] = {k: round(v, 3) for k, v in sorted(tot64.items(), key=lambda x: -x[1])}
        out = {
            "metric": METRIC, "value": nq / (t_mx * 1e-3), "unit": "quartets/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_mx, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nbf": pairs.nbf, "screened_quartets": nq,
                       "primitive_quartets": pairs.nprimquartets, "l2": "flushed (256 MB write) between timed steps",
                       "pair_build_ms": round(pair_ms, 2), "mixed_tau": g.get_option("mixed_tau"),
                       "mixed_tsmall": g.get_option("mixed_tsmall"), "mixed_fp32_quartets": n32,
                       "mixed_fp64_quartets": n64, "mixed_prim_tau": g.get_option("prim_tau"),
                       "mixed_fp64_tier_primitive_quartets": sum(v["fp64"]["nprimq"] for v in split.values()),
                       "parallelism": f"one molecule split over {world} GPUs (cost-balanced quartet rows, "
                                      "one all-reduce of J and K per build)" if world > 1 else "1 GPU"},
            "mixed": {"ms_per_step": t_mx, "primitive_quartets_per_s": pairs.nprimquartets / (t_mx * 1e-3),
                      "cartesian_integrals_per_s": None if n_cart is None else n_cart / (t_mx * 1e-3),
                      "energy_Eh": E_mx, "errors_vs_oracle": err_mx,
                      "fp32_share_of_flops": sum(v["fp32"]["flops"] for v in split.values()) / tot_flops,
                      "fp64_or_df_kernel_ms": fp64_part, "fp32_kernel_ms": fp32_part,
                      "df_tier": bool(g.get_option("df_tier")), "df_kernels_top": df_kernels,
                      "fp32_kernels_top": roof_fp32},
            "fp64": fp64,
            "e2e": {"value": nq / (t_e2e * 1e-3), "unit": "quartets/s", "ms_per_step": t_e2e,
                    "h2d_bytes_per_step": int(Dh.numel() * 8), "d2h_bytes_per_step": int(JKh.numel() * 8)},
            "roofline": {"bound": "alu", "kernel": f"eri_jk_{dom_cls} {dom_prec}", "achieved": achieved / 1e12,
                         "peak": dom_peak / 1e12, "unit": "TFLOP/s", "frac": achieved / dom_peak,
                         "traffic": None if traf is None else traf.get("bytes_per_launch"),
                         "traffic_source": None if traf is None else traf.get("source"),
                         "peak_source": f"measured {'FFMA' if dom_prec == 'fp32' else 'DFMA'} microbenchmark "
                                        "(jk_fma_peak) on this GPU" + (" (double-float kernel: FP64 operations it "
                                        "replaces per second against the DFMA peak)" if dom_prec == "df" else ""),
                         "fp32_peak_tflops": peak32 / 1e12, "fp64_peak_tflops": peak64 / 1e12},
            "class_ms_mixed": {f"{k[0]} {k[1]}": round(v, 3)
                               for k, v in sorted(tot_mx.items(), key=lambda x: -x[1])[:14]},
            "gpu_launches": int(lmx),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        if "rpath" in legs:
            out["rpath"] = guarded(rpath_leg, g, pairs, Dt, J, K)
        if "pure" in legs:
            out["pure_d_shells"] = guarded(pure_leg, g, pairs, stream, flush, args.steps)
        pairs.free()
        if "grad" in legs:
            out["gradient"] = guarded(grad_leg, g, stream, flush, 1)
        if "batch" in legs:
            out["batched"] = guarded(batch_leg, g, stream, flush, args.batch_mols, args.batch_steps)
        if "large" in legs:
            out["large"] = guarded(large_leg, g, stream, args.large_parts, args.large_samples)
        print(json.dumps(out), flush=True)
    else:
        pairs.free()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
