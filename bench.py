"""Benchmark: screened shell quartets/s and J/K build time, mixed vs FP64, on
the 32-atom l<=2 workload (480 Cartesian basis functions, Schwarz 1e-10).

One step = one J/K build (jk_build) of the whole workload: every screened
shell quartet evaluated, contracted into J and K and symmetrised.  The shell
pairs (a per-geometry object) are built once before timing; their build time
is reported separately.  ``value`` is the mixed-precision build's screened
quartets/s summed over ranks; the FP64 build is timed the same way and
reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank builds its own copy of the workload (independent
problems, weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
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


def pure_leg(g, pairs, Dt, J, K, stream, flush, steps):
    """Event-timed pure-basis steps: T D T^T, the mixed build, T^T J T and
    T^T K T.  The pure density is T^T D T of the workload's density."""
    import torch
    Dp = g.sph_transform(pairs, Dt, "to_pure")
    Dc = torch.empty_like(Dt)
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
            "energy_Eh": g.jk_energy(Dp, Jp, Kp), "steps": steps}


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

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    mol, D = molgen.config(CONFIG)
    thresh = molgen.CONFIG_THRESH[CONFIG]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    pairs = g.ShellPairs(mol, thresh)
    torch.cuda.synchronize()
    pair_ms = 1e3 * (time.perf_counter() - t0)
    Dt = torch.from_numpy(D).to(dev)
    J = torch.empty_like(Dt)
    K = torch.empty_like(Dt)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def timed_steps(prec, steps, warmup, profile=False):
        for _ in range(warmup):
            g.jk_build(pairs, Dt, prec, J, K)
        barrier()
        evs = []
        prof = {}
        launches = 0
        for _ in range(steps):
            flush.fill_(1)  # L2 flush between timed iterations, outside the events
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.jk_build(pairs, Dt, prec, J, K)
            e1.record(stream)
            evs.append((e0, e1))
            launches += g.last_launches(pairs)
            if profile:
                for r in g.profile(pairs):
                    key = (r["cls"], r["prec"])
                    prof.setdefault(key, []).append(r["ms"])
        barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, prof, launches

    # FMA peaks of this GPU (own microbenchmark)
    peak64 = g.fma_peak("fp64", 4000)
    peak32 = g.fma_peak("mixed", 20000)

    clocks = ClockSampler(local)
    clocks.start()
    # the headline: the mixed build (W warm-up + K timed steps)
    ms_mx, _, lmx = timed_steps("mixed", args.steps, args.warmup)
    E_mx = g.jk_energy(Dt, J, K)
    J_mx, K_mx = J.clone(), K.clone()
    n32, n64 = g.last_split(pairs)
    clk = clocks.stop()
    # per-kernel event timings and per-precision work of one more mixed build
    g.set_option("profile", 1)
    _, prof_mx, _ = timed_steps("mixed", 1, 0, profile=True)
    g.set_option("profile", 0)
    split = {s["cls"]: s for s in g.split_stats(pairs)}
    # the plain FP64 form beside it (fewer steps: it is ~3x slower)
    g.set_option("profile", 1)
    ms64, prof64, _ = timed_steps("fp64", min(args.steps, 2), 1, profile=True)
    g.set_option("profile", 0)
    E64 = g.jk_energy(Dt, J, K)
    dJ = float((J_mx - J).abs().max())
    dK = float((K_mx - K).abs().max())

    # end to end through the public API: pinned host D -> device, build, J and K back to pinned host
    Dh = torch.from_numpy(D).pin_memory()
    Jh = torch.empty(Dh.shape, dtype=torch.float64).pin_memory()
    Kh = torch.empty(Dh.shape, dtype=torch.float64).pin_memory()
    Dd = torch.empty_like(Dt)
    e2e = []
    for k in range(1 + args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Dd.copy_(Dh, non_blocking=True)
        g.jk_build(pairs, Dd, "mixed", J, K)
        Jh.copy_(J, non_blocking=True)
        Kh.copy_(K, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if k >= 1:
            e2e.append(e0.elapsed_time(e1))

    nq = pairs.nquartets
    t_mx = sum(ms_mx) / len(ms_mx)
    t_64 = sum(ms64) / len(ms64)
    t_e2e = sum(e2e) / len(e2e)
    # max over ranks (each rank ran its own copy of the workload: weak scaling)
    from paper_2412_13203_gb300 import shard
    t_mx, t_64, t_e2e = shard.max_over_ranks([t_mx, t_64, t_e2e], device=dev)

    # roofline of the dominant kernel of the mixed build: algorithmic operations
    # of the generated code for the quartets that launch processed / its
    # event-timed duration, against the measured FMA peak of its precision
    stats = {s["cls"]: s for s in g.class_stats(pairs)}
    per_mx = {k: float(np.mean(v)) for k, v in prof_mx.items()}
    dom_cls, dom_prec = max(per_mx, key=per_mx.get)
    dom_flops = split[dom_cls]["fp32" if dom_prec == "fp32" else "fp64"]["flops"]
    dom_peak = peak32 if dom_prec == "fp32" else peak64
    achieved = dom_flops / (per_mx[(dom_cls, dom_prec)] * 1e-3)
    tot_flops = sum(s["flops"] for s in stats.values())
    try:
        n_cart = cartesian_integrals(stats)
    except (KeyError, ValueError, IndexError):
        n_cart = None
    per = {k[0]: float(np.mean(v)) for k, v in prof64.items() if k[1] == "fp64"}
    dom64 = max(per, key=per.get)
    ach64 = stats[dom64]["flops"] / (per[dom64] * 1e-3)

    # the same workload with its d shells pure: transform D to the Cartesian
    # basis, mixed build, transform J and K back (reported beside the
    # headline; the headline above is the Cartesian build)
    try:
        pure = pure_leg(g, pairs, Dt, J, K, stream, flush, args.steps)
    except Exception as e:  # noqa: BLE001 -- reported, never fatal to the line
        pure = {"error": f"{type(e).__name__}: {e}"}

    out = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            rate, n, dt, thr = oracle_sample_rate(mol, D, thresh, args.cpu_seconds)
            cpu = {"value": rate, "unit": "quartets/s", "cores": thr, "kind": "oracle",
                   "sample": f"{n} random screened unique shell quartets of the same workload ({dt:.1f} s)",
                   "single_thread": oracle_single_thread_rate(args.cpu_single_seconds)}
        out = {
            "metric": METRIC, "value": nq * world / (t_mx * 1e-3), "unit": "quartets/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_mx, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nbf": pairs.nbf, "screened_quartets": nq,
                       "primitive_quartets": pairs.nprimquartets, "l2": "flushed (256 MB write) between timed steps",
                       "pair_build_ms": round(pair_ms, 2), "mixed_tau": g.get_option("mixed_tau"),
                       "mixed_tsmall": g.get_option("mixed_tsmall"), "mixed_fp32_quartets": n32,
                       "mixed_fp64_quartets": n64},
            "fp64": {"value": nq * world / (t_64 * 1e-3), "unit": "quartets/s", "ms_per_step": t_64,
                     "steps": min(args.steps, 2), "energy_Eh": E64, "flops_per_s": tot_flops / (t_64 * 1e-3),
                     "roofline": {"bound": "alu", "kernel": f"eri_jk_{dom64} fp64", "achieved": ach64 / 1e12,
                                  "peak": peak64 / 1e12, "unit": "TFLOP/s", "frac": ach64 / peak64}},
            "mixed": {"ms_per_step": t_mx,
                      "primitive_quartets_per_s": pairs.nprimquartets * world / (t_mx * 1e-3),
                      "cartesian_integrals_per_s": None if n_cart is None else n_cart * world / (t_mx * 1e-3),
                      "energy_Eh": E_mx, "energy_minus_fp64_Eh": E_mx - E64,
                      "max_abs_dJ_vs_fp64": dJ, "max_abs_dK_vs_fp64": dK,
                      "fp32_share_of_flops": sum(v["fp32"]["flops"] for v in split.values()) / tot_flops},
            "e2e": {"value": nq * world / (t_e2e * 1e-3), "unit": "quartets/s", "ms_per_step": t_e2e,
                    "h2d_bytes_per_step": int(Dh.numel() * 8), "d2h_bytes_per_step": int(2 * Jh.numel() * 8)},
            "roofline": {"bound": "alu", "kernel": f"eri_jk_{dom_cls} {dom_prec}", "achieved": achieved / 1e12,
                         "peak": dom_peak / 1e12, "unit": "TFLOP/s", "frac": achieved / dom_peak, "traffic": None,
                         "peak_source": f"measured {'FFMA' if dom_prec == 'fp32' else 'DFMA'} microbenchmark "
                                        "(jk_fma_peak) on this GPU",
                         "fp32_peak_tflops": peak32 / 1e12, "fp64_peak_tflops": peak64 / 1e12},
            "class_ms_mixed": {f"{k[0]} {k[1]}": round(v, 3)
                               for k, v in sorted(per_mx.items(), key=lambda x: -x[1])[:12]},
            "class_ms_fp64": {k: round(v, 3) for k, v in sorted(per.items(), key=lambda x: -x[1])},
            "pure_d_shells": pure,
            "gpu_launches": int(lmx),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    pairs.free()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
