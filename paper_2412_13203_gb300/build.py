"""Build the sm_103a shared library: run the McMurchie-Davidson generator, then
compile every translation unit with nvcc in parallel and link
``_build/libgb300eri.so`` next to this file."""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
GEN = os.path.join(BUILD, "gen")
LIB = os.path.join(BUILD, "libgb300eri.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", CSRC, "-I", os.path.join(ROOT, "include")] + ARCH


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _digest(paths, extra=""):
    h = hashlib.sha1(extra.encode())
    for p in paths:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def build(force: bool = False, lmax: int = 3, jobs: int | None = None, verbose: bool = False) -> str:
    sys.path.insert(0, os.path.join(HERE, "codegen"))
    try:
        import md_codegen
        import sph_codegen
    finally:
        sys.path.pop(0)
    os.makedirs(GEN, exist_ok=True)
    gen_files, _ = md_codegen.generate(GEN, lmax)
    gen_files.append(sph_codegen.emit(GEN))
    hand = [os.path.join(CSRC, "runtime.cu")]
    headers = [os.path.join(CSRC, "eri_device.cuh"), os.path.join(CSRC, "sph_transform.cuh"),
               os.path.join(CSRC, "split_kernels.cuh"), os.path.join(CSRC, "one_electron.cuh"),
               os.path.join(ROOT, "include", "gb300_eri.h")]
    srcs = hand + gen_files
    objs = []
    todo = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        stamp = o + ".sha"
        d = _digest([s] + headers, " ".join(NVCC_FLAGS))
        objs.append(o)
        if force or not os.path.exists(o) or not os.path.exists(stamp) or open(stamp).read() != d:
            todo.append((s, o, stamp, d))
    nv = nvcc()

    def comp(item):
        s, o, stamp, d = item
        cmd = [nv, "-c", s, "-o", o + ".tmp"] + NVCC_FLAGS
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {s}:\n{r.stderr[-4000:]}")
        os.replace(o + ".tmp", o)
        with open(stamp, "w") as f:
            f.write(d)
        return s, r.stderr

    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or max(2, os.cpu_count() or 2)) as ex:
            for s, err in ex.map(comp, todo):
                if verbose and err:
                    print(err)
    if todo or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([nv, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"], check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import time
    t = time.time()
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
    print(f"built in {time.time() - t:.1f}s")
