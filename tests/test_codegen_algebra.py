"""The generated McMurchie-Davidson code against the oracle, on the CPU.

The straight-line (flat) FP64 and FP32 bodies and the FP32 ket-component-range
bodies that the generator emits for the CUDA kernels are translated line by
line into Python and evaluated in double precision for random primitive
quartets, with the oracle's Boys function; the contracted block must equal the
oracle's Obara-Saika/HRR block.  This checks the generator's algebra (Hermite
E and R recursions, the FP32 scaled recursion with the prefactor folded into
the E products, the Cartesian transforms, component order) without a GPU;
the GPU tests check the compiled kernels."""
import math
import os
import re
import sys

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "paper_2412_13203_gb300", "codegen"))
import md_codegen as mg  # noqa: E402


class V:
    def __init__(self, x=0.0, y=0.0, z=0.0, w=0.0):
        self.x, self.y, self.z, self.w = x, y, z, w


def _split_top(s, sep):
    out, depth, cur = [], 0, ""
    for ch in s:
        if ch == "(":
            depth += 1
        elif ch == ")":
            depth -= 1
        if ch == sep and depth == 0:
            out.append(cur)
            cur = ""
        else:
            cur += ch
    if cur.strip():
        out.append(cur)
    return out


def to_python(body):
    """Translate a generated flat body (C) into Python source."""
    lines, ind = [], 0
    for raw in body.split("\n"):
        line = raw.split("//")[0].strip()
        if not line or line.startswith("#pragma"):
            continue
        line = re.sub(r"\b(\d+\.\d*|\d+)f\b", r"\1", line)
        line = re.sub(r"\b__fdividef\(", "_div(", line)
        line = re.sub(r"\brsqrtf?\(", "_rsqrt(", line)
        line = re.sub(r"\bfmaf?\(", "_fma(", line)
        m = re.match(r"(?:float|double) acc\[(\d+)\];$", line)
        if m:
            lines.append(" " * ind + f"acc = [0.0] * {m.group(1)}")
            continue
        if re.match(r"for \(int i = 0; i < \d+; \+\+i\) acc\[i\] = 0;$", line):
            continue
        m = re.match(r"for \(int ip = ipart; ip < ib\.z; ip \+= nsplit\) \{$", line)
        if m:
            lines.append(" " * ind + "for ip in range(ipart, ib.z, nsplit):")
            ind += 4
            continue
        if re.match(r"for \(int jq = 0; jq < ik\.z; \+\+jq\) \{$", line):
            lines.append(" " * ind + "for jq in range(ik.z):")
            ind += 4
            continue
        if line == "}":
            ind -= 4
            continue
        m = re.match(r"(?:float|double) F\[(\d+)\];$", line)
        if m:
            continue
        m = re.match(r"gb::boys_(?:f64|mixed)<(\d+)>\(T, F.*\);$", line)
        if m:
            lines.append(" " * ind + f"F = _boys({m.group(1)}, T)")
            continue
        for stmt in _split_top(line.rstrip(";"), ";"):
            stmt = stmt.strip()
            stmt = re.sub(r"^(?:const )?(?:float|double)[24]? ", "", stmt)
            for part in re.split(r",\s*(?=[A-Za-z_]\w*\s*=[^=])", stmt):
                lines.append(" " * ind + part.strip())
    assert ind == 0
    return "\n".join(lines)


def _pair_data(a, b):
    """Primitive-pair data as the pair builder forms it (FP64 and FP32 layouts)."""
    (Ra, ea, ca), (Rb, eb, cb) = a, b
    pp, pp2, ppf, ppf2 = [], [], [], []
    AB = Ra - Rb
    for i in range(len(ea)):
        for j in range(len(eb)):
            al, be = ea[i], eb[j]
            p = al + be
            P = (al * Ra + be * Rb) / p
            kap = math.sqrt(2 * math.pi ** 2.5) * math.exp(-al * be / p * AB @ AB) * ca[i] * cb[j] / p
            pp.append(V(*P, p))
            pp2.append(V(kap, 0.5 / p))
            PA, PB = -be / p * AB, al / p * AB
            ppf.append(V(*PA, p))
            ppf2.append(V(*PB, kap))
    return pp, pp2, ppf, ppf2


def _run(body, bra, ket, shells):
    ns = {"_fma": lambda a, b, c: a * b + c, "_rsqrt": lambda x: 1.0 / math.sqrt(x), "_div": lambda a, b: a / b,
          "_boys": lambda L, T: list(oracle.boys(L, float(T)))}
    A_, B_, C_, D_ = shells
    bra_pp = _pair_data((A_[0], A_[2], A_[3]), (B_[0], B_[2], B_[3]))
    ket_pp = _pair_data((C_[0], C_[2], C_[3]), (D_[0], D_[2], D_[3]))
    nb = len(bra_pp[0])
    pairs = V()
    pairs.pp, pairs.pp2 = bra_pp[0] + ket_pp[0], bra_pp[1] + ket_pp[1]
    pairs.ppf, pairs.ppf2 = bra_pp[2] + ket_pp[2], bra_pp[3] + ket_pp[3]
    ns.update(pairs=pairs, ib=V(0, 0, nb, 0), ik=V(0, 0, len(ket_pp[0]), nb), ipart=0, nsplit=1,
              A=V(*A_[0]), B=V(*B_[0]), C=V(*C_[0]), Dd=V(*D_[0]))
    AC = A_[0] - C_[0]
    ns.update(ACx=AC[0], ACy=AC[1], ACz=AC[2], boys=None, boysf=None, tsmall=0.0)
    exec(to_python(body), ns)
    return np.array(ns["acc"])


def _shells(rng, ls, kmax):
    out = []
    for l in ls:
        k = int(rng.integers(1, kmax + 1))
        out.append((rng.uniform(-1.0, 1.0, 3), l, np.exp(rng.uniform(np.log(0.2), np.log(8.0), k)),
                    rng.uniform(0.2, 1.0, k)))
    return out


FLAT = [(b, k, "double") for b, k in mg.class_pairs(2) if mg.use_flat(b, k, "f64")] + \
       [(b, k, "float") for b, k in mg.class_pairs(2) if mg.use_flat(b, k, "f32")]


@pytest.mark.parametrize("bra,ket,real", FLAT, ids=[mg.class_name(b, k) + "-" + r for b, k, r in FLAT])
def test_flat_body_matches_oracle(bra, ket, real):
    rng = np.random.default_rng(sum(bra) * 17 + sum(ket) * 5 + (real == "float"))
    sh = _shells(rng, [bra[0], bra[1], ket[0], ket[1]], 2)
    body, _ = mg.gen_quartet_body(bra, ket, real, True)
    got = _run(body, bra, ket, sh)
    ref = oracle.eri_quartet(sh).reshape(-1)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), np.abs(got - ref).max()


RANGE = [(b, k) for b, k in mg.class_pairs(2) if mg.crange_groups(b, k)]


@pytest.mark.parametrize("bra,ket", RANGE, ids=[mg.class_name(b, k) for b, k in RANGE])
def test_fp32_range_bodies_cover_the_block(bra, ket):
    """The FP32 range kernels of a class: their ranges partition the ket
    components and each range body equals its slice of the oracle block."""
    rng = np.random.default_rng(sum(bra) * 31 + sum(ket))
    sh = _shells(rng, [bra[0], bra[1], ket[0], ket[1]], 1)
    ref = oracle.eri_quartet(sh)
    na, nb, nc, nd = ref.shape
    groups = mg.crange_groups(bra, ket)
    assert [c for c0, c1 in groups for c in range(c0, c1)] == list(range(nc))
    for c0, c1 in groups:
        cds = [c * nd + d for c in range(c0, c1) for d in range(nd)]
        body, _ = mg.gen_quartet_body(bra, ket, "float", True, cds)
        got = _run(body, bra, ket, sh).reshape(na * nb, len(cds))
        want = ref.reshape(na * nb, nc * nd)[:, cds]
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max()), (c0, np.abs(got - want).max())
