"""McMurchie-Davidson code generator for the per-class ERI kernels.

For a primitive quartet [ab|cd] the McMurchie-Davidson form is

  [ab|cd] = 2 pi^(5/2) / (p q sqrt(p+q)) K_AB K_CD
            sum_{tuv} E^{ab}_{tuv} sum_{tau nu phi} (-1)^{tau+nu+phi} E^{cd}_{tau nu phi}
            R_{t+tau, u+nu, v+phi}(rho, P - Q)

with the 1-D Hermite expansion coefficients (per axis)
  E^{i+1,j}_t = E^{ij}_{t-1} / (2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1}
  E^{i,j+1}_t = E^{ij}_{t-1} / (2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1},  E^{00}_0 = 1,
and the Hermite Coulomb integrals
  R^{(n)}_{000} = (-2 rho)^n F_n(rho |PQ|^2),
  R^{(n)}_{t+1,u,v} = t R^{(n+1)}_{t-1,u,v} + X_PQ R^{(n+1)}_{tuv}   (same for u, v).

This is the recurrence the paper's Graph Compiler turns into straight-line
code (Sec. 5, stages 2 and 4: a DAG of intermediate results emitted bottom-up
from the [00|00] base case), but built on Hermite E/R instead of the
paper's HGP recurrences.  Per shell quartet the generated kernel

  1. loops over bra primitive pairs; per pair it forms the bra E products,
  2. loops over ket primitive pairs; per pair it forms the signed ket E
     products, evaluates F_0..F_L, builds R_{tuv} and accumulates the
     half-transformed X[tuv][cd] (contracted over ket primitives),
  3. applies the bra transform into the contracted Cartesian block
     acc[ab][cd] (contracted over bra primitives),
  4. digests the block into J' and K' (fused, atomics).

Emission forms (chosen per class and precision):
  * "flat": everything straight-line, values in registers (small classes;
    FP32 kernels up to FLAT_F32_VALUES block values);
  * FP32 ket-component ranges: the large l <= 2 classes' FP32 work as one
    straight-line kernel per range of ket components c, each launched over
    all quartets (crange_groups);
  * "loop": R stored in a (L+1)^3 cube, the ket-component loop runtime, the
    per-axis E tables in small arrays (FP64 work of the large classes);
  * "chunk": classes with an f shell, one thread per ket component c, a rolled
    R recursion and bra E products in a local array (compact code).
Every kernel decodes work items (a quartet split over up to split_of()
threads by its bra primitive pairs) heaviest first.

The generator also prints the exact FMA/FLOP count per primitive quartet of
every class (used for the FLOP roofline).

Run:  python md_codegen.py OUTDIR
"""
from __future__ import annotations

import math
import os
import sys

PAIR_CLASSES = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1), (3, 2), (3, 3)]
LMAX = 3


def comps(l):
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def ncart(l):
    return (l + 1) * (l + 2) // 2


def herm(L):
    """Hermite triples (t,u,v) with t+u+v <= L, ordered by total then lexicographic desc."""
    out = []
    for tot in range(L + 1):
        for t in range(tot, -1, -1):
            for u in range(tot - t, -1, -1):
                out.append((t, u, tot - t - u))
    return out


# ---------------------------------------------------------------- symbolic emitter
class Sym:
    __slots__ = ("c", "name")

    def __init__(self, c=None, name=None):
        self.c, self.name = c, name

    @property
    def const(self):
        return self.name is None

    def __repr__(self):
        return self.name if self.name is not None else repr(self.c)


ONE = Sym(1.0)
ZERO = Sym(0.0)

DFL = "gb::dfl"  # double-float value type of the device header (hi + lo floats)


def df_literal(c):
    """A constant as a double-float literal: hi the nearest float, lo the
    nearest float to the remainder (split here, so no FP64 operation is emitted)."""
    import struct
    f32 = lambda x: struct.unpack("f", struct.pack("f", x))[0]
    hi = f32(float(c))
    lo = f32(float(c) - hi)
    return f"{DFL}({hi!r}f, {lo!r}f)" if lo != 0.0 else f"{DFL}({hi!r}f)"


class Emitter:
    def __init__(self, real):
        self.real = real
        self.lines = []
        self.flops = 0

    def lit(self, c):
        if self.real == "float":
            return f"{c!r}f" if not float(c).is_integer() else f"{float(c):.1f}f"
        if self.real == DFL:
            return df_literal(c)
        return repr(float(c))

    def val(self, s: Sym):
        return s.name if not s.const else self.lit(s.c)

    def emit(self, line):
        self.lines.append(line)

    def define(self, name, expr):
        self.lines.append(f"const {self.real} {name} = {expr};")
        return Sym(name=name)

    def lincomb(self, terms, name):
        """sum of factor * value, factors are Sym; folds constants."""
        const = 0.0
        var = []
        for f, v in terms:
            if f.const and v.const:
                const += f.c * v.c
            elif f.const:
                if f.c != 0.0:
                    var.append((f.c, v.name))
            elif v.const:
                if v.c != 0.0:
                    var.append((v.c, f.name))
            else:
                var.append((1.0, f"{f.name} * {v.name}"))
        if not var:
            return Sym(const)
        if len(var) == 1 and const == 0.0 and var[0][0] == 1.0 and "*" not in var[0][1]:
            return Sym(name=var[0][1])
        parts = []
        for c, e in var:
            if c == 1.0:
                parts.append(e)
            elif c == -1.0:
                parts.append(f"-({e})")
            else:
                parts.append(f"{self.lit(c)} * {e}")
            self.flops += 1 if c == 1.0 or c == -1.0 else 2
        if const != 0.0:
            parts.append(self.lit(const))
            self.flops += 1
        self.flops -= 1
        return self.define(name, " + ".join(parts))

    def product(self, factors, name):
        c = 1.0
        names = []
        for f in factors:
            if f.const:
                c *= f.c
            else:
                names.append(f.name)
        if c == 0.0:
            return ZERO
        if not names:
            return Sym(c)
        if len(names) == 1 and c == 1.0:
            return Sym(name=names[0])
        expr = " * ".join(names)
        self.flops += len(names) - 1
        if c != 1.0:
            if c == -1.0:
                expr = f"-({expr})"
            else:
                expr = f"{self.lit(c)} * {expr}"
                self.flops += 1
        return self.define(name, expr)


def gen_E_axis(em: Emitter, tag, la, lb, PA, PB, inv2p, sign=False):
    """E[(i, j, t)] for i <= la, j <= lb.  With sign, E_t is multiplied by (-1)^t."""
    E = {(0, 0, 0): ONE}
    for i in range(la):
        for t in range(i + 2):
            terms = []
            if t >= 1:
                terms.append((inv2p, E.get((i, 0, t - 1), ZERO)))
            terms.append((PA, E.get((i, 0, t), ZERO)))
            terms.append((Sym(float(t + 1)), E.get((i, 0, t + 1), ZERO)))
            E[(i + 1, 0, t)] = em.lincomb(terms, f"{tag}{i + 1}_0_{t}")
    for j in range(lb):
        for i in range(la + 1):
            for t in range(i + j + 2):
                terms = []
                if t >= 1:
                    terms.append((inv2p, E.get((i, j, t - 1), ZERO)))
                terms.append((PB, E.get((i, j, t), ZERO)))
                terms.append((Sym(float(t + 1)), E.get((i, j, t + 1), ZERO)))
                E[(i, j + 1, t)] = em.lincomb(terms, f"{tag}{i}_{j + 1}_{t}")
    if sign:
        out = {}
        for (i, j, t), s in E.items():
            if t % 2 == 1:
                if s.const:
                    out[(i, j, t)] = Sym(-s.c)
                else:
                    out[(i, j, t)] = em.define(f"{tag}n{i}_{j}_{t}", f"-{s.name}")
            else:
                out[(i, j, t)] = s
        return out
    return E


def gen_products(em, tag, la, lb, Ex, Ey, Ez, extra=None):
    """Per Cartesian component pair (a, b): list of (hermite triple, Sym).
    ``extra`` (a Sym) multiplies every product (prefactor folding)."""
    out = []
    for ia, a in enumerate(comps(la)):
        for ib, b in enumerate(comps(lb)):
            lst = []
            for t in range(a[0] + b[0] + 1):
                for u in range(a[1] + b[1] + 1):
                    for v in range(a[2] + b[2] + 1):
                        fac = [Ex[(a[0], b[0], t)], Ey[(a[1], b[1], u)], Ez[(a[2], b[2], v)]]
                        if extra is not None:
                            fac.append(extra)
                        s = em.product(fac, f"{tag}{ia}_{ib}_{t}{u}{v}")
                        if not (s.const and s.c == 0.0):
                            lst.append(((t, u, v), s))
            out.append(lst)
    return out


def gen_R_scaled(em, L, F, PQs, r2):
    """R^{(0)}_{tuv} for t+u+v <= L by the scaled recursion (FP32 kernels).

    With Rs^{(n)} = R^{(n)} / (2 rho)^n (prefactor left out, it is folded
    into the E products):  Rs^{(n)}_{000} = (-1)^n F_n and
    Rs^{(n)}_{t+1,u,v} = (2 rho t) Rs^{(n+1)}_{t-1,u,v} + (2 rho X_PQ) Rs^{(n+1)}_{tuv},
    so Rs^{(0)} = R^{(0)} / pref while no intermediate grows like (2 rho)^L
    (which overflows FP32 for tight exponents)."""
    prev = {}
    for n in range(L, -1, -1):
        cur = {}
        for (t, u, v) in herm(L - n):
            if (t, u, v) == (0, 0, 0):
                cur[(t, u, v)] = Sym(name=f"{F}[{n}]") if n % 2 == 0 else em.define(f"r{n}_000", f"-{F}[{n}]")
                continue
            if t > 0:
                a, lo1, lo2, X = t - 1, (t - 1, u, v), (t - 2, u, v), PQs[0]
            elif u > 0:
                a, lo1, lo2, X = u - 1, (t, u - 1, v), (t, u - 2, v), PQs[1]
            else:
                a, lo1, lo2, X = v - 1, (t, u, v - 1), (t, u, v - 2), PQs[2]
            terms = [(Sym(name=X), prev[lo1])]
            if a > 0:
                terms.append((Sym(name=f"{r2}{a}"), prev[lo2]))
            cur[(t, u, v)] = em.lincomb(terms, f"r{n}_{t}_{u}_{v}")
        prev = cur
    return prev


def gen_R(em, L, pref, m2r, F, PQ):
    """R^{(0)}_{tuv} for t+u+v <= L.  Returns dict (t,u,v) -> Sym."""
    pw = [Sym(name=pref)]
    for n in range(1, L + 1):
        pw.append(em.product([pw[-1], Sym(name=m2r)], f"pw{n}"))
    prev = {}
    for n in range(L, -1, -1):
        cur = {}
        for (t, u, v) in herm(L - n):
            if (t, u, v) == (0, 0, 0):
                cur[(t, u, v)] = em.product([pw[n], Sym(name=f"{F}[{n}]")], f"r{n}_000")
                continue
            if t > 0:
                a, lo1, lo2, X = t - 1, (t - 1, u, v), (t - 2, u, v), PQ[0]
            elif u > 0:
                a, lo1, lo2, X = u - 1, (t, u - 1, v), (t, u - 2, v), PQ[1]
            else:
                a, lo1, lo2, X = v - 1, (t, u, v - 1), (t, u, v - 2), PQ[2]
            terms = [(Sym(name=X), prev[lo1])]
            if a > 0:
                terms.append((Sym(float(a)), prev[lo2]))
            cur[(t, u, v)] = em.lincomb(terms, f"r{n}_{t}_{u}_{v}")
        prev = cur
    return prev


def hidx(h):
    return {x: i for i, x in enumerate(h)}


# ---------------------------------------------------------------- kernel body
def class_name(bra, ket):
    return f"{bra[0]}{bra[1]}{ket[0]}{ket[1]}"


def quartet_counts(bra, ket):
    la, lb = bra
    lc, ld = ket
    L = la + lb + lc + ld
    HAB = len(herm(la + lb))
    S_ab = sum(math.prod(a[i] + b[i] + 1 for i in range(3)) for a in comps(la) for b in comps(lb))
    S_cd = sum(math.prod(a[i] + b[i] + 1 for i in range(3)) for a in comps(lc) for b in comps(ld))
    NCD = ncart(lc) * ncart(ld)
    NAB = ncart(la) * ncart(lb)
    return dict(L=L, HAB=HAB, S_ab=S_ab, S_cd=S_cd, NAB=NAB, NCD=NCD,
                xket=HAB * S_cd, bra=S_ab * NCD, R=math.comb(L + 4, 4))


def use_flat(bra, ket, prec="f64"):
    """Straight-line form with the contracted and half-transformed blocks in
    registers.  An FP32 value takes one register, an FP64 value two, so the
    FP32 kernels keep larger classes in registers."""
    c = quartet_counts(bra, ket)
    vals = c["NAB"] * c["NCD"] + c["HAB"] * c["NCD"]
    if prec == "f32" and max(bra + ket) <= 2:
        return vals <= FLAT_F32_VALUES and c["xket"] + c["bra"] <= 4500
    return vals <= 200 and c["xket"] + c["bra"] <= 2500


FLAT_F32_VALUES = 250


def crange_groups(bra, ket):
    """FP32 kernels of the l <= 2 classes too large for one straight-line
    kernel: one straight-line kernel per range of ket components c, each
    launched over all quartets (so no kernel carries more than one code path
    and the instruction cache holds it), each digesting its part of the block.
    Ranges are sized to at most CRANGE_VALUES block values."""
    if max(bra + ket) > 2 or use_flat(bra, ket, "f32"):
        return None
    c = quartet_counts(bra, ket)
    nc, nd = ncart(ket[0]), ncart(ket[1])
    per_c = (c["NAB"] + c["HAB"]) * nd
    g = max(1, CRANGE_VALUES // per_c)
    return [(c0, min(nc, c0 + g)) for c0 in range(0, nc, g)]


CRANGE_VALUES = 150

# Resident blocks of 128 threads per SM the FP32 class kernels are compiled
# for (__launch_bounds__ minimum; None: the compiler's choice, up to 255
# registers a thread).
F32_MIN_BLOCKS = None


PRIM_CUT = (
    "int jq0 = 0, jq1 = ik.z;\n"
    "if (pmode) {  // primitive split of a mixed build's FP64 list (gb::prim_range)\n"
    "  gb::prim_range(pairs.pq, ib.w + ip, ik.w, ik.z, pthr, pmode, jq0, jq1);\n"
    "  if (jq0 >= jq1) continue;\n"
    "}")


def gen_quartet_body(bra, ket, real, mode_flat, cds=None, rpath=None):
    """Device code computing acc[NAB*NCD] for one shell quartet (flat mode with
    `cds`: only those ket component pairs, acc[NAB*len(cds)]).

    Expects in scope: pairs (PairsView), bra/ket indices, ib/ik (int4 info),
    A, B, C, Dd centres (double4 or float4 per precision), boys tables."""
    la, lb = bra
    lc, ld = ket
    L = la + lb + lc + ld
    cnt = quartet_counts(bra, ket)
    NAB, NCD, HAB = cnt["NAB"], cnt["NCD"], cnt["HAB"]
    if cds is None:
        cds = list(range(NCD))
    assert mode_flat or len(cds) == NCD
    NS = len(cds)  # ket component pairs computed here
    f32 = real == "float"
    dfm = real == DFL        # double-float: FP32-pipe arithmetic, FP32-style scaled R and folded prefactors
    sc = f32 or dfm
    em = Emitter(real)
    hb = herm(la + lb)
    hbi = hidx(hb)
    L1 = L + 1
    E = em.emit
    pp, pp2 = ("pairs.ppf", "pairs.ppf2") if f32 else ("pairs.pp", "pairs.pp2")
    vec = "float" if f32 else "double"
    fma = "fmaf" if f32 else "fma"
    # the contracted block is held in the kernel's own precision: FP64 for
    # FP64 quartets; FP32 for FP32 quartets (a sum over <= 64 bra primitive
    # pairs of terms of one sign pattern; J and K still accumulate in FP64)
    E(f"{real} acc[{NAB * NS}];")
    E(f"#pragma unroll\nfor (int i = 0; i < {NAB * NS}; ++i) acc[i] = 0;")
    if not mode_flat:
        E(f"{real} Xl[{HAB * NCD}];")
        E(f"{real} Rc[{L1 * L1 * L1}];")
    E("for (int ip = ipart; ip < ib.z; ip += nsplit) {")
    E(PRIM_CUT)
    if dfm:
        E("const float4* pd_ = pairs.ppd + 5 * (ib.w + ip);")
        E("const float4 u0 = pd_[0], u1 = pd_[1], u2 = pd_[2], u3 = pd_[3], u4 = pd_[4];")
        E("const gb::dfl PAx(u0.x, u0.y), PAy(u0.z, u0.w), PAz(u1.x, u1.y);")
        E("const gb::dfl PBx(u1.z, u1.w), PBy(u2.x, u2.y), PBz(u2.z, u2.w);")
        E("const gb::dfl p(u3.x, u3.y), kp(u3.z, u3.w), inv2p(u4.x, u4.y);")
        E("const gb::dfl PCx = PAx + ACx, PCy = PAy + ACy, PCz = PAz + ACz;  // P - C")
    elif f32:
        # P - A, P - B and A - C were formed in FP64 and rounded once
        E("const float4 pa = pairs.ppf[ib.w + ip]; const float4 pb = pairs.ppf2[ib.w + ip];")
        E("const float p = pa.w, kp = pb.w, inv2p = __fdividef(0.5f, p);")
        E("const float PAx = pa.x, PAy = pa.y, PAz = pa.z;")
        E("const float PBx = pb.x, PBy = pb.y, PBz = pb.z;")
        E("const float PCx = PAx + ACx, PCy = PAy + ACy, PCz = PAz + ACz;  // P - C")
    else:
        E(f"const {vec}4 pa = {pp}[ib.w + ip]; const {vec}2 pb = {pp2}[ib.w + ip];")
        E(f"const {real} p = pa.w, kp = pb.x, inv2p = pb.y;")
        E(f"const {real} PAx = pa.x - A.x, PAy = pa.y - A.y, PAz = pa.z - A.z;")
        E(f"const {real} PBx = pa.x - B.x, PBy = pa.y - B.y, PBz = pa.z - B.z;")
    # X accumulators
    if mode_flat:
        for h in range(HAB):
            for k in range(NS):
                E(f"{real} x{h}_{k} = 0;")
    else:
        E(f"for (int i = 0; i < {HAB * NCD}; ++i) Xl[i] = 0;")
    E("for (int jq = jq0; jq < jq1; ++jq) {")
    if dfm:
        E("const float4* qd_ = pairs.ppd + 5 * (ik.w + jq);")
        E("const float4 w0 = qd_[0], w1 = qd_[1], w2 = qd_[2], w3 = qd_[3], w4 = qd_[4];")
        E("const gb::dfl QCx(w0.x, w0.y), QCy(w0.z, w0.w), QCz(w1.x, w1.y);")
        E("const gb::dfl QDx(w1.z, w1.w), QDy(w2.x, w2.y), QDz(w2.z, w2.w);")
        E("const gb::dfl q(w3.x, w3.y), kq(w3.z, w3.w), inv2q(w4.x, w4.y);")
    elif f32:
        E("const float4 qa = pairs.ppf[ik.w + jq]; const float4 qb = pairs.ppf2[ik.w + jq];")
        E("const float q = qa.w, kq = qb.w, inv2q = __fdividef(0.5f, q);")
        E("const float QCx = qa.x, QCy = qa.y, QCz = qa.z;")
        E("const float QDx = qb.x, QDy = qb.y, QDz = qb.z;")
    else:
        E(f"const {vec}4 qa = {pp}[ik.w + jq]; const {vec}2 qb = {pp2}[ik.w + jq];")
        E(f"const {real} q = qa.w, kq = qb.x, inv2q = qb.y;")
        E(f"const {real} QCx = qa.x - C.x, QCy = qa.y - C.y, QCz = qa.z - C.z;")
        E(f"const {real} QDx = qa.x - Dd.x, QDy = qa.y - Dd.y, QDz = qa.z - Dd.z;")
    em.flops = 0
    inv2q = Sym(name="inv2q")
    Ekx = gen_E_axis(em, "ekx", lc, ld, Sym(name="QCx"), Sym(name="QDx"), inv2q, sign=True)
    Eky = gen_E_axis(em, "eky", lc, ld, Sym(name="QCy"), Sym(name="QDy"), inv2q, sign=True)
    Ekz = gen_E_axis(em, "ekz", lc, ld, Sym(name="QCz"), Sym(name="QDz"), inv2q, sign=True)
    if sc:
        E(f"const {real} PQx = PCx - QCx, PQy = PCy - QCy, PQz = PCz - QCz;")
    else:
        E(f"const {real} PQx = pa.x - qa.x, PQy = pa.y - qa.y, PQz = pa.z - qa.z;")
    if dfm:
        E("const gb::dfl rs = gb::df_rsqrt(p + q);")
        E("const gb::dfl kqrs = kq * rs;")
    elif f32:
        E("const float rs = rsqrtf(p + q);")
        E("const float kqrs = kq * rs;")
    else:
        E("const double rs = rsqrt(p + q);")
    if mode_flat:
        kprod = gen_products(em, "ek", lc, ld, Ekx, Eky, Ekz, Sym(name="kqrs") if sc else None)
    flops_eket = em.flops
    em.flops = 0
    E(f"const {real} rho = p * q * rs * rs;")
    E(f"const {real} T = rho * (PQx * PQx + PQy * PQy + PQz * PQz);")
    if sc:
        E(f"const {real} r2 = rho + rho;")
        E(f"const {real} PQsx = r2 * PQx, PQsy = r2 * PQy, PQsz = r2 * PQz;")
        for a in range(1, L):
            E(f"const {real} r2k{a} = {float(a)!r}f * r2;")
    else:
        E(f"const {real} pref = kp * kq * rs;")
        E(f"const {real} m2r = -2 * rho;")
    E(f"{real} F[{L + 1}];")
    if dfm:
        E(f"gb::boys_df<{L}>(T, F, boysd);")
    elif f32:
        E(f"gb::boys_mixed<{L}>(T, F, boys, boysf, tsmall);")
    else:
        E(f"gb::boys_f64<{L}>(T, F, boys);")
    flops_setup = 16 + (kBoysCost(L))
    lam = rpath if rpath is not None else R_PATH_LAMBDA
    if mode_flat and lam is not None:
        R = gen_R_path(em, L, r_targets(bra, ket, cds), sc, lam)
    elif sc:
        R = gen_R_scaled(em, L, "F", ("PQsx", "PQsy", "PQsz"), "r2k")
    else:
        R = gen_R(em, L, "pref", "m2r", "F", ("PQx", "PQy", "PQz"))
    flops_R = em.flops
    em.flops = 0
    if mode_flat:
        for h, (t, u, v) in enumerate(hb):
            for k, cd in enumerate(cds):
                for (tau, nu, phi), s in kprod[cd]:
                    r = R[(t + tau, u + nu, v + phi)]
                    E(f"x{h}_{k} = {fma}({em.val(s)}, {em.val(r)}, x{h}_{k});")
                    em.flops += 2
    else:
        # cube store of R^(0)
        for (t, u, v), s in R.items():
            E(f"Rc[{(t * L1 + u) * L1 + v}] = {em.val(s)};")
        # per-axis E arrays
        for ax, Ek in (("x", Ekx), ("y", Eky), ("z", Ekz)):
            n = (lc + 1) * (ld + 1) * (lc + ld + 1)
            E(f"{real} ek{ax}a[{n}];")
            for i in range(lc + 1):
                for j in range(ld + 1):
                    for t in range(lc + ld + 1):
                        s = Ek.get((i, j, t), ZERO)
                        E(f"ek{ax}a[{(i * (ld + 1) + j) * (lc + ld + 1) + t}] = {em.val(s)};")
        cdl = [(c, d) for c in comps(lc) for d in comps(ld)]
        E(f"#pragma unroll 1\nfor (int cd = 0; cd < {NCD}; ++cd) {{")
        E(f"const int cx = c_cd_tab_{lc}{ld}[cd * 6 + 0], cy = c_cd_tab_{lc}{ld}[cd * 6 + 1], cz = c_cd_tab_{lc}{ld}[cd * 6 + 2];")
        E(f"const int dx = c_cd_tab_{lc}{ld}[cd * 6 + 3], dy = c_cd_tab_{lc}{ld}[cd * 6 + 4], dz = c_cd_tab_{lc}{ld}[cd * 6 + 5];")
        for h in range(HAB):
            E(f"{real} xh{h} = Xl[{h} * {NCD} + cd];")
        E("for (int tau = 0; tau <= cx + dx; ++tau) {")
        E(f"const {real} ex = ekxa[(cx * {ld + 1} + dx) * {lc + ld + 1} + tau]{' * kqrs' if sc else ''};")
        E("for (int nu = 0; nu <= cy + dy; ++nu) {")
        E(f"const {real} exy = ex * ekya[(cy * {ld + 1} + dy) * {lc + ld + 1} + nu];")
        E("for (int phi = 0; phi <= cz + dz; ++phi) {")
        E(f"const {real} e = exy * ekza[(cz * {ld + 1} + dz) * {lc + ld + 1} + phi];")
        E(f"const {real}* Rb = Rc + (tau * {L1} + nu) * {L1} + phi;")
        for h, (t, u, v) in enumerate(hb):
            E(f"xh{h} = {fma}(e, Rb[{(t * L1 + u) * L1 + v}], xh{h});")
        E("}}}")
        for h in range(HAB):
            E(f"Xl[{h} * {NCD} + cd] = xh{h};")
        E("}")
        em.flops += 2 * cnt["xket"]
    flops_x = em.flops
    E("}  // ket primitives")
    # bra E coefficients and products, emitted after the ket loop so that
    # they hold no registers while it runs
    em.flops = 0
    inv2p = Sym(name="inv2p")
    Ebx = gen_E_axis(em, "ebx", la, lb, Sym(name="PAx"), Sym(name="PBx"), inv2p)
    Eby = gen_E_axis(em, "eby", la, lb, Sym(name="PAy"), Sym(name="PBy"), inv2p)
    Ebz = gen_E_axis(em, "ebz", la, lb, Sym(name="PAz"), Sym(name="PBz"), inv2p)
    bprod = gen_products(em, "eb", la, lb, Ebx, Eby, Ebz, Sym(name="kp") if sc else None)
    flops_ebra = em.flops
    # bra transform
    em.flops = 0
    if mode_flat:
        for ab in range(NAB):
            for k in range(NS):
                expr = _dot(em, fma, [(sv, f"x{hbi[h]}_{k}") for h, sv in bprod[ab]])
                E(f"acc[{ab * NS + k}] += {expr};")
    else:
        E(f"#pragma unroll 1\nfor (int cd = 0; cd < {NCD}; ++cd) {{")
        for h in range(HAB):
            E(f"const {real} xh{h} = Xl[{h} * {NCD} + cd];")
        for ab in range(NAB):
            expr = _dot(em, fma, [(sv, f"xh{hbi[h]}") for h, sv in bprod[ab]])
            E(f"acc[{ab} * {NCD} + cd] += {expr};")
        E("}")
        em.flops = 2 * cnt["bra"]
    flops_bra = em.flops
    E("}  // bra primitives")
    body = "\n".join(em.lines)
    stats = dict(flops_per_primq=flops_setup + flops_R + flops_x + flops_eket,
                 flops_per_brap=flops_bra + flops_ebra, flat=mode_flat, **cnt)
    return body, stats


def use_chunk(bra, ket):
    """Classes with an f shell beyond the flat size: one thread per (shell
    quartet, Cartesian component c of the ket's first shell), so that the
    per-thread block is NAB x ND instead of NAB x NC x ND and the generated
    code stays compact (per-axis E arrays, R cube, bra E products in a local
    array)."""
    return max(bra + ket) >= 3 and (not use_flat(bra, ket) or sum(bra + ket) > 4)


def gen_R_rolled(em, L, f32):
    """R^{(0)}_{tuv}, t+u+v <= L, into the cube Rc (side L+1) by loops, in
    place: level n overwrites level n+1 from the highest total t+u+v down,
    so every value it reads (totals s-1 and s-2 of level n+1) is still there.
    FP64: R^{(n)}_{000} = pref (-2 rho)^n F_n,
          R^{(n)}_{t+1,u,v} = t R^{(n+1)}_{t-1,u,v} + X_PQ R^{(n+1)}_{tuv};
    FP32: the scaled form of gen_R_scaled (prefactor folded into the E products)."""
    E = em.emit
    L1 = L + 1
    real = "float" if f32 else "double"
    fma = "fmaf" if f32 else "fma"
    if f32:
        E(f"Rc[0] = {'-' if L % 2 else ''}F[{L}];")
    else:
        E(f"double pwv[{L + 1}];")
        E("pwv[0] = pref;")
        E(f"#pragma unroll\nfor (int n = 1; n <= {L}; ++n) pwv[n] = pwv[n - 1] * m2r;")
        E(f"Rc[0] = pwv[{L}] * F[{L}];")
    X = ("PQsx", "PQsy", "PQsz") if f32 else ("PQx", "PQy", "PQz")
    step = "r2" if f32 else "1.0"
    E(f"#pragma unroll\nfor (int n = {L - 1}; n >= 0; --n) {{")
    E(f"#pragma unroll 1\nfor (int s_ = {L} - n; s_ >= 1; --s_)")
    E("for (int t = s_; t >= 0; --t)")
    E("for (int u = s_ - t; u >= 0; --u) {")
    E("  const int v = s_ - t - u;")
    E(f"  const int o = (t * {L1} + u) * {L1} + v;")
    E(f"  {real} r;")
    E(f"  if (t > 0) {{ r = {X[0]} * Rc[o - {L1 * L1}]; if (t > 1) r = {fma}(({real})(t - 1) * {step}, Rc[o - {2 * L1 * L1}], r); }}")
    E(f"  else if (u > 0) {{ r = {X[1]} * Rc[o - {L1}]; if (u > 1) r = {fma}(({real})(u - 1) * {step}, Rc[o - {2 * L1}], r); }}")
    E(f"  else {{ r = {X[2]} * Rc[o - 1]; if (v > 1) r = {fma}(({real})(v - 1) * {step}, Rc[o - 2], r); }}")
    E("  Rc[o] = r;")
    E("}")
    if f32:
        E("Rc[0] = (n & 1) ? -F[n] : F[n];")
    else:
        E("Rc[0] = pwv[n] * F[n];")
    E("}")


def support(la, lb):
    """Per Cartesian pair (a, b): its Hermite support [(t, u, v)] in order."""
    out = []
    for a in comps(la):
        for b in comps(lb):
            out.append([(t, u, v) for t in range(a[0] + b[0] + 1) for u in range(a[1] + b[1] + 1)
                        for v in range(a[2] + b[2] + 1)])
    return out


def support_table(la, lb):
    """Packed per-axis indices of every support element: ix | iy << 8 | iz << 16,
    each the offset of E^{a_i b_i}_t in that axis's array."""
    T = la + lb + 1
    rows = []
    for (a, b), sup in zip([(a, b) for a in comps(la) for b in comps(lb)], support(la, lb)):
        for (t, u, v) in sup:
            ix = (a[0] * (lb + 1) + b[0]) * T + t
            iy = (a[1] * (lb + 1) + b[1]) * T + u
            iz = (a[2] * (lb + 1) + b[2]) * T + v
            rows.append(ix | (iy << 8) | (iz << 16))
    return f"static __device__ __constant__ int c_bsup_{la}{lb}[{len(rows)}] = {{{', '.join(map(str, rows))}}};", len(rows)


def gen_quartet_body_chunk(bra, ket, real):
    """Device code computing acc[NAB*ND] (one ket component c = ci) of one
    shell quartet.  Expects in scope: pairs, ib, ik, ci, the centres (FP64:
    A, B, C, Dd; FP32: ACx, ACy, ACz) and the Boys tables."""
    la, lb = bra
    lc, ld = ket
    L = la + lb + lc + ld
    L1 = L + 1
    cnt = quartet_counts(bra, ket)
    NAB, HAB = cnt["NAB"], cnt["HAB"]
    nd = ncart(ld)
    f32 = real == "float"
    fma = "fmaf" if f32 else "fma"
    em = Emitter(real)
    E = em.emit
    hb = herm(la + lb)
    hbi = hidx(hb)
    sup = support(la, lb)
    S_ab = sum(len(x) for x in sup)
    TB, TK = la + lb + 1, lc + ld + 1
    E(f"{real} acc[{NAB * nd}];")
    E(f"#pragma unroll\nfor (int i = 0; i < {NAB * nd}; ++i) acc[i] = 0;")
    E(f"{real} Xl[{HAB * nd}];")
    E(f"{real} Rc[{L1 * L1 * L1}];")
    E(f"{real} Ebp[{S_ab}];")
    E(f"const int cx = c_comp_{lc}[3 * ci], cy = c_comp_{lc}[3 * ci + 1], cz = c_comp_{lc}[3 * ci + 2];")
    E("for (int ip = ipart; ip < ib.z; ip += nsplit) {")
    E(PRIM_CUT)
    if f32:
        E("const float4 pa = pairs.ppf[ib.w + ip]; const float4 pb = pairs.ppf2[ib.w + ip];")
        E("const float p = pa.w, kp = pb.w, inv2p = __fdividef(0.5f, p);")
        E("const float PAx = pa.x, PAy = pa.y, PAz = pa.z;")
        E("const float PBx = pb.x, PBy = pb.y, PBz = pb.z;")
        E("const float PCx = PAx + ACx, PCy = PAy + ACy, PCz = PAz + ACz;  // P - C")
    else:
        E("const double4 pa = pairs.pp[ib.w + ip]; const double2 pb = pairs.pp2[ib.w + ip];")
        E("const double p = pa.w, kp = pb.x, inv2p = pb.y;")
        E("const double PAx = pa.x - A.x, PAy = pa.y - A.y, PAz = pa.z - A.z;")
        E("const double PBx = pa.x - B.x, PBy = pa.y - B.y, PBz = pa.z - B.z;")
    inv2p = Sym(name="inv2p")
    for ax in "xyz":
        Eb = gen_E_axis(em, f"eb{ax}", la, lb, Sym(name=f"PA{ax}"), Sym(name=f"PB{ax}"), inv2p)
        E(f"{real} eb{ax}a[{(la + 1) * (lb + 1) * TB}];")
        for i in range(la + 1):
            for j in range(lb + 1):
                for t in range(TB):
                    E(f"eb{ax}a[{(i * (lb + 1) + j) * TB + t}] = {em.val(Eb.get((i, j, t), ZERO))};")
    E(f"#pragma unroll 4\nfor (int k = 0; k < {S_ab}; ++k) {{")
    E(f"  const int w = c_bsup_{la}{lb}[k];")
    E(f"  Ebp[k] = ebxa[w & 255] * ebya[(w >> 8) & 255] * ebza[w >> 16]{' * kp' if f32 else ''};")
    E("}")
    E(f"for (int i = 0; i < {HAB * nd}; ++i) Xl[i] = 0;")
    E("for (int jq = jq0; jq < jq1; ++jq) {")
    if f32:
        E("const float4 qa = pairs.ppf[ik.w + jq]; const float4 qb = pairs.ppf2[ik.w + jq];")
        E("const float q = qa.w, kq = qb.w, inv2q = __fdividef(0.5f, q);")
        E("const float QCx = qa.x, QCy = qa.y, QCz = qa.z;")
        E("const float QDx = qb.x, QDy = qb.y, QDz = qb.z;")
        E("const float PQx = PCx - QCx, PQy = PCy - QCy, PQz = PCz - QCz;")
        E("const float rs = rsqrtf(p + q);")
        E("const float kqrs = kq * rs;")
    else:
        E("const double4 qa = pairs.pp[ik.w + jq]; const double2 qb = pairs.pp2[ik.w + jq];")
        E("const double q = qa.w, kq = qb.x, inv2q = qb.y;")
        E("const double QCx = qa.x - C.x, QCy = qa.y - C.y, QCz = qa.z - C.z;")
        E("const double QDx = qa.x - Dd.x, QDy = qa.y - Dd.y, QDz = qa.z - Dd.z;")
        E("const double PQx = pa.x - qa.x, PQy = pa.y - qa.y, PQz = pa.z - qa.z;")
        E("const double rs = rsqrt(p + q);")
    inv2q = Sym(name="inv2q")
    for ax in "xyz":
        Ek = gen_E_axis(em, f"ek{ax}", lc, ld, Sym(name=f"QC{ax}"), Sym(name=f"QD{ax}"), inv2q, sign=True)
        E(f"{real} ek{ax}a[{(lc + 1) * (ld + 1) * TK}];")
        for i in range(lc + 1):
            for j in range(ld + 1):
                for t in range(TK):
                    E(f"ek{ax}a[{(i * (ld + 1) + j) * TK + t}] = {em.val(Ek.get((i, j, t), ZERO))};")
    E(f"const {real} rho = p * q * rs * rs;")
    E(f"const {real} T = rho * (PQx * PQx + PQy * PQy + PQz * PQz);")
    if f32:
        E("const float r2 = 2.0f * rho;")
        E("const float PQsx = r2 * PQx, PQsy = r2 * PQy, PQsz = r2 * PQz;")
    else:
        E("const double pref = kp * kq * rs;")
        E("const double m2r = -2 * rho;")
    E(f"{real} F[{L + 1}];")
    if f32:
        E(f"gb::boys_mixed<{L}>(T, F, boys, boysf, tsmall);")
    else:
        E(f"gb::boys_f64<{L}>(T, F, boys);")
    gen_R_rolled(em, L, f32)
    # ket transform of the chunk's components (c = ci, d = 0..nd-1)
    E(f"#pragma unroll 1\nfor (int d = 0; d < {nd}; ++d) {{")
    E(f"const int dx = c_comp_{ld}[3 * d], dy = c_comp_{ld}[3 * d + 1], dz = c_comp_{ld}[3 * d + 2];")
    for h in range(HAB):
        E(f"{real} xh{h} = Xl[{h} * {nd} + d];")
    E("for (int tau = 0; tau <= cx + dx; ++tau) {")
    E(f"const {real} ex = ekxa[(cx * {ld + 1} + dx) * {TK} + tau]{' * kqrs' if f32 else ''};")
    E("for (int nu = 0; nu <= cy + dy; ++nu) {")
    E(f"const {real} exy = ex * ekya[(cy * {ld + 1} + dy) * {TK} + nu];")
    E("for (int phi = 0; phi <= cz + dz; ++phi) {")
    E(f"const {real} e = exy * ekza[(cz * {ld + 1} + dz) * {TK} + phi];")
    E(f"const {real}* Rb = Rc + (tau * {L1} + nu) * {L1} + phi;")
    for h, (t, u, v) in enumerate(hb):
        E(f"xh{h} = {fma}(e, Rb[{(t * L1 + u) * L1 + v}], xh{h});")
    E("}}}")
    for h in range(HAB):
        E(f"Xl[{h} * {nd} + d] = xh{h};")
    E("}")
    E("}  // ket primitives")
    # bra transform: acc[ab][d] += sum_k Ebp[k] X[h_k][d]
    E(f"#pragma unroll 1\nfor (int d = 0; d < {nd}; ++d) {{")
    for h in range(HAB):
        E(f"const {real} xh{h} = Xl[{h} * {nd} + d];")
    k = 0
    for ab in range(NAB):
        terms = []
        for (t, u, v) in sup[ab]:
            terms.append(f"Ebp[{k}]")
            k += 1
        expr = None
        for j, (t, u, v) in enumerate(sup[ab]):
            x = f"xh{hbi[(t, u, v)]}"
            expr = f"{terms[j]} * {x}" if expr is None else f"{fma}({terms[j]}, {x}, {expr})"
        E(f"acc[{ab} * {nd} + d] += {expr};")
    E("}")
    E("}  // bra primitives")
    flops_primq = 16 + kBoysCost(L) + 3 * cnt["R"] + 2 * HAB * cnt["S_cd"]
    flops_brap = 2 * S_ab * cnt["NCD"] + 2 * S_ab
    return "\n".join(em.lines), dict(flops_per_primq=flops_primq, flops_per_brap=flops_brap, flat=False, chunk=True,
                                     **cnt)



def _dot(em, fma, terms):
    """sum of coefficient * variable as a chain of FMAs (coefficient 1 folded)."""
    expr = None
    for sv, x in terms:
        unit = sv.const and sv.c == 1.0
        if expr is None:
            expr = x if unit else f"{em.val(sv)} * {x}"
            em.flops += 0 if unit else 1
        else:
            expr = f"({expr} + {x})" if unit else f"{fma}({em.val(sv)}, {x}, {expr})"
            em.flops += 1 if unit else 2
    return expr


def kBoysCost(L):
    # Taylor evaluation (8 FMA) + exp Taylor (8 FMA) + 2 per downward step (FMA + MUL)
    return 8 + (8 + 2 * L if L > 0 else 0)


CD_TAB_DONE = set()


def cd_table(lc, ld):
    rows = []
    for c in comps(lc):
        for d in comps(ld):
            rows += list(c) + list(d)
    return f"static __device__ __constant__ int c_cd_tab_{lc}{ld}[{len(rows)}] = {{{', '.join(map(str, rows))}}};"


def item_split(P, z):
    """Work items of one quartet (gb::item_split): the largest divisor of the
    bra pair's primitive-pair count z not above P."""
    d = min(P, z)
    while d > 1 and z % d:
        d -= 1
    return max(d, 1)


def split_of(bra, ket):
    """Most threads one shell quartet's bra primitive pairs are spread over:
    heavy classes are split so that the launch balances over quartets of very
    different primitive counts (1 to K^4); light ones are not (each part
    digests its partial block, which costs more than it saves there)."""
    if use_chunk(bra, ket):
        return 1
    c = quartet_counts(bra, ket)
    work = c["xket"] + 3 * c["R"]
    return 8 if work >= 1000 else (4 if work >= 300 else 1)


def gen_class_kernels(bra, ket):
    la, lb = bra
    lc, ld = ket
    na, nb, nc, nd = ncart(la), ncart(lb), ncart(lc), ncart(ld)
    flat = use_flat(bra, ket)
    chunk = use_chunk(bra, ket)
    nch = nc if chunk else 1  # threads per shell quartet
    P = split_of(bra, ket)    # bra primitive pairs of a quartet spread over up to P threads
    out = []
    stats = None
    precs = [("f64", "double"), ("f32", "float")] + ([("df", DFL)] if has_df(bra, ket) else [])
    for prec, real in precs:
        flat = use_flat(bra, ket, "f64" if prec == "df" else prec)
        name = class_name(bra, ket)
        # warp-run pre-reduction of the digestion (FP32 flat and range kernels):
        # J'_ab over the lanes of a row, the other targets over the lanes of a
        # quartet split over bra primitive pairs (classes with P > 1)
        warp = WARP_DIGEST.get(prec, False) and not chunk
        wtpl = f", {real}, true, {'true' if P > 1 else 'false'}" if warp else ""
        wargs = ", ws" if warp else ""
        # kernel variants of this precision: (name suffix, body, digest call, block size)
        variants = []
        if chunk:
            body, st = gen_quartet_body_chunk(bra, ket, real)
            variants.append(("", body, f"gb::digest_chunk<{na}, {nb}, {nc}, {nd}>(acc, ci, ib.x, ib.y, ik.x, ik.y, "
                                       f"{{dm}}, Jm, Km, Jlm, Klm, nbf);", na * nb * nd))
        elif prec == "f32" and crange_groups(bra, ket):
            for c0, c1 in crange_groups(bra, ket):
                cds = [c * nd + d for c in range(c0, c1) for d in range(nd)]
                body, st = gen_quartet_body(bra, ket, real, True, cds)
                variants.append((f"_c{c0}", body, f"gb::digest_crange<{na}, {nb}, {nc}, {nd}, {c0}, {c1}{wtpl}>(acc, ib.x, "
                                                  f"ib.y, ik.x, ik.y, {{dm}}, Jm, Km, Jlm, Klm, nbf{wargs});",
                                 na * nb * len(cds)))
            if (bra, ket) in RPATH_CLASSES:
                # the same ranges with the R recursion order of Algorithm 1
                # (greedy path search, lambda of fewest operations per range)
                for c0, c1 in crange_groups(bra, ket):
                    cds = [c * nd + d for c in range(c0, c1) for d in range(nd)]
                    body, _ = gen_quartet_body(bra, ket, real, True, cds, rpath=best_lambda(bra, ket, cds))
                    variants.append((f"r_c{c0}", body, f"gb::digest_crange<{na}, {nb}, {nc}, {nd}, {c0}, {c1}{wtpl}>(acc, "
                                                       f"ib.x, ib.y, ik.x, ik.y, {{dm}}, Jm, Km, Jlm, Klm, nbf{wargs});",
                                     na * nb * len(cds)))
        else:
            body, st = gen_quartet_body(bra, ket, real, flat)
            wt, wa = (wtpl, wargs) if flat else ("", "")
            variants.append(("", body, f"gb::{'digest' if flat else 'digest_loop'}<{na}, {nb}, {nc}, {nd}{wt}>"
                                       f"(acc, ib.x, ib.y, ik.x, ik.y, {{dm}}, Jm, Km, Jlm, Klm, nbf{wa});", na * nb * nc * nd))
        if prec == "f64":
            stats = st
        if real == "float":
            centres = ("  const float4 ah = pairs.Ahl[2 * bra], al = pairs.Ahl[2 * bra + 1];\n"
                       "  const float4 ch = pairs.Ahl[2 * ket], cl = pairs.Ahl[2 * ket + 1];\n"
                       "  // A - C from the split centres: no FP64 operation in an FP32 kernel\n"
                       "  const float ACx = (ah.x - ch.x) + (al.x - cl.x), ACy = (ah.y - ch.y) + (al.y - cl.y),\n"
                       "              ACz = (ah.z - ch.z) + (al.z - cl.z);")
            dmat = "Dfm"
        elif real == DFL:
            centres = ("  const float4 ah = pairs.Ahl[2 * bra], al = pairs.Ahl[2 * bra + 1];\n"
                       "  const float4 ch = pairs.Ahl[2 * ket], cl = pairs.Ahl[2 * ket + 1];\n"
                       "  // A - C in double-float from the split centres\n"
                       "  const gb::dfl ACx = (gb::dfl(ah.x) - gb::dfl(ch.x)) + (gb::dfl(al.x) - gb::dfl(cl.x));\n"
                       "  const gb::dfl ACy = (gb::dfl(ah.y) - gb::dfl(ch.y)) + (gb::dfl(al.y) - gb::dfl(cl.y));\n"
                       "  const gb::dfl ACz = (gb::dfl(ah.z) - gb::dfl(ch.z)) + (gb::dfl(al.z) - gb::dfl(cl.z));")
            dmat = "Ddm"
        else:
            centres = "  const double4 A = pairs.A[bra], B = pairs.B[bra], C = pairs.A[ket], Dd = pairs.B[ket];"
            dmat = "Dm"
        lbounds = f"128, {F32_MIN_BLOCKS}" if prec == "f32" and F32_MIN_BLOCKS else "128"
        for suffix, body, digest, nacc in variants:
            warpk = warp and ", ws);" in digest
            # primitive mode 1: the bra and ket primitive pairs are sorted by their
            # Schwarz factors, so an item whose first bra primitive pair misses the
            # cut with the largest ket one has no primitive quartet to evaluate
            early = ("" if warpk else
                     "  if (pmode == 1 && __fmul_rn(__ldg(pairs.pq + ib.w + ipart), __ldg(pairs.pq + ik.w)) < pthr)\n"
                     "    continue;  // nothing of this item reaches the cut: no digestion either\n")
            loop_head = (
                "  const long long stride = (long long)gridDim.x * blockDim.x;\n"
                "  for (long long t0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~(GB_WARP_SIZE - 1)); "
                "t0 < total; t0 += stride) {\n"
                "  // warp-uniform loop: every lane takes part in the digestion's shuffles\n"
                "  const long long tid = t0 + (threadIdx.x & (GB_WARP_SIZE - 1));\n"
                "  const bool act = tid < total;\n"
                "  const long long rt = act ? total - 1 - tid : 0;"
                if warpk else
                "  for (long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x; tid < total;\n"
                "       tid += (long long)gridDim.x * blockDim.x) {\n"
                "  const long long rt = total - 1 - tid;")
            warp_tail = (
                "  if (!act) {\n"
                "#pragma unroll\n"
                f"    for (int i = 0; i < {nacc}; ++i) acc[i] = 0;\n"
                "  }\n"
                "  const gb::WarpSeg ws = gb::warp_seg(act ? (unsigned)row : 0x80000000u | (threadIdx.x & 31),\n"
                "                                      act ? (unsigned)((qt - ipart) & 0x7fffffff) : 0x80000000u | (threadIdx.x & 31), act);"
                if warpk else "")
            out.append(f"""
__global__ void __launch_bounds__({lbounds}) eri_jk_{name}_{prec}{suffix}(const gb::JKArgs args) {{
  // persistent grid-stride loop over the quartets of this launch; the total is
  // read on the device (last entry of the row prefix) so launches need no host sync
  // Work items: rows.start is the prefix of items per row, a row's quartet
  // being split into gb::item_split({P}, K_ab) items over its bra primitive pairs; each
  // item runs as {nch} thread(s) (one per Cartesian component of the ket's
  // first shell).  Items are taken from the end: the rows are ordered by
  // ascending ket primitive count, so the heaviest work goes first and the
  // tail of the launch is light.
  // a launch may cover a sub-range of a class's rows (partial builds): its work
  // items are start[0] .. start[nrows] - 1
  const long long base = args.rows.start[0];
  const long long total = (args.rows.start[args.rows.nrows] - base) * {nch};
  const double* __restrict__ boys = args.boys;
  const float* __restrict__ boysf = args.boysf;
  const float2* __restrict__ boysd = args.boysd;
  const float tsmall = args.tsmall;
  (void)boys; (void)boysf; (void)boysd; (void)tsmall;
{loop_head}
  const long long qq = rt / {nch};
  const int ci = (int)(rt - qq * {nch});
  const long long qt = base + qq;
  (void)ci;
  int row;
  long long li;
  gb::locate_row(args.rows, qt, row, li);
  const int bra = __ldg(args.rows.bra + row);
  gb::PairsView pairs = args.pairs;
  const double* Dm = args.D;
  const float* Dfm = args.Df;
  const gb::dfl* Ddm = args.Ddf;
  double* Jm = args.J;
  double* Km = args.K;
  double* Jlm = args.Jlo;
  double* Klm = args.Klo;
  int nbf = args.nbf;
  (void)Dm; (void)Dfm; (void)Ddm; (void)Jlm; (void)Klm;
  if (args.mols) {{
    const gb::BatchMol& bm = args.mols[args.row_mol[row]];
    pairs = bm.pairs; Dm = bm.D; Dfm = bm.Df; Ddm = bm.Ddf; Jm = bm.J; Km = bm.K; nbf = bm.nbf;
    Jlm = bm.Jlo; Klm = bm.Klo;
  }}
  const int4 ib = pairs.info[bra];
  const int nsplit = gb::item_split({P}, ib.z);
  const long long qo = li / nsplit;
  const int ipart = (int)(li - qo * nsplit);
  const int ket = args.rows.klist ? __ldg(args.rows.klist + __ldg(args.rows.kofs + row) + qo)
                                  : __ldg(args.rows.ket0 + row) + (int)qo;
  const int4 ik = pairs.info[ket];
  const int pmode = args.pmode;
  const float pthr = pmode ? __ldg(args.rows.kthr + __ldg(args.rows.kofs + row) + qo) : 0.f;
{early}{centres}
{indent(body)}
  {real} s = 1;
  if (ib.x == ib.y) s *= 0.5f;
  if (ik.x == ik.y) s *= 0.5f;
  if (bra == ket) s *= 0.5f;
#pragma unroll
  for (int i = 0; i < {nacc}; ++i) acc[i] *= s;
{warp_tail}
  {digest.format(dm=dmat)}
  }}
}}
""")
        if bra == ket and prec == "f64":
            nab = na * nb
            if chunk:
                sbody = body  # the chunked FP64 body of this class (one ket component c = ci)
                diag = (f"  for (int b = 0; b < {nb}; ++b)\n"
                        f"    dg[ci * {nb} + b] = acc[(ci * {nb} + b) * {nd} + b];")
            else:
                sbody = body_f64_for_schwarz(bra, ket)
                diag = f"  for (int d = 0; d < {nab}; ++d) dg[d] = acc[d * {nab} + d];"
            out.append(f"""
__global__ void __launch_bounds__(128) eri_schwarz_{la}{lb}(const gb::SchwarzArgs sa) {{
  // one thread per (pair, component c = ci of shell a, part ipart of the bra
  // primitive pairs): the partial diagonal elements (ab|ab)_ii of its bra
  // primitive pairs go to its own slots of sa.diag (zeroed by the caller);
  // gb::k_schwarz_finish adds the parts in a fixed order and takes
  // Q = sqrt(max_i |(ab|ab)_ii|), so Q does not depend on scheduling
  constexpr int S = gb::kSchwarzSplit;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)sa.count * {nch} * S) return;
  const int ipart = (int)(tid % S);
  const long long pc = tid / S;
  const int i = (int)(pc / {nch}), ci = (int)(pc - (long long)i * {nch});
  (void)ci;
  const int bra = sa.first + i, ket = bra;
  const gb::PairsView& pairs = sa.pairs;
  const double* __restrict__ boys = sa.boys;
  const float* __restrict__ boysf = nullptr;
  const float tsmall = 0.f;
  (void)boysf; (void)tsmall;
  const int4 ib = pairs.info[bra], ik = ib;
  const int nsplit = min(S, ib.z);
  if (ipart >= nsplit) return;
  const double4 A = pairs.A[bra], B = pairs.B[bra], C = A, Dd = B;
  const int pmode = 0;  // every primitive quartet
  const float pthr = 0.f;
  (void)pthr;
{indent(sbody)}
  double* dg = sa.diag + ((size_t)i * S + ipart) * {nab};
{diag}
}}
""")
    return "".join(out), stats


_BODY_CACHE = {}


def body_f64_for_schwarz(bra, ket):
    key = (bra, ket)
    if key not in _BODY_CACHE:
        _BODY_CACHE[key] = gen_quartet_body(bra, ket, "double", use_flat(bra, ket))[0]
    return _BODY_CACHE[key]


# ---------------------------------------------------------------- gradient kernels
def comp_table(l):
    rows = []
    for c in comps(l):
        rows += list(c)
    return f"static __device__ __constant__ int c_comp_{l}[{len(rows)}] = {{{', '.join(map(str, rows))}}};"


def _store_axis_array(E, em, name, li, lj, E_axis, real="double"):
    """Write per-axis E[(i,j,t)] (i <= li, j <= lj) into a flat local array."""
    T = li + lj + 1
    E(f"{real} {name}[{(li + 1) * (lj + 1) * T}];")
    for i in range(li + 1):
        for j in range(lj + 1):
            for t in range(T):
                sv = E_axis.get((i, j, t), ZERO)
                E(f"{name}[{(i * (lj + 1) + j) * T + t}] = {em.val(sv)};")


def use_grad_chunk(bra, ket):
    """Derivative kernels of classes with an f shell: one thread per (work
    item, Cartesian component c of the ket's first shell), as the J/K chunked
    form, so that the per-thread arrays hold NAB x ND (not NAB x NC x ND)
    values and the R cube is filled by the rolled recursion.  In one piece
    the (ff|ff) derivative kernel needs a 410 KB stack frame per thread."""
    return max(bra + ket) >= 3


def grad_threads(bra, ket):
    """Threads per work item of a derivative kernel."""
    return ncart(ket[0]) if use_grad_chunk(bra, ket) else 1


def gen_grad_kernel(bra, ket, prec="f64"):
    """Nuclear-gradient kernel of one class, FP64 or FP32 (the mixed gradient's
    small-bound quartets), plus its launcher for both.

    Per unique shell quartet: Gamma_abcd = s (4 D_ab D_cd - D_ac D_bd - D_ad D_bc)
    (the weight of (ab|cd) in E = tr(DJ)/2 - tr(DK)/4 summed over its eight
    images, s the degeneracy factor); derivative integrals by the shift rule
    d/dA_x phi_a = 2 alpha phi_{a+1x} - a_x phi_{a-1x}, which in the Hermite
    expansion only changes the x-axis coefficient:
      E'^{ab}_t = 2 alpha E^{a_x+1, b_x}_t - a_x E^{a_x-1, b_x}_t  (centre A),
      E'^{ab}_t = 2 beta  E^{a_x, b_x+1}_t - b_x E^{a_x, b_x-1}_t  (centre B),
    the same on the ket for centre C, and dI/dD = -(dI/dA + dI/dB + dI/dC)
    (translational invariance).  The FP32 form works from the centre
    differences formed in FP64 and rounded once (as the FP32 J/K kernels), with
    the scaled R recursion (prefactor folded into the ket and bra weights), Gamma
    formed in FP64 from D and rounded, and the per-item gradient sums added to
    dE/dR in FP64.  Both forms walk the work items of a launch (rows.start[0]
    .. rows.start[nrows] - 1, read on the device) with a grid-stride loop,
    heaviest first, and read explicit ket lists where the rows carry them."""
    la, lb = bra
    lc, ld = ket
    L = la + lb + lc + ld
    L1 = L + 1            # highest Hermite order needed
    S = L1 + 1            # cube side of R
    na, nb, nc, nd = ncart(la), ncart(lb), ncart(lc), ncart(ld)
    NAB, NCD = na * nb, nc * nd
    h1 = herm(la + lb + 1)
    h0 = herm(la + lb)
    H1, H0 = len(h1), len(h0)
    f32 = prec == "f32"
    real = "float" if f32 else "double"
    fma = "fmaf" if f32 else "fma"
    zero = "0.0f" if f32 else "0.0"
    em = Emitter(real)
    E = em.emit
    name = class_name(bra, ket)
    TB = la + lb + 3      # t range of the bra arrays (i <= la+1, j <= lb+1)
    TK = lc + ld + 2      # t range of the ket arrays (i <= lc+1, j <= ld)
    chunk = use_grad_chunk(bra, ket)
    nthr = nc if chunk else 1
    NCDx = nd if chunk else NCD  # ket component pairs per thread
    P = split_of(bra, ket)
    E(f"__global__ void __launch_bounds__(128) eri_grad_{name}_{prec}(const gb::GradArgs args) {{")
    E("const long long base = args.rows.start[0];")
    E(f"const long long total = (args.rows.start[args.rows.nrows] - base) * {nthr};")
    E("for (long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x; gt < total;")
    E("     gt += (long long)gridDim.x * blockDim.x) {")
    # work items as in the J/K kernels: a quartet split into item_split(P, K_ab) items
    # over its bra primitive pairs, heaviest rows (largest ket primitive count,
    # at the end of the range) first so that the launch tail is light
    E("const long long rt = total - 1 - gt;")
    E(f"const long long it = rt / {nthr};")
    E(f"const int cthr = (int)(rt - it * {nthr});")
    E("(void)cthr;")
    E("int row;")
    E("long long li;")
    E("gb::locate_row(args.rows, base + it, row, li);")
    E("const int bra = __ldg(args.rows.bra + row);")
    E("const gb::PairsView& pairs = args.pairs;")
    E("const double* __restrict__ boys = args.boys;")
    E("const float* __restrict__ boysf = args.boysf;")
    E("const float tsmall = args.tsmall;")
    E("(void)boysf; (void)tsmall;")
    E("const double* __restrict__ Dm = args.D;")
    E("const int n = args.nbf;")
    E("const int4 ib = pairs.info[bra];")
    E(f"const int nsplit = gb::item_split({P}, ib.z);")
    E("const long long qo = li / nsplit;")
    E("const int ipart = (int)(li - qo * nsplit);")
    E("const int ket = args.rows.klist ? __ldg(args.rows.klist + __ldg(args.rows.kofs + row) + qo)")
    E("                                : __ldg(args.rows.ket0 + row) + (int)qo;")
    E("const int4 ik = pairs.info[ket];")
    E("const int pmode = args.pmode;")
    E("const float pthr = pmode ? __ldg(args.rows.kthr + __ldg(args.rows.kofs + row) + qo) : 0.f;")
    E("if (pmode == 1 && __fmul_rn(__ldg(pairs.pq + ib.w + ipart), __ldg(pairs.pq + ik.w)) < pthr)")
    E("  continue;  // primitive mode 1: nothing of this item reaches the cut")
    if f32:
        E("const float4 ah = pairs.Ahl[2 * bra], al = pairs.Ahl[2 * bra + 1];")
        E("const float4 ch = pairs.Ahl[2 * ket], cl = pairs.Ahl[2 * ket + 1];")
        E("const float ACx = (ah.x - ch.x) + (al.x - cl.x), ACy = (ah.y - ch.y) + (al.y - cl.y),")
        E("            ACz = (ah.z - ch.z) + (al.z - cl.z);")
    else:
        E("const double4 A = pairs.A[bra], B = pairs.B[bra], C = pairs.A[ket], Dd = pairs.B[ket];")
    E("double s = 1.0;")
    E("if (ib.x == ib.y) s *= 0.5;")
    E("if (ik.x == ik.y) s *= 0.5;")
    E("if (bra == ket) s *= 0.5;")
    E(f"{real} G[{NAB * NCDx}];")
    E(f"for (int ab = 0; ab < {NAB}; ++ab) {{")
    E(f"  const int a = ib.x + ab / {nb}, b = ib.y + ab % {nb};")
    E(f"  for (int cd = 0; cd < {NCDx}; ++cd) {{")
    if chunk:
        E("    const int c = ik.x + cthr, d = ik.y + cd;")
    else:
        E(f"    const int c = ik.x + cd / {nd}, d = ik.y + cd % {nd};")
    E(f"    G[ab * {NCDx} + cd] = ({real})(s * (4.0 * Dm[(size_t)a * n + b] * Dm[(size_t)c * n + d] - Dm[(size_t)a * n + c] * Dm[(size_t)b * n + d] - Dm[(size_t)a * n + d] * Dm[(size_t)b * n + c]));")
    E("  }")
    E("}")
    E(f"{real} gA[3] = {{0, 0, 0}}, gB[3] = {{0, 0, 0}}, gC[3] = {{0, 0, 0}};")
    E(f"{real} X[{H1 * NCDx}];")
    E(f"{real} XC[{3 * H0 * NCDx}];")
    E(f"{real} Rc[{S * S * S}];")
    E("for (int ip = ipart; ip < ib.z; ip += nsplit) {")
    E(PRIM_CUT)
    if f32:
        E("const float4 pa = pairs.ppf[ib.w + ip]; const float4 pb = pairs.ppf2[ib.w + ip];")
        E("const float p = pa.w, kp = pb.w, inv2p = __fdividef(0.5f, p);")
        E("const float alpha = (float)pairs.alpha[ib.w + ip], beta = p - alpha;")
        E("const float PAx = pa.x, PAy = pa.y, PAz = pa.z;")
        E("const float PBx = pb.x, PBy = pb.y, PBz = pb.z;")
        E("const float PCx = PAx + ACx, PCy = PAy + ACy, PCz = PAz + ACz;  // P - C")
    else:
        E("const double4 pa = pairs.pp[ib.w + ip]; const double2 pb = pairs.pp2[ib.w + ip];")
        E("const double p = pa.w, kp = pb.x, inv2p = pb.y, alpha = pairs.alpha[ib.w + ip], beta = p - alpha;")
        E("const double PAx = pa.x - A.x, PAy = pa.y - A.y, PAz = pa.z - A.z;")
        E("const double PBx = pa.x - B.x, PBy = pa.y - B.y, PBz = pa.z - B.z;")
    inv2p = Sym(name="inv2p")
    for ax in "xyz":
        Eb = gen_E_axis(em, f"gb{ax}", la + 1, lb + 1, Sym(name=f"PA{ax}"), Sym(name=f"PB{ax}"), inv2p)
        _store_axis_array(E, em, f"eb{ax}", la + 1, lb + 1, Eb, real)
    E(f"for (int i = 0; i < {H1 * NCDx}; ++i) X[i] = 0;")
    E(f"for (int i = 0; i < {3 * H0 * NCDx}; ++i) XC[i] = 0;")
    E("for (int jq = jq0; jq < jq1; ++jq) {")
    if f32:
        E("const float4 qa = pairs.ppf[ik.w + jq]; const float4 qb = pairs.ppf2[ik.w + jq];")
        E("const float q = qa.w, kq = qb.w, inv2q = __fdividef(0.5f, q), gam2 = 2.0f * (float)pairs.alpha[ik.w + jq];")
        E("const float QCx = qa.x, QCy = qa.y, QCz = qa.z;")
        E("const float QDx = qb.x, QDy = qb.y, QDz = qb.z;")
    else:
        E("const double4 qa = pairs.pp[ik.w + jq]; const double2 qb = pairs.pp2[ik.w + jq];")
        E("const double q = qa.w, kq = qb.x, inv2q = qb.y, gam2 = 2.0 * pairs.alpha[ik.w + jq];")
        E("const double QCx = qa.x - C.x, QCy = qa.y - C.y, QCz = qa.z - C.z;")
        E("const double QDx = qa.x - Dd.x, QDy = qa.y - Dd.y, QDz = qa.z - Dd.z;")
    inv2q = Sym(name="inv2q")
    for ax in "xyz":
        Ek = gen_E_axis(em, f"gk{ax}", lc + 1, ld, Sym(name=f"QC{ax}"), Sym(name=f"QD{ax}"), inv2q, sign=True)
        _store_axis_array(E, em, f"ek{ax}", lc + 1, ld, Ek, real)
    if f32:
        E("const float PQx = PCx - QCx, PQy = PCy - QCy, PQz = PCz - QCz;")
        E("const float rs = rsqrtf(p + q);")
        E("const float kqrs = kq * rs;  // ket weight of the scaled R (the bra weight kp follows below)")
        E("const float rho = p * q * rs * rs;")
        E("const float T = rho * (PQx * PQx + PQy * PQy + PQz * PQz);")
        E("const float r2 = 2.0f * rho;")
        E("const float PQsx = r2 * PQx, PQsy = r2 * PQy, PQsz = r2 * PQz;")
        for a in range(1, L1):
            E(f"const float r2k{a} = {float(a)!r}f * r2;")
        E(f"float F[{L1 + 1}];")
        E(f"gb::boys_mixed<{L1}>(T, F, boys, boysf, tsmall);")
    else:
        E("const double PQx = pa.x - qa.x, PQy = pa.y - qa.y, PQz = pa.z - qa.z;")
        E("const double rs = rsqrt(p + q);")
        E("const double rho = p * q * rs * rs;")
        E("const double T = rho * (PQx * PQx + PQy * PQy + PQz * PQz);")
        E("const double pref = kp * kq * rs;")
        E("const double m2r = -2 * rho;")
        E(f"double F[{L1 + 1}];")
        E(f"gb::boys_f64<{L1}>(T, F, boys);")
    if chunk:
        gen_R_rolled(em, L1, f32)
    else:
        R = gen_R_scaled(em, L1, "F", ("PQsx", "PQsy", "PQsz"), "r2k") if f32 else \
            gen_R(em, L1, "pref", "m2r", "F", ("PQx", "PQy", "PQz"))
        for (t, u, v), sv in R.items():
            E(f"Rc[{(t * S + u) * S + v}] = {em.val(sv)};")
    kw = " * kqrs" if f32 else ""
    E(f"for (int cd = 0; cd < {NCDx}; ++cd) {{")
    if chunk:
        E("  const int c = cthr, d = cd;")
    else:
        E(f"  const int c = cd / {nd}, d = cd % {nd};")
    E(f"  const int cx = c_comp_{lc}[3 * c], cy = c_comp_{lc}[3 * c + 1], cz = c_comp_{lc}[3 * c + 2];")
    E(f"  const int dx = c_comp_{ld}[3 * d], dy = c_comp_{ld}[3 * d + 1], dz = c_comp_{ld}[3 * d + 2];")
    # X over H1
    for k in range(H1):
        E(f"  {real} xh{k} = X[{k * NCDx} + cd];")
    E("  for (int tau = 0; tau <= cx + dx; ++tau) {")
    E(f"    const {real} ex = ekx[(cx * {ld + 1} + dx) * {TK} + tau]{kw};")
    E("    for (int nu = 0; nu <= cy + dy; ++nu) {")
    E(f"      const {real} exy = ex * eky[(cy * {ld + 1} + dy) * {TK} + nu];")
    E("      for (int phi = 0; phi <= cz + dz; ++phi) {")
    E(f"        const {real} e = exy * ekz[(cz * {ld + 1} + dz) * {TK} + phi];")
    E(f"        const {real}* Rb = Rc + (tau * {S} + nu) * {S} + phi;")
    for k, (t, u, v) in enumerate(h1):
        E(f"        xh{k} = {fma}(e, Rb[{(t * S + u) * S + v}], xh{k});")
    E("  }}}")
    for k in range(H1):
        E(f"  X[{k * NCDx} + cd] = xh{k};")
    # XC for the three directions
    for di, ax in enumerate("xyz"):
        cc = {"x": ("cx", "dx"), "y": ("cy", "dy"), "z": ("cz", "dz")}
        E("  {")
        for k in range(H0):
            E(f"  {real} xc{k} = XC[{(di * H0 + k) * NCDx} + cd];")
        rng = {a: (f"{cc[a][0]} + {cc[a][1]}" + (" + 1" if a == ax else "")) for a in "xyz"}
        idx = {"x": "tau", "y": "nu", "z": "phi"}

        def coef(a):
            c, d = cc[a]
            v = idx[a]
            if a != ax:
                return f"ek{a}[({c} * {ld + 1} + {d}) * {TK} + {v}]"
            return (f"(gam2 * ek{a}[(({c} + 1) * {ld + 1} + {d}) * {TK} + {v}]"
                    f" - ({c} > 0 ? {c} * ek{a}[(({c} - 1) * {ld + 1} + {d}) * {TK} + {v}] : {zero}))")
        E(f"  for (int tau = 0; tau <= {rng['x']}; ++tau) {{")
        E(f"    const {real} ex = {coef('x')}{kw};")
        E(f"    for (int nu = 0; nu <= {rng['y']}; ++nu) {{")
        E(f"      const {real} exy = ex * {coef('y')};")
        E(f"      for (int phi = 0; phi <= {rng['z']}; ++phi) {{")
        E(f"        const {real} e = exy * {coef('z')};")
        E(f"        const {real}* Rb = Rc + (tau * {S} + nu) * {S} + phi;")
        for k, (t, u, v) in enumerate(h0):
            E(f"        xc{k} = {fma}(e, Rb[{(t * S + u) * S + v}], xc{k});")
        E("  }}}")
        for k in range(H0):
            E(f"  XC[{(di * H0 + k) * NCDx} + cd] = xc{k};")
        E("  }")
    E("}")  # cd
    E("}  // ket primitives")
    # contraction with Gamma
    TBs = TB
    two = "2.0f" if f32 else "2.0"
    one = "1.0f" if f32 else "1.0"
    E(f"for (int ab = 0; ab < {NAB}; ++ab) {{")
    E(f"  const int a = ab / {nb}, b = ab % {nb};")
    E(f"  const int ax_ = c_comp_{la}[3 * a], ay_ = c_comp_{la}[3 * a + 1], az_ = c_comp_{la}[3 * a + 2];")
    E(f"  const int bx_ = c_comp_{lb}[3 * b], by_ = c_comp_{lb}[3 * b + 1], bz_ = c_comp_{lb}[3 * b + 2];")
    E("  const int ai[3] = {ax_, ay_, az_}, bi[3] = {bx_, by_, bz_};")
    E(f"  const {real}* ebv[3] = {{ebx, eby, ebz}};")
    E(f"  for (int cd = 0; cd < {NCDx}; ++cd) {{")
    E(f"    const {real} g = G[ab * {NCDx} + cd]{' * kp' if f32 else ''};")
    E("    if (g == 0) continue;")
    # plain bra E over H0 for the C derivative; derivative bra E over H1 for A and B
    E("    for (int dir = 0; dir < 3; ++dir) {")
    E(f"      {real} vA = 0, vB = 0, vC = 0;")
    E("      const int rx = ai[0] + bi[0] + (dir == 0), ry = ai[1] + bi[1] + (dir == 1), rz = ai[2] + bi[2] + (dir == 2);")
    E("      for (int t = 0; t <= rx; ++t) for (int u = 0; u <= ry; ++u) for (int v = 0; v <= rz; ++v) {")
    E("        const int tt[3] = {t, u, v};")
    E(f"        {real} fA = {one}, fB = {one}, f0 = {one};")
    E("        for (int k = 0; k < 3; ++k) {")
    E(f"          const {real}* e = ebv[k];")
    E(f"          const {real} base = e[(ai[k] * {lb + 2} + bi[k]) * {TBs} + tt[k]];")
    E("          if (k == dir) {")
    E(f"            const {real} up_a = e[((ai[k] + 1) * {lb + 2} + bi[k]) * {TBs} + tt[k]];")
    E(f"            const {real} dn_a = ai[k] > 0 ? e[((ai[k] - 1) * {lb + 2} + bi[k]) * {TBs} + tt[k]] : {zero};")
    E(f"            const {real} up_b = e[(ai[k] * {lb + 2} + bi[k] + 1) * {TBs} + tt[k]];")
    E(f"            const {real} dn_b = bi[k] > 0 ? e[(ai[k] * {lb + 2} + bi[k] - 1) * {TBs} + tt[k]] : {zero};")
    E(f"            fA *= {two} * alpha * up_a - ai[k] * dn_a;")
    E(f"            fB *= {two} * beta * up_b - bi[k] * dn_b;")
    E("            f0 *= base;")
    E("          } else { fA *= base; fB *= base; f0 *= base; }")
    E("        }")
    E("        const int tot = t + u + v;")
    E("        const int h = tot * (tot + 1) * (tot + 2) / 6 + (tot - t) * (tot - t + 1) / 2 + (tot - t - u);")
    E(f"        const {real} xv = X[h * {NCDx} + cd];")
    E(f"        vA = {fma}(fA, xv, vA);")
    E(f"        vB = {fma}(fB, xv, vB);")
    E(f"        if (tot <= {la + lb} && t <= ai[0] + bi[0] && u <= ai[1] + bi[1] && v <= ai[2] + bi[2])")
    E(f"          vC = {fma}(f0, XC[(dir * {H0} + h) * {NCDx} + cd], vC);")
    E("      }")
    E(f"      gA[dir] = {fma}(g, vA, gA[dir]);")
    E(f"      gB[dir] = {fma}(g, vB, gB[dir]);")
    E(f"      gC[dir] = {fma}(g, vC, gC[dir]);")
    E("    }")
    E("  }")
    E("}")
    E("}  // bra primitives")
    E("const int2 atb = args.atoms[bra], atk = args.atoms[ket];")
    E("for (int k = 0; k < 3; ++k) {  // the item's sums, added in FP64")
    E("  atomicAdd(args.grad + 3 * atb.x + k, (double)gA[k]);")
    E("  atomicAdd(args.grad + 3 * atb.y + k, (double)gB[k]);")
    E("  atomicAdd(args.grad + 3 * atk.x + k, (double)gC[k]);")
    E("  atomicAdd(args.grad + 3 * atk.y + k, -((double)gA[k] + (double)gB[k] + (double)gC[k]));")
    E("}")
    E("}")  # grid-stride loop
    E("}")
    if f32:
        E(f"""
int launch_grad_{name}(int prec, const gb::GradArgs& a, int grid, cudaStream_t s) {{
  if (grid <= 0) return 0;
  if (prec == 0) eri_grad_{name}_f64<<<grid, 128, 0, s>>>(a);
  else eri_grad_{name}_f32<<<grid, 128, 0, s>>>(a);
  return (int)cudaGetLastError();
}}""")
    return "\n".join(em.lines) + "\n"


# ---------------------------------------------------------------- path search (analysis)
def r_targets(bra, ket, cds=None):
    """The Hermite integrals R^(0)_{tuv} a kernel body reads: bra Hermite
    index plus the support of every ket component pair it computes."""
    hb = herm(bra[0] + bra[1])
    cdl = [(c, d) for c in comps(ket[0]) for d in comps(ket[1])]
    out = set()
    for k in (range(len(cdl)) if cds is None else cds):
        c, d = cdl[k]
        for tau in range(c[0] + d[0] + 1):
            for nu in range(c[1] + d[1] + 1):
                for phi in range(c[2] + d[2] + 1):
                    out.update((0, t + tau, u + nu, v + phi) for (t, u, v) in hb)
    return out


def _r_children(node, axis):
    n, *k = node
    one = list(k)
    one[axis] -= 1
    kids = [(n + 1, *one)]
    if k[axis] >= 2:
        two = list(k)
        two[axis] -= 2
        kids.append((n + 1, *two))
    return kids


def r_path(targets, lam=None, rng=None):
    """Nodes R^(n)_{tuv} needed to reach `targets` through the recursion
    R^(n)_{k} = (k_i - 1) R^(n+1)_{k - 2e_i} + X_i R^(n+1)_{k - e_i}.

    lam None: the fixed order the emitted code uses (reduce t first, then u,
    then v).  Otherwise the greedy search of the paper's Graph Compiler
    (Sec. 5, Algorithm 1): going down from the highest total angular momentum,
    every node takes the axis ("recurrence position") of least cost
    (new - reused) + lam * (angular momentum of the new nodes).  rng (a
    random.Random): every node takes a random valid axis instead, the
    baseline the paper compares its search with.
    Returns {node: axis or None}."""
    chosen = {}
    todo = set(targets)
    while todo:
        top = max(sum(x[1:]) for x in todo)
        level = sorted(x for x in todo if sum(x[1:]) == top)
        todo -= set(level)
        for node in level:
            if top == 0:
                chosen[node] = None
                continue
            axes = [i for i in range(3) if node[1 + i] > 0]
            if rng is not None:
                best = rng.choice(axes)
            elif lam is None:
                best = axes[0]
            else:
                def cost(i):
                    kids = _r_children(node, i)
                    new = [c for c in kids if c not in chosen and c not in todo]
                    return (len(new) - (len(kids) - len(new))) + lam * sum(sum(c[1:]) for c in new)
                best = min(axes, key=cost)
            chosen[node] = best
            todo.update(c for c in _r_children(node, best) if c not in chosen)
    return chosen


def has_df(bra, ket):
    """Classes that also carry a double-float kernel (the mixed build's
    largest-bound quartets): every l <= 2 class (the f classes' chunked form
    keeps FP64)."""
    return max(bra + ket) <= 2


# Warp-run pre-reduction of the digestion per precision (flat and range
# digestion forms; see gb::WarpSeg).
WARP_DIGEST = {"f32": True, "f64": False}

# Classes whose FP32 range kernels are also emitted with Algorithm 1's
# recursion order (launched when the library's R-path option is set): the
# three with the largest FP32 share of the l <= 2 workloads.
RPATH_CLASSES = [((2, 2), (2, 2)), ((2, 2), (2, 1)), ((2, 1), (2, 1))]
RPATH_LAMBDAS = (0.0, 0.5, 1.0, 2.0)


def best_lambda(bra, ket, cds):
    """The lambda of Algorithm 1's cost whose path over the R values a
    kernel reads has the fewest operations (ties: the smallest lambda)."""
    t = r_targets(bra, ket, cds)
    return min(RPATH_LAMBDAS, key=lambda lam: (r_path_flops(r_path(t, lam)), lam))


# Recursion order of the R values in the straight-line kernels: None keeps the
# fixed t-then-u-then-v order over full levels (the code the GPU runs has been
# measured with); a number selects Algorithm 1's greedy search with that lambda
# over only the R values the kernel reads (checked on the CPU, not yet timed).
R_PATH_LAMBDA = None


def gen_R_path(em, L, targets, f32, lam):
    """R^(0) for `targets` along the path r_path(targets, lam): deepest level
    first; FP64 with the prefactor in the base values, FP32 in the scaled form
    of gen_R_scaled (names PQs*, r2k*, F as there)."""
    path = r_path(targets, lam)
    X = ("PQsx", "PQsy", "PQsz") if f32 else ("PQx", "PQy", "PQz")
    sym = {}
    if not f32:
        depth = max(n for (n, t, u, v) in path)
        pw = [Sym(name="pref")]
        for n in range(1, depth + 1):
            pw.append(em.product([pw[-1], Sym(name="m2r")], f"pw{n}"))
    for node in sorted(path, key=lambda x: (-x[0], x[1:])):
        n, t, u, v = node
        ax = path[node]
        if ax is None:
            if f32:
                sym[node] = Sym(name=f"F[{n}]") if n % 2 == 0 else em.define(f"r{n}_000", f"-F[{n}]")
            else:
                sym[node] = em.product([pw[n], Sym(name=f"F[{n}]")], f"r{n}_000")
            continue
        k = (t, u, v)[ax]
        kids = _r_children(node, ax)
        terms = [(Sym(name=X[ax]), sym[kids[0]])]
        if len(kids) == 2:
            terms.append((Sym(name=f"r2k{k - 1}") if f32 else Sym(float(k - 1)), sym[kids[1]]))
        sym[node] = em.lincomb(terms, f"r{n}_{t}_{u}_{v}")
    return {(t, u, v): sym[(0, t, u, v)] for (_, t, u, v) in targets}


def r_path_flops(chosen):
    """Operations of a recursion path: one multiply per node plus one FMA
    where the node has a second child (the F_n base values are not counted)."""
    return sum(0 if ax is None else len(_r_children(n, ax)) for n, ax in chosen.items())


def path_report(lmax=2, lams=(0.0, 0.5, 1.0, 2.0), random_paths=0):
    """Per class: R recursion operations of the kernels as emitted (fixed
    order, per FP32 range kernel where the class has them), with the greedy
    path search at the best lam and, if random_paths > 0, the mean over that
    many random paths (seeded).  Rows (class, fixed, greedy[, random])."""
    import random
    rows = []
    for bra, ket in class_pairs(lmax):
        groups = crange_groups(bra, ket)
        nd = ncart(ket[1])
        sets = [None] if not groups else [[c * nd + d for c in range(c0, c1) for d in range(nd)] for c0, c1 in groups]
        fixed = sum(r_path_flops(r_path(r_targets(bra, ket, cds))) for cds in sets)
        greedy = sum(min(r_path_flops(r_path(r_targets(bra, ket, cds), lam)) for lam in lams) for cds in sets)
        row = (class_name(bra, ket), fixed, greedy)
        if random_paths:
            rnd = sum(r_path_flops(r_path(r_targets(bra, ket, cds), rng=random.Random(1000 * k + j)))
                      for k in range(random_paths) for j, cds in enumerate(sets)) / random_paths
            row += (rnd,)
        rows.append(row)
    return rows



def indent(s, n=2):
    return "\n".join(" " * n + l for l in s.split("\n"))


def class_pairs(lmax):
    pcs = [pc for pc in PAIR_CLASSES if pc[0] <= lmax]
    return [(pcs[i], pcs[j]) for i in range(len(pcs)) for j in range(i + 1)]


GRAD_LMAX = 3  # derivative kernels for every class (f classes in the chunked form)


def generate(outdir, lmax=LMAX, nfiles=None):
    os.makedirs(outdir, exist_ok=True)
    qs = class_pairs(lmax)
    gqs = class_pairs(min(lmax, GRAD_LMAX))
    if nfiles is None:
        nfiles = max(8, len(qs) // 3)
    # spread classes over translation units by generated code size (compile
    # time grows with it), largest first onto the lightest unit
    code_of = {}
    sized = []
    for bra, ket in qs:
        code_of[(bra, ket)] = gen_class_kernels(bra, ket)
        sized.append((len(code_of[(bra, ket)][0]), bra, ket))
    sized.sort(reverse=True)
    bins = [[] for _ in range(nfiles)]
    load = [0] * nfiles
    for w, bra, ket in sized:
        k = load.index(min(load))
        bins[k].append((bra, ket))
        load[k] += w + 2000
    header = '#include "eri_device.cuh"\n'
    stats_all = {}
    files = []
    for k, items in enumerate(bins):
        if not items:
            continue
        src = [header]
        kets = sorted({ket for _, ket in items})
        for ket in kets:
            src.append(cd_table(*ket))
        src += [comp_table(l) for l in range(lmax + 1)]
        for bra_ in sorted({bra for bra, ket in items if use_chunk(bra, ket)}):
            src.append(support_table(*bra_)[0])
        for bra, ket in items:
            code, st = code_of[(bra, ket)]
            src.append(code)
            stats_all[class_name(bra, ket)] = st
            name = class_name(bra, ket)
            if crange_groups(bra, ket):
                f32_launches = "\n".join(f"    eri_jk_{name}_f32_c{c0}<<<grid, block, 0, s>>>(a);"
                                          for c0, _ in crange_groups(bra, ket))
            else:
                f32_launches = f"    eri_jk_{name}_f32<<<grid, block, 0, s>>>(a);"
            rpath = ""
            if (bra, ket) in RPATH_CLASSES and crange_groups(bra, ket):
                rl = "\n".join(f"    eri_jk_{name}_f32r_c{c0}<<<grid, block, 0, s>>>(a);" for c0, _ in crange_groups(bra, ket))
                rpath = f"  else if (prec == 2) {{  // FP32, Algorithm 1's recursion order\n{rl}\n  }}\n"
            dfl_launch = (f"  else if (prec == 3) eri_jk_{name}_df<<<grid, block, 0, s>>>(a);  // double-float\n"
                          if has_df(bra, ket) else
                          f"  else if (prec == 3) eri_jk_{name}_f64<<<grid, block, 0, s>>>(a);  // no double-float form\n")
            src.append(f"""
int launch_jk_{name}(int prec, const gb::JKArgs& a, int grid, int block, cudaStream_t s) {{
  if (grid <= 0) return 0;
  if (prec == 0) eri_jk_{name}_f64<<<grid, block, 0, s>>>(a);
{dfl_launch}{rpath}  else {{
{f32_launches}
  }}
  return (int)cudaGetLastError();
}}
""")
            if bra == ket:
                nthr = ncart(bra[0]) if use_chunk(bra, ket) else 1
                src.append(f"""
int launch_schwarz_{bra[0]}{bra[1]}(const gb::SchwarzArgs& a, cudaStream_t s) {{
  if (a.count <= 0) return 0;
  const int bs = 128;
  eri_schwarz_{bra[0]}{bra[1]}<<<(unsigned)(((long long)a.count * {nthr} * gb::kSchwarzSplit + bs - 1) / bs), bs, 0, s>>>(a);
  return (int)cudaGetLastError();
}}
""")
        fn = os.path.join(outdir, f"md_classes_{k}.cu")
        _write_if_changed(fn, "".join(src))
        files.append(fn)
    # gradient kernels, spread over translation units by generated code size
    ngf = max(4, len(gqs) // 5)
    gbins = [[] for _ in range(ngf)]
    gload = [0] * ngf
    gcode = {q: gen_grad_kernel(*q, "f64") + gen_grad_kernel(*q, "f32") for q in gqs}
    for bra, ket in sorted(gqs, key=lambda x: -len(gcode[x])):
        k = gload.index(min(gload))
        gbins[k].append((bra, ket))
        gload[k] += len(gcode[(bra, ket)])
    for k, items in enumerate(gbins):
        if not items:
            continue
        src = [header] + [comp_table(l) for l in range(min(lmax, GRAD_LMAX) + 1)]
        for bra, ket in items:
            src.append(gcode[(bra, ket)])
        fn = os.path.join(outdir, f"md_grad_{k}.cu")
        _write_if_changed(fn, "".join(src))
        files.append(fn)
    # dispatch
    d = ['#include "eri_device.cuh"', "namespace gbgen {"]
    d.append("}")
    for bra, ket in qs:
        d.append(f"int launch_jk_{class_name(bra, ket)}(int prec, const gb::JKArgs& a, int grid, int block, cudaStream_t s);")
    pcs = [pc for pc in PAIR_CLASSES if pc[0] <= lmax]
    for pc in pcs:
        d.append(f"int launch_schwarz_{pc[0]}{pc[1]}(const gb::SchwarzArgs& a, cudaStream_t s);")
    for bra, ket in gqs:
        d.append(f"int launch_grad_{class_name(bra, ket)}(int prec, const gb::GradArgs& a, int grid, cudaStream_t s);")
    n = len(pcs)
    d.append("typedef int (*jk_launch_fn)(int, const gb::JKArgs&, int, int, cudaStream_t);")
    d.append("typedef int (*schwarz_launch_fn)(const gb::SchwarzArgs&, cudaStream_t);")
    tab = []
    for i in range(n):
        row = []
        for j in range(n):
            row.append(f"launch_jk_{class_name(pcs[i], pcs[j])}" if j <= i else "nullptr")
        tab.append("{" + ", ".join(row) + "}")
    d.append(f"extern \"C\" int gb_num_pair_classes() {{ return {n}; }}")
    d.append("typedef int (*grad_launch_fn)(int, const gb::GradArgs&, int, cudaStream_t);")
    gtab = []
    for i in range(n):
        row = [f"launch_grad_{class_name(pcs[i], pcs[j])}" if j <= i and (pcs[i], pcs[j]) in gqs else "nullptr"
               for j in range(n)]
        gtab.append("{" + ", ".join(row) + "}")
    d.append(f"static const grad_launch_fn k_grad_tab[{n}][{n}] = {{{', '.join(gtab)}}};")
    d.append("// -1: no derivative kernel for this class (shells above the gradient lmax)")
    d.append("// prec 0: FP64 derivative kernel, 1: FP32 (mixed gradient); grid-stride over the launch's items\n"
             "int gb_launch_grad(int bra_cls, int ket_cls, int prec, const gb::GradArgs& a, int grid, cudaStream_t s) {\n"
             "  return k_grad_tab[bra_cls][ket_cls] ? k_grad_tab[bra_cls][ket_cls](prec, a, grid, s) : -1;\n}")
    gthr = []
    for i in range(n):
        gthr.append("{" + ", ".join(str(grad_threads(pcs[i], pcs[j]) if j <= i else 1) for j in range(n)) + "}")
    d.append(f"static const int k_grad_threads_tab[{n}][{n}] = {{{', '.join(gthr)}}};")
    d.append("// threads per work item of a derivative kernel (f classes: one per ket component c)")
    d.append("int gb_grad_threads(int bra_cls, int ket_cls) { return k_grad_threads_tab[bra_cls][ket_cls]; }")
    d.append(f"int gb_grad_lmax() {{ return {min(lmax, GRAD_LMAX)}; }}")
    thr = []
    for prec in ("f64", "f32"):
        rows_ = []
        for i in range(n):
            row = []
            for j in range(n):
                t = 1
                if j <= i and use_chunk(pcs[i], pcs[j]):
                    t = ncart(pcs[j][0])
                row.append(str(t))
            rows_.append("{" + ", ".join(row) + "}")
        thr.append("{" + ", ".join(rows_) + "}")
    d.append(f"static const int k_threads_tab[2][{n}][{n}] = {{{', '.join(thr)}}};")
    spl = []
    for i in range(n):
        spl.append("{" + ", ".join(str(split_of(pcs[i], pcs[j]) if j <= i else 1) for j in range(n)) + "}")
    d.append(f"static const int k_split_tab[{n}][{n}] = {{{', '.join(spl)}}};")
    d.append("// most work items one shell quartet of a class is split into (over its bra primitive pairs)")
    d.append("int gb_class_split(int bra_cls, int ket_cls) { return k_split_tab[bra_cls][ket_cls]; }")
    d.append("// threads per shell quartet of a class kernel (prec 0: FP64, 1: FP32)")
    d.append("int gb_class_threads(int bra_cls, int ket_cls, int prec) { return k_threads_tab[prec][bra_cls][ket_cls]; }")
    d.append(f"static const jk_launch_fn k_jk_tab[{n}][{n}] = {{{', '.join(tab)}}};")
    d.append(f"static const schwarz_launch_fn k_sw_tab[{n}] = {{{', '.join(f'launch_schwarz_{pc[0]}{pc[1]}' for pc in pcs)}}};")
    d.append("""
int gb_launch_jk(int bra_cls, int ket_cls, int prec, const gb::JKArgs& a, int grid, int block, cudaStream_t s) {
  return k_jk_tab[bra_cls][ket_cls](prec, a, grid, block, s);
}
int gb_launch_schwarz(int cls, const gb::SchwarzArgs& a, cudaStream_t s) {
  return k_sw_tab[cls](a, s);
}
""")
    # flop table for roofline accounting
    rows = []
    for bra, ket in qs:
        st = stats_all[class_name(bra, ket)]
        rows.append(f"{{{st['flops_per_primq']}, {st['flops_per_brap']}}}")
    d.append(f"static const int k_class_flops[{len(qs)}][2] = {{{', '.join(rows)}}};")
    d.append("""
// Algorithmic FP operations of the generated code: per primitive quartet and per
// (shell quartet x bra primitive pair); -1 if the class is not compiled.
int gb_class_flops(int bra_cls, int ket_cls, int* per_primq, int* per_brap) {
  if (bra_cls < 0 || ket_cls < 0 || ket_cls > bra_cls || bra_cls >= gb_num_pair_classes()) return -1;
  const int idx = bra_cls * (bra_cls + 1) / 2 + ket_cls;
  *per_primq = k_class_flops[idx][0];
  *per_brap = k_class_flops[idx][1];
  return 0;
}
""")
    fn = os.path.join(outdir, "md_dispatch.cu")
    _write_if_changed(fn, "\n".join(d) + "\n")
    files.append(fn)
    return files, stats_all


def _write_if_changed(fn, text):
    if os.path.exists(fn) and open(fn).read() == text:
        return
    with open(fn, "w") as f:
        f.write(text)


if __name__ == "__main__":
    out = sys.argv[1] if len(sys.argv) > 1 else "_gen"
    lmax = int(sys.argv[2]) if len(sys.argv) > 2 else 2
    files, stats = generate(out, lmax)
    for k, v in stats.items():
        print(k, "flat" if v["flat"] else "loop", "flops/primq", v["flops_per_primq"], "flops/brap", v["flops_per_brap"])
