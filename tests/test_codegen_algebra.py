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
        if ch in "([":
            depth += 1
        elif ch in ")]":
            depth -= 1
        if ch == sep and depth == 0:
            out.append(cur)
            cur = ""
        else:
            cur += ch
    if cur.strip():
        out.append(cur)
    return out


class _Ptr:
    """`const T* q = base + off`: q[k] reads base[off + k]."""

    def __init__(self, base, off):
        self.base, self.off = base, off

    def __getitem__(self, k):
        return self.base[self.off + k]


_FOR = re.compile(r"for \(int (\w+) = (.+?); \1 (<=|<|>=) (.+?); (\+\+\1|--\1|\1 \+= \w+)\)\s*(\{?)\s*(.*)$")


def _expr(e):
    e = re.sub(r"\b(\d+\.\d*|\d+)f\b", r"\1", e)
    e = re.sub(r"\b__fdividef\(", "_div(", e)
    e = re.sub(r"\brsqrtf?\(", "_rsqrt(", e)
    e = re.sub(r"\bfmaf?\(", "_fma(", e)
    e = re.sub(r"\((?:double|float|int)\)\(", "float(", e)
    m = re.search(r"\(([^()]+)\) \? (.+?) : (.+)$", e)
    if m:
        e = e[:m.start()] + f"({m.group(2)} if ({m.group(1)}) else {m.group(3)})"
    return e


def _stmt(st):
    """One C statement (no control flow) -> Python lines."""
    st = st.strip().rstrip(";").strip()
    if not st:
        return []
    m = re.match(r"^gb::boys_(?:f64|mixed)<(\d+)>\(T, F.*\)$", st)
    if m:
        return [f"F = _boys({m.group(1)}, T)"]
    m = re.match(r"^(?:const )?(?:int|float|double)[24]?\* (\w+) = (\w+) \+ (.+)$", st)
    if m:
        return [f"{m.group(1)} = _Ptr({m.group(2)}, {_expr(m.group(3))})"]
    m = re.match(r"^(?:float|double|int) (\w+)\[(\d+)\]$", st)
    if m:
        return [f"{m.group(1)} = [0.0] * {m.group(2)}"]
    m = re.match(r"^(?:float|double) (\w+)$", st)
    if m:
        return [f"{m.group(1)} = 0.0"]
    st = re.sub(r"^(?:const )?(?:float|double|int)[24]? ", "", st)
    return [_expr(p.strip()) for p in re.split(r",\s*(?=[A-Za-z_]\w*\s*=[^=])", st)]


def _if_chain(line):
    """`[else ][if (c) ]{ s1; if (c2) s2; }` -> (keyword header, body lines)."""
    m = re.match(r"^(else )?(?:if \((.+?)\) )?\{ (.*) \}$", line)
    kw = ("elif" if m.group(1) else "if") if m.group(2) else "else"
    head = f"{kw} {_expr(m.group(2))}:" if m.group(2) else "else:"
    body = []
    for st in _split_top(m.group(3), ";"):
        st = st.strip()
        mm = re.match(r"^if \((.+?)\) (.+)$", st)
        if mm:
            body.append(f"if {_expr(mm.group(1))}: " + "; ".join(_stmt(mm.group(2))))
        else:
            body += _stmt(st)
    return head, body


def to_python(body):
    """Translate a generated kernel body (C) into Python source.  The bodies
    run here with every primitive quartet (primitive mode 0): the primitive
    split's block (mg.PRIM_CUT) is reduced to its mode-0 ket range; the split
    itself is exercised by tests/test_kernel_emulation.py."""
    body = body.replace(mg.PRIM_CUT, "int jq0 = 0, jq1 = ik.z;")
    out, ind, stack, pending = [], 0, [], 0

    def emit(s, extra=0):
        out.append(" " * (ind + extra) + s)

    for raw in body.split("\n"):
        line = raw.split("//")[0].strip()
        if not line or line.startswith("#pragma"):
            continue
        m = _FOR.match(line)
        if m:
            var, a, op, b, step, brace, rest = m.groups()
            a, b = _expr(a), _expr(b)
            if step.startswith("--"):
                rng = f"range({a}, ({b}) - 1, -1)"
            elif "+=" in step:
                rng = f"range({a}, {b}, {step.split('+=')[1].strip()})"
            else:
                rng = f"range({a}, {b}{' + 1' if op == '<=' else ''})"
            emit(f"for {var} in {rng}:")
            ind += 4
            if brace:
                stack.append(1 + pending)
                pending = 0
            elif rest:
                for s_ in _stmt(rest):
                    emit(s_)
                ind -= 4
            else:
                pending += 1
            continue
        if re.match(r"^(else )?(if \(.+?\) )?\{ .* \}$", line):
            head, lines = _if_chain(line)
            emit(head)
            for s_ in lines:
                emit(s_, 4)
            continue
        if re.fullmatch(r"\}+", line):
            for _ in line:
                ind -= 4 * stack.pop()
            continue
        if line.startswith("}"):
            ind -= 4 * stack.pop()
            continue
        for st in _split_top(line, ";"):
            for s_ in _stmt(st):
                emit(s_)
    assert ind == 0 and not stack, (ind, stack)
    return "\n".join(out)


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


def _run(body, bra, ket, shells, ci=0):
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
    ns.update(ACx=AC[0], ACy=AC[1], ACz=AC[2], boys=None, boysf=None, tsmall=0.0, ci=ci)
    for l in range(4):
        ns[f"c_comp_{l}"] = [x for c in mg.comps(l) for x in c]
    lc, ld = ket
    ns[f"c_cd_tab_{lc}{ld}"] = [x for c in mg.comps(lc) for d in mg.comps(ld) for x in c + d]
    txt = mg.support_table(*bra)[0]
    ns[f"c_bsup_{bra[0]}{bra[1]}"] = [int(v) for v in txt[txt.index("{") + 1:txt.index("}")].split(",")]
    ns["_Ptr"] = _Ptr
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


LOOP = [(b, k) for b, k in mg.class_pairs(2) if not mg.use_flat(b, k, "f64")]


@pytest.mark.parametrize("bra,ket", LOOP, ids=[mg.class_name(b, k) for b, k in LOOP])
def test_loop_body_matches_oracle(bra, ket):
    """FP64 looped form of the large l <= 2 classes (R cube, runtime loops)."""
    rng = np.random.default_rng(sum(bra) * 13 + sum(ket) * 3)
    sh = _shells(rng, [bra[0], bra[1], ket[0], ket[1]], 2)
    body, _ = mg.gen_quartet_body(bra, ket, "double", False)
    got = _run(body, bra, ket, sh)
    ref = oracle.eri_quartet(sh).reshape(-1)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), np.abs(got - ref).max()


def _ordered(x, y):
    ix, iy = mg.PAIR_CLASSES.index(x), mg.PAIR_CLASSES.index(y)
    return (x, y) if ix >= iy else (y, x)


CHUNK = [c for c in (_ordered(*xy) for xy in [((3, 0), (1, 1)), ((3, 1), (1, 1)), ((3, 0), (2, 2)), ((3, 2), (2, 1)),
                                              ((3, 3), (1, 0)), ((3, 3), (3, 3)), ((3, 1), (3, 0))])
         if mg.use_chunk(*c)]


@pytest.mark.parametrize("bra,ket", CHUNK, ids=[mg.class_name(b, k) for b, k in CHUNK])
@pytest.mark.parametrize("real", ["double", "float"])
def test_chunk_body_matches_oracle(bra, ket, real):
    """Classes with an f shell: one thread per ket component c (rolled R
    recursion, support tables); the threads of a quartet assemble the block."""
    rng = np.random.default_rng(sum(bra) * 7 + sum(ket) + (real == "float"))
    sh = _shells(rng, [bra[0], bra[1], ket[0], ket[1]], 1)
    ref = oracle.eri_quartet(sh)
    na, nb, nc, nd = ref.shape
    body, _ = mg.gen_quartet_body_chunk(bra, ket, real)
    for ci in range(nc):
        got = _run(body, bra, ket, sh, ci).reshape(na * nb, nd)
        want = ref[:, :, ci, :].reshape(na * nb, nd)
        assert np.abs(got - want).max() <= 1e-11 * max(1.0, np.abs(ref).max()), (ci, np.abs(got - want).max())


@pytest.mark.parametrize("lam", [None, 0.0, 1.0, "random"])
def test_r_path_search_is_a_valid_recursion(lam):
    """The recursion paths (fixed order, the Algorithm-1 greedy search and a
    random order, the paper's baseline):
    every target is reached, every chosen node's children are on the path,
    and the recursion evaluated along the path reproduces the Hermite R
    values of the fixed-order code (random rho, P-Q, F_n)."""
    rng = np.random.default_rng(5)
    for bra, ket in [((1, 1), (1, 0)), ((2, 1), (2, 1)), ((2, 2), (1, 1))]:
        T = mg.r_targets(bra, ket)
        if lam == "random":
            import random
            path = mg.r_path(T, rng=random.Random(17))
        else:
            path = mg.r_path(T, lam)
        assert T <= set(path)
        for node, ax in path.items():
            if ax is not None:
                assert all(c in path for c in mg._r_children(node, ax))
        L = sum(bra) + sum(ket)
        X = rng.uniform(-1, 1, 3)
        F = rng.uniform(0.1, 1, L + 1)
        memo = {}

        def R(node):  # evaluate along the chosen axes
            if node not in memo:
                n, *k = node
                ax = path[node]
                if ax is None:
                    memo[node] = F[n]
                else:
                    kids = mg._r_children(node, ax)
                    val = X[ax] * R(kids[0])
                    if len(kids) == 2:
                        val += (k[ax] - 1) * R(kids[1])
                    memo[node] = val
            return memo[node]
        ref_path = mg.r_path(T, None)
        memo_ref = {}

        def Rref(node):
            if node not in memo_ref:
                n, *k = node
                ax = ref_path[node]
                memo_ref[node] = F[n] if ax is None else (
                    X[ax] * Rref(mg._r_children(node, ax)[0]) +
                    ((k[ax] - 1) * Rref(mg._r_children(node, ax)[1]) if k[ax] >= 2 else 0.0))
            return memo_ref[node]
        for t in T:
            assert abs(R(t) - Rref(t)) <= 1e-12 * max(1.0, abs(Rref(t)))


def test_path_search_never_costs_more():
    for name, fixed, greedy in mg.path_report():
        assert greedy <= fixed, name


def test_path_search_against_random_paths():
    """Algorithm 1 is compared with random recursion orders in the paper;
    over the R values the l <= 2 kernels read, the searched paths need
    about a fifth fewer operations than random ones (mean of 5 seeds).  The
    greedy search is not optimal class by class: for a few small classes a
    random order is as cheap or slightly cheaper on average."""
    rows = mg.path_report(random_paths=5)
    greedy = sum(r[2] for r in rows)
    rnd = sum(r[3] for r in rows)
    assert 1.15 < rnd / greedy < 1.35


@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_path_searched_r_emission(monkeypatch, lam):
    """With the Algorithm-1 recursion order switched on, the straight-line
    FP64/FP32 bodies and the FP32 range bodies still equal the oracle."""
    monkeypatch.setattr(mg, "R_PATH_LAMBDA", lam)
    rng = np.random.default_rng(int(lam * 10) + 3)
    for bra, ket in [((1, 1), (1, 0)), ((2, 1), (1, 1)), ((2, 0), (2, 0))]:
        sh = _shells(rng, [bra[0], bra[1], ket[0], ket[1]], 2)
        ref = oracle.eri_quartet(sh).reshape(-1)
        for real in ("double", "float"):
            body, _ = mg.gen_quartet_body(bra, ket, real, True)
            got = _run(body, bra, ket, sh)
            assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (bra, ket, real)
    bra, ket = (2, 1), (2, 1)
    sh = _shells(rng, [2, 1, 2, 1], 1)
    ref = oracle.eri_quartet(sh)
    na, nb, nc, nd = ref.shape
    for c0, c1 in mg.crange_groups(bra, ket):
        cds = [c * nd + d for c in range(c0, c1) for d in range(nd)]
        body, _ = mg.gen_quartet_body(bra, ket, "float", True, cds)
        got = _run(body, bra, ket, sh).reshape(na * nb, len(cds))
        want = ref.reshape(na * nb, nc * nd)[:, cds]
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())


def test_item_split_divides_the_bra_primitive_pairs():
    """Work items per quartet: a divisor of K_ab (every item of a quartet runs
    the same number of bra primitive pairs), the largest one not above the
    class's split P; K_ab <= P keeps one item per bra primitive pair."""
    for P in (1, 4, 8):
        for z in range(1, 65):
            d = mg.item_split(P, z)
            assert 1 <= d <= min(P, z) and z % d == 0
            assert not any(z % e == 0 for e in range(d + 1, min(P, z) + 1))
            if z <= P:
                assert d == z
    assert [mg.item_split(8, z) for z in (9, 10, 12, 15, 18, 25, 36)] == [3, 5, 6, 5, 6, 5, 6]
