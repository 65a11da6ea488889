"""CPU emulation of the generated ERI kernels (test infrastructure only).

The kernel text the generator emits for the GPU library is compiled as plain
C++ with host stand-ins for the few CUDA names it uses (tests/emu/cuda_runtime.h)
and run one thread at a time: the grid-stride loops of the J/K kernels then
visit every work item in order, the gradient kernels are called once per
quartet.  Pair data, quartet rows, work-item prefixes and the Boys table are
built here in Python as the library's runtime builds them; J/K/gradient come
out exactly as the kernels compute them (the FP32 kernels in real FP32), so the
tests can hold every generated kernel against the oracle without a GPU."""
from __future__ import annotations

import concurrent.futures as cf
import ctypes as C
import hashlib
import math
import os
import re
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, os.path.join(ROOT, "paper_2412_13203_gb300", "codegen"))
import md_codegen as mg  # noqa: E402

BUILD = os.path.join(HERE, "_emu_build")
KBOYS_ROWS, KBOYS_TAYLOR, KBOYS_NGRID, KLMAX_BOYS, KBOYS_LO_SLOT = 15, 8, 1281, 13, 5


def _sources(lmax, only=None, ntu=8):
    """Translation units: `ntu` holding the kernels (spread by size, compiled
    in parallel) and one holding the dispatch entry points."""
    qs = [q for q in mg.class_pairs(lmax) if only is None or q in only]
    gqs = [q for q in mg.class_pairs(min(lmax, mg.GRAD_LMAX)) if q in qs]
    head = ['#include "eri_device.cuh"']
    head += [mg.comp_table(l) for l in range(lmax + 1)]
    for ket in sorted({k for _, k in qs}):
        head.append(mg.cd_table(*ket))
    for bra in sorted({b for b, k in qs if mg.use_chunk(b, k)}):
        head.append(mg.support_table(*bra)[0])
    pcs = [pc for pc in mg.PAIR_CLASSES if pc[0] <= lmax]
    jk_cases, grad_cases, sw_cases, decls = [], [], [], []
    tus = [list(head) for _ in range(ntu)]
    load_ = [0] * ntu
    for bra, ket in qs:
        code = mg.gen_class_kernels(bra, ket)[0]
        if (bra, ket) in gqs:
            g = mg.gen_grad_kernel(bra, ket, "f64") + mg.gen_grad_kernel(bra, ket, "f32")
            code += g[:g.index("\nint launch_grad_")]
        k = load_.index(min(load_))
        tus[k].append(code)
        load_[k] += len(code)
        decls += ["void " + m + ";" for m in re.findall(r"void (?:__launch_bounds__\([^)]*\) )?(eri_\w+\(const gb::\w+ \w+\))", code)]
        name = mg.class_name(bra, ket)
        key = pcs.index(bra) * 16 + pcs.index(ket)
        if mg.crange_groups(bra, ket):
            f32 = " ".join(f"eri_jk_{name}_f32_c{c0}(a);" for c0, _ in mg.crange_groups(bra, ket))
        else:
            f32 = f"eri_jk_{name}_f32(a);"
        dfc = f"else if (prec == 3) eri_jk_{name}_{'df' if mg.has_df(bra, ket) else 'f64'}(a); "
        if (bra, ket) in mg.RPATH_CLASSES and mg.crange_groups(bra, ket):
            # prec 2: the FP32 range kernels emitted with Algorithm 1's recursion order
            f32r = " ".join(f"eri_jk_{name}_f32r_c{c0}(a);" for c0, _ in mg.crange_groups(bra, ket))
            jk_cases.append(f"    case {key}: if (prec == 0) eri_jk_{name}_f64(a); else if (prec == 2) {{ {f32r} }} "
                            f"{dfc}else {{ {f32} }} return 0;")
        else:
            jk_cases.append(f"    case {key}: if (prec == 0) eri_jk_{name}_f64(a); {dfc}else {{ {f32} }} return 0;")
        if bra == ket:
            nthr = mg.ncart(bra[0]) if mg.use_chunk(bra, ket) else 1
            nab = mg.ncart(bra[0]) * mg.ncart(bra[1])
            sw_cases.append(f"    case {pcs.index(bra)}: nab = {nab}; diag.assign((size_t)count * gb::kSchwarzSplit * nab, 0.0); "
                            f"sa.diag = diag.data(); for (blockIdx.x = 0; "
                            f"blockIdx.x < (unsigned)(count * {nthr} * gb::kSchwarzSplit); "
                            f"++blockIdx.x) eri_schwarz_{bra[0]}{bra[1]}(sa); break;")
        if (bra, ket) in gqs:
            gthr = mg.grad_threads(bra, ket)  # threads per work item (chunked f classes: ket components)
            # grid-stride kernels: one call (one block of one thread) visits every item
            grad_cases.append(f"    case {key}: if (prec == 0) eri_grad_{name}_f64(g); else eri_grad_{name}_f32(g); return 0;")
    src = ['#include "eri_device.cuh"', "#include <vector>", "#include <deque>", "emu_dim3 blockIdx, threadIdx, blockDim, gridDim;"] + decls
    src.append("""
static std::deque<std::vector<float4>> g_ahl;  // split centres of every view built (kept alive)
// double-float data of the problem being emulated (emu_set_df), read by the next views and launches
static const float4* g_ppd = nullptr;
static const float2* g_boysd = nullptr;
static const gb::dfl* g_ddf = nullptr;
extern "C" void emu_set_df(const float4* ppd, const float2* boysd, const void* ddf) {
    g_ppd = ppd; g_boysd = boysd; g_ddf = (const gb::dfl*)ddf;
}
// primitive split (emu_set_prim): primitive Schwarz factors of the next views,
// per-list-entry cuts and the primitive mode of the next launches
static const float* g_pq = nullptr;
static const float* g_kthr = nullptr;
static int g_pmode = 0;
extern "C" void emu_set_prim(const float* pq, const float* kthr, int pmode) {
    g_pq = pq; g_kthr = kthr; g_pmode = pmode;
}
// explicit ket lists of the next emu_grad call (nullptr: contiguous kets)
static const long long* g_gkofs = nullptr;
static const int* g_gklist = nullptr;
extern "C" void emu_set_grad_lists(const long long* kofs, const int* klist) { g_gkofs = kofs; g_gklist = klist; }
static gb::PairsView pv(int npair, const int4* info, const double4* A, const double4* B, const double4* pp,
                        const double2* pp2, const float4* ppf, const float4* ppf2, const double* alpha) {
    gb::PairsView v;
    std::memset(&v, 0, sizeof(v));
    v.npair = npair; v.info = info; v.A = A; v.B = B; v.pp = pp; v.pp2 = pp2; v.ppf = ppf; v.ppf2 = ppf2;
    v.alpha = alpha;
    // the runtime's k_centres_hl: centre of a as hi = (float)A and lo = (float)(A - hi)
    g_ahl.emplace_back(2 * (size_t)npair);
    for (int i = 0; i < npair; ++i) {
        const float hx = (float)A[i].x, hy = (float)A[i].y, hz = (float)A[i].z;
        g_ahl.back()[2 * i] = float4{hx, hy, hz, 0.f};
        g_ahl.back()[2 * i + 1] = float4{(float)(A[i].x - hx), (float)(A[i].y - hy), (float)(A[i].z - hz), 0.f};
    }
    v.Ahl = g_ahl.back().data();
    v.ppd = g_ppd;
    v.pq = g_pq;
    return v;
}
extern "C" int emu_jk(int X, int Y, int prec, int npair, const int4* info, const double4* A, const double4* B,
                      const double4* pp, const double2* pp2, const float4* ppf, const float4* ppf2,
                      const double* alpha, int nrows, const long long* start, const int* bra, const int* ket0,
                      const long long* kofs, const int* klist,
                      const double* boys, const float* boysf, float tsmall, const double* D, const float* Df,
                      double* J, double* K, int nbf) {
    gb::JKArgs a;
    std::memset(&a, 0, sizeof(a));
    a.pairs = pv(npair, info, A, B, pp, pp2, ppf, ppf2, alpha);
    a.rows.nrows = nrows; a.rows.start = start; a.rows.bra = bra; a.rows.ket0 = ket0;
    a.rows.kofs = kofs; a.rows.klist = klist;
    a.rows.kthr = klist ? g_kthr : nullptr;
    a.pmode = klist && g_kthr ? g_pmode : 0;
    a.boys = boys; a.boysf = boysf; a.tsmall = tsmall; a.D = D; a.Df = Df; a.J = J; a.K = K; a.nbf = nbf;
    a.boysd = g_boysd; a.Ddf = g_ddf;
    blockIdx = {0, 0, 0}; threadIdx = {0, 0, 0}; blockDim = {1, 1, 1}; gridDim = {1, 1, 1};
    switch (X * 16 + Y) {
""" + "\n".join(jk_cases) + """
    }
    return -1;
}
extern "C" int emu_jk_batched(int X, int Y, int prec, int nmol, const int* npair, void* const* info, void* const* A,
                              void* const* B, void* const* pp, void* const* pp2, void* const* ppf, void* const* ppf2,
                              void* const* D, void* const* Df, void* const* J, void* const* K, const int* nbf,
                              int nrows, const long long* start, const int* bra, const int* ket0, const int* rowmol,
                              const double* boys, const float* boysf, float tsmall) {
    std::vector<gb::BatchMol> bm(nmol);
    for (int m = 0; m < nmol; ++m) {
        std::memset(&bm[m], 0, sizeof(gb::BatchMol));
        bm[m].pairs = pv(npair[m], (const int4*)info[m], (const double4*)A[m], (const double4*)B[m],
                         (const double4*)pp[m], (const double2*)pp2[m], (const float4*)ppf[m], (const float4*)ppf2[m],
                         nullptr);
        bm[m].D = (const double*)D[m]; bm[m].Df = (float*)Df[m];
        bm[m].J = (double*)J[m]; bm[m].K = (double*)K[m]; bm[m].nbf = nbf[m];
    }
    gb::JKArgs a;
    std::memset(&a, 0, sizeof(a));
    a.rows.nrows = nrows; a.rows.start = start; a.rows.bra = bra; a.rows.ket0 = ket0;
    a.boys = boys; a.boysf = boysf; a.tsmall = tsmall; a.mols = bm.data(); a.row_mol = rowmol;
    blockIdx = {0, 0, 0}; threadIdx = {0, 0, 0}; blockDim = {1, 1, 1}; gridDim = {1, 1, 1};
    switch (X * 16 + Y) {
""" + "\n".join(jk_cases) + """
    }
    return -1;
}
extern "C" int emu_schwarz(int X, int npair, const int4* info, const double4* A, const double4* B,
                           const double4* pp, const double2* pp2, int first, int count, const double* boys,
                           double* Q) {
    gb::SchwarzArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.pairs = pv(npair, info, A, B, pp, pp2, nullptr, nullptr, nullptr);
    sa.first = first; sa.count = count; sa.boys = boys; sa.Q = Q;
    threadIdx = {0, 0, 0}; blockDim = {1, 1, 1}; gridDim = {1, 1, 1};
    std::vector<double> diag;
    int nab = 0;
    switch (X) {
""" + "\n".join(sw_cases) + """
    default: return -1;
    }
    // the runtime's k_schwarz_finish: parts added in order, sqrt of the largest |diagonal|
    for (int i = 0; i < count; ++i) {
        double m = 0.0;
        for (int d = 0; d < nab; ++d) {
            double v = 0.0;
            for (int p = 0; p < gb::kSchwarzSplit; ++p) v += diag[((size_t)i * gb::kSchwarzSplit + p) * nab + d];
            m = std::fmax(m, std::fabs(v));
        }
        Q[i] = std::sqrt(m);
    }
    return 0;
}
extern "C" int emu_grad(int X, int Y, int prec, int npair, const int4* info, const double4* A, const double4* B,
                        const double4* pp, const double2* pp2, const float4* ppf, const float4* ppf2,
                        const double* alpha, int nrows, const long long* start, const int* bra, const int* ket0,
                        const double* boys, const float* boysf, float tsmall, const double* D, int nbf,
                        const int2* atoms, double* grad) {
    gb::GradArgs g;
    std::memset(&g, 0, sizeof(g));
    g.pairs = pv(npair, info, A, B, pp, pp2, ppf, ppf2, alpha);
    g.rows.nrows = nrows; g.rows.start = start; g.rows.bra = bra; g.rows.ket0 = ket0;
    g.rows.kofs = g_gkofs; g.rows.klist = g_gklist;
    g.rows.kthr = g_gklist ? g_kthr : nullptr;
    g.pmode = g_gklist && g_kthr ? g_pmode : 0;
    g.boys = boys; g.boysf = boysf; g.tsmall = tsmall; g.D = D; g.nbf = nbf; g.atoms = atoms; g.grad = grad;
    blockIdx = {0, 0, 0}; threadIdx = {0, 0, 0}; blockDim = {1, 1, 1}; gridDim = {1, 1, 1};
    switch (X * 16 + Y) {
""" + "\n".join(grad_cases) + """
    }
    return -1;
}
""")
    return ["\n".join(t) for t in tus if len(t) > len(head)], "\n".join(src)


_LIBS = {}


def load(lmax=2, only=None):
    """Compile (cached by source hash) and load the emulation library of the
    class pairs `only` (all classes up to lmax if None)."""
    key = (lmax, None if only is None else tuple(sorted(only)))
    if key in _LIBS:
        return _LIBS[key]
    tus, disp = _sources(lmax, only)
    hdrs = [os.path.join(ROOT, "paper_2412_13203_gb300", "csrc", "eri_device.cuh"),
            os.path.join(HERE, "emu", "cuda_runtime.h")]
    h = hashlib.sha1("".join(tus + [disp]).encode())
    for p in hdrs:
        h.update(open(p, "rb").read())
    os.makedirs(BUILD, exist_ok=True)
    stem = os.path.join(BUILD, f"emu_{lmax}_{h.hexdigest()[:12]}")
    lib = stem + ".so"
    if not os.path.exists(lib):
        flags = ["-std=c++17", "-O1", "-fPIC", "-w", "-I", os.path.join(HERE, "emu"),
                 "-I", os.path.join(ROOT, "paper_2412_13203_gb300", "csrc"), "-I", os.path.join(ROOT, "include")]

        def compile_one(i_src):
            i, text = i_src
            cpp, obj = f"{stem}_{i}.cpp", f"{stem}_{i}.o"
            with open(cpp, "w") as f:
                f.write(text)
            subprocess.run(["g++", "-c", cpp, "-o", obj] + flags, check=True)
            return obj

        with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
            objs = list(ex.map(compile_one, enumerate(tus + [disp])))
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-shared", "-o", tmp] + objs, check=True)
        os.replace(tmp, lib)
    _LIBS[key] = C.CDLL(lib)
    return _LIBS[key]


def boys_tables(oracle):
    """The Boys Taylor table in the library's layout: F_{m+j}(T_k)/j! for
    T_k = k/16, m = 0..13, and exp(-T_k)/j! in the last row (values from the
    oracle's Boys function); the FP32 copy holds the low part of each row's
    leading term in the slot the FP32 evaluation does not use."""
    tab = np.zeros((KBOYS_NGRID, KBOYS_ROWS, KBOYS_TAYLOR))
    fact = np.array([math.factorial(j) for j in range(KBOYS_TAYLOR)], dtype=float)
    for k in range(KBOYS_NGRID):
        T = k / 16.0
        F = oracle.boys(KLMAX_BOYS + KBOYS_TAYLOR, T)
        for m in range(KLMAX_BOYS + 1):
            tab[k, m] = F[m:m + KBOYS_TAYLOR] / fact
        tab[k, KLMAX_BOYS + 1] = math.exp(-T) / fact
    tabf = tab.astype(np.float32)
    # slot 5 of every FP32 row: the low part of its leading term
    tabf[:, :, KBOYS_LO_SLOT] = (tab[:, :, 0] - tabf[:, :, 0].astype(np.float64)).astype(np.float32)
    return tab.ravel(), tabf.ravel()


class Problem:
    """Pairs, rows and matrices of one molecule, laid out as the library's
    runtime lays them out (pairs canonicalised l_a >= l_b, grouped by class;
    for bra class = ket class only kets up to the bra)."""

    def __init__(self, mol, D, oracle, lmax=2, own_classes=False, q_order=False, prim_sort=False):
        self.mol, self.lmax = mol, lmax
        c = oracle.normalize(mol)
        l, K, off, atom = mol.shell_l, mol.shell_nprim, mol.shell_prim_offset, mol.shell_atom
        S = len(l)
        bf = np.concatenate([[0], np.cumsum([(x + 1) * (x + 2) // 2 for x in l])])[:-1]
        self.pcs = [pc for pc in mg.PAIR_CLASSES if pc[0] <= lmax]
        pairs = []
        for i in range(S):
            for j in range(i + 1):
                a, b = (j, i) if l[j] > l[i] else (i, j)
                pairs.append((self.pcs.index((int(l[a]), int(l[b]))), a, b))
        Q = oracle.schwarz(mol)
        if q_order:  # as the runtime: inside a class by Schwarz factor, largest first
            pairs.sort(key=lambda x: (x[0], -Q[x[1], x[2]], x[1], x[2]))
        else:
            pairs.sort()
        info, A, B, pp, pp2, ppf, ppf2, alpha, atoms, ppd, pq = [], [], [], [], [], [], [], [], [], [], []
        s2 = math.sqrt(2 * math.pi ** 2.5)
        for cls, a, b in pairs:
            Ra, Rb = mol.xyz[atom[a]], mol.xyz[atom[b]]
            AB = Ra - Rb
            info.append((bf[a], bf[b], K[a] * K[b], len(pp)))
            A.append((*Ra, Q[a, b]))
            B.append((*Rb, 0.0))
            atoms.append((atom[a], atom[b]))
            order = [(u, v) for u in range(K[a]) for v in range(K[b])]
            if prim_sort:
                # as the pair build: each primitive pair's Schwarz factor (the oracle's
                # diagonal (pp|pp) of the two one-primitive shells, normalised
                # contraction coefficients included), largest first
                qv = []
                for u, v in order:
                    sa = (Ra, int(l[a]), [mol.exps[off[a] + u]], [c[off[a] + u]])
                    sb = (Rb, int(l[b]), [mol.exps[off[b] + v]], [c[off[b] + v]])
                    e = oracle.eri_quartet([sa, sb, sa, sb])
                    n2 = e.shape[0] * e.shape[1]
                    qv.append(math.sqrt(float(np.abs(np.diag(e.reshape(n2, n2))).max())))
                rank = sorted(range(len(order)), key=lambda k: (-qv[k], k))
                order = [order[k] for k in rank]
                pq += [qv[k] for k in rank]
            for u, v in order:
                al, be = mol.exps[off[a] + u], mol.exps[off[b] + v]
                p = al + be
                kap = s2 * math.exp(-al * be / p * (AB @ AB)) * c[off[a] + u] * c[off[b] + v] / p
                pp.append((*((al * Ra + be * Rb) / p), p))
                pp2.append((kap, 0.5 / p))
                ppf.append((*(-be / p * AB), p))
                ppf2.append((*(al / p * AB), kap))
                ppd.append((*(-be / p * AB), *(al / p * AB), p, kap, 0.5 / p))
                alpha.append(al)
        self.cls = np.array([x[0] for x in pairs])
        self.pair_shells = [(a, b) for _, a, b in pairs]
        present = sorted(set(self.cls.tolist()))
        # compile every class when the molecule spans all l <= 2 classes (shared,
        # cached library), else only the classes this molecule has
        self.only = None if (lmax == 2 and not own_classes) else \
            {(self.pcs[x], self.pcs[y]) for x in present for y in present if y <= x}
        f = lambda x, t: np.ascontiguousarray(np.array(x, dtype=t))
        self.info, self.atoms = f(info, np.int32), f(atoms, np.int32)
        self.A, self.B, self.pp, self.pp2 = f(A, np.float64), f(B, np.float64), f(pp, np.float64), f(pp2, np.float64)
        self.ppf, self.ppf2, self.alpha = f(ppf, np.float32), f(ppf2, np.float32), f(alpha, np.float64)
        self.pq = f(pq, np.float32) if prim_sort else None
        self.D = np.ascontiguousarray(D, dtype=np.float64)
        self.Df = self.D.astype(np.float32)
        # double-float data as the runtime lays them out: 5 float4 per primitive pair
        # ((P-A)x,(P-A)y | (P-A)z,(P-B)x | (P-B)y,(P-B)z | p,kappa | 1/2p,-), each value hi, lo
        v = np.array(ppd, dtype=np.float64).reshape(-1, 9)
        hl = np.zeros((v.shape[0], 20), dtype=np.float32)
        hl[:, 0:18:2] = v.astype(np.float32)
        hl[:, 1:18:2] = (v - v.astype(np.float32).astype(np.float64)).astype(np.float32)
        self.ppd = np.ascontiguousarray(hl)
        self.Ddf = np.ascontiguousarray(np.stack([self.Df, (self.D - self.Df.astype(np.float64)).astype(np.float32)],
                                                 axis=-1))
        self.nbf = D.shape[0]
        self.boys, self.boysf = boys_tables(oracle)
        bh = self.boys.astype(np.float32)
        self.boysd = np.ascontiguousarray(np.stack([bh, (self.boys - bh.astype(np.float64)).astype(np.float32)], axis=-1))

    def rows(self, X, Y, items=True):
        """Rows (bra, first ket, quartet count) of class pair (X, Y) and their
        prefix: of work items (item_split(P, K_ab) per quartet) or of quartets."""
        bras = np.where(self.cls == X)[0]
        kets = np.where(self.cls == Y)[0]
        if len(bras) == 0 or len(kets) == 0:
            return None
        P = mg.split_of(self.pcs[X], self.pcs[Y])
        bra, ket0, cnt = [], [], []
        for i in bras:
            n = (i - kets[0] + 1) if X == Y else len(kets)
            bra.append(i)
            ket0.append(kets[0])
            cnt.append(n * (mg.item_split(P, int(self.info[i, 2])) if items else 1))
        start = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
        return np.array(bra, np.int32), np.array(ket0, np.int32), start

    def _p(self, a):
        return a.ctypes.data_as(C.c_void_p)

    def prim_cuts(self, bra, klist, taup):
        """Per list entry the primitive cut taup / max|D| over the quartet's six
        D blocks, in FP32 (the runtime's list fill)."""
        off = self.mol.shell_offsets()
        nc = [(int(x) + 1) * (int(x) + 2) // 2 for x in self.mol.shell_l]
        blk = lambda x, y: float(np.abs(self.Df[off[x]:off[x] + nc[x], off[y]:off[y] + nc[y]]).max())
        a, b = self.pair_shells[bra]
        out = []
        for j in klist:
            c, d = self.pair_shells[j]
            dq = np.float32(max(blk(a, b), blk(c, d), blk(a, c), blk(a, d), blk(b, c), blk(b, d)))
            out.append(np.float32(taup) / dq)
        return out

    def jk(self, prec, tsmall=1.0, lists=False, pmode=0, taup=0.0):
        """J and K from the class kernels of one precision (0 FP64, 1 FP32, 2 FP32
        in Algorithm 1's order, 3 double-float).  lists=True hands every row's
        kets to the kernels as an explicit ket list (the form of a mixed build's
        FP64 and demoted lists), in reversed order.  pmode 1 / 2 (with lists and
        a primitive-sorted problem): only the primitive quartets at / below the
        cut taup / max|D| of each quartet (JKArgs::pmode)."""
        lib = load(self.lmax, self.only)
        lib.emu_set_df(self._p(self.ppd), self._p(self.boysd), self._p(self.Ddf))
        assert pmode == 0 or (lists and self.pq is not None)
        J = np.zeros((self.nbf, self.nbf))
        K = np.zeros((self.nbf, self.nbf))
        for X in range(len(self.pcs)):
            for Y in range(X + 1):
                r = self.rows(X, Y)
                if r is None:
                    continue
                bra, ket0, start = r
                kofs = klist = None
                if lists:
                    cnt = np.array([(i - ket0[k] + 1) if X == Y else int((self.cls == Y).sum())
                                    for k, i in enumerate(bra)], dtype=np.int64)
                    kofs = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
                    klist = np.concatenate([np.arange(k0, k0 + c)[::-1] for k0, c in zip(ket0, cnt)]).astype(np.int32)
                    ket0 = np.zeros_like(ket0)
                kthr = None
                if pmode:
                    kthr = np.ascontiguousarray(np.concatenate(
                        [self.prim_cuts(int(i), klist[kofs[k]:kofs[k + 1]], taup) for k, i in enumerate(bra)]),
                        dtype=np.float32)
                    lib.emu_set_prim(self._p(self.pq), self._p(kthr), pmode)
                else:
                    lib.emu_set_prim(None if self.pq is None else self._p(self.pq), None, 0)
                rc = lib.emu_jk(X, Y, prec, len(self.info), self._p(self.info), self._p(self.A), self._p(self.B),
                                self._p(self.pp), self._p(self.pp2), self._p(self.ppf), self._p(self.ppf2),
                                self._p(self.alpha), len(bra), self._p(start), self._p(bra), self._p(ket0),
                                None if kofs is None else self._p(kofs), None if klist is None else self._p(klist),
                                self._p(self.boys), self._p(self.boysf), C.c_float(tsmall), self._p(self.D),
                                self._p(self.Df), self._p(J), self._p(K), self.nbf)
                assert rc == 0
        return J + J.T, K + K.T

    def schwarz(self):
        """Q_ab of every pair from the generated Schwarz kernels (pair order
        of this problem), for comparison with the oracle's."""
        lib = load(self.lmax, self.only)
        Q = np.zeros(len(self.info))
        for X in range(len(self.pcs)):
            idx = np.where(self.cls == X)[0]
            if len(idx) == 0:
                continue
            rc = lib.emu_schwarz(X, len(self.info), self._p(self.info), self._p(self.A), self._p(self.B),
                                 self._p(self.pp), self._p(self.pp2), int(idx[0]), len(idx), self._p(self.boys),
                                 Q[idx[0]:].ctypes.data_as(C.c_void_p))
            assert rc == 0
        return Q

    def grad(self, prec=0, tsmall=0.0, lists=False, pmode=0, taup=0.0):
        """dE/dR from the derivative kernels of one precision (0 FP64, 1 FP32);
        lists / pmode / taup as for jk() (the mixed gradient's FP64 list and its
        primitive split)."""
        lib = load(self.lmax, self.only)
        assert pmode == 0 or (lists and self.pq is not None)
        g = np.zeros((self.mol.xyz.shape[0], 3))
        for X in range(len(self.pcs)):
            for Y in range(X + 1):
                r = self.rows(X, Y)
                if r is None:
                    continue
                bra, ket0, start = r
                kofs = klist = kthr = None
                if lists:
                    cnt = np.array([(i - ket0[k] + 1) if X == Y else int((self.cls == Y).sum())
                                    for k, i in enumerate(bra)], dtype=np.int64)
                    kofs = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
                    klist = np.concatenate([np.arange(k0, k0 + c)[::-1] for k0, c in zip(ket0, cnt)]).astype(np.int32)
                    if pmode:
                        kthr = np.ascontiguousarray(np.concatenate(
                            [self.prim_cuts(int(i), klist[kofs[k]:kofs[k + 1]], taup) for k, i in enumerate(bra)]),
                            dtype=np.float32)
                lib.emu_set_prim(None if self.pq is None else self._p(self.pq),
                                 None if kthr is None else self._p(kthr), pmode)
                lib.emu_set_grad_lists(None if kofs is None else self._p(kofs),
                                       None if klist is None else self._p(klist))
                rc = lib.emu_grad(X, Y, prec, len(self.info), self._p(self.info), self._p(self.A), self._p(self.B),
                                  self._p(self.pp), self._p(self.pp2), self._p(self.ppf), self._p(self.ppf2),
                                  self._p(self.alpha), len(bra), self._p(start), self._p(bra), self._p(ket0),
                                  self._p(self.boys), self._p(self.boysf), C.c_float(tsmall), self._p(self.D),
                                  self.nbf, self._p(self.atoms), self._p(g))
                lib.emu_set_grad_lists(None, None)
                assert rc == 0
        return g


def jk_batched(problems, prec, tsmall=1.0):
    """J and K of several molecules through the kernels' batched mode: the
    rows of all molecules concatenated per class, each tagged with its
    molecule, the molecule's pairs and matrices looked up per row."""
    lmax = problems[0].lmax
    lib = load(lmax, None)
    nmol = len(problems)
    Js = [np.zeros((p.nbf, p.nbf)) for p in problems]
    Ks = [np.zeros((p.nbf, p.nbf)) for p in problems]
    arr = lambda xs: (C.c_void_p * nmol)(*[x.ctypes.data for x in xs])
    ptrs = dict(info=arr([p.info for p in problems]), A=arr([p.A for p in problems]), B=arr([p.B for p in problems]),
                pp=arr([p.pp for p in problems]), pp2=arr([p.pp2 for p in problems]),
                ppf=arr([p.ppf for p in problems]), ppf2=arr([p.ppf2 for p in problems]),
                D=arr([p.D for p in problems]), Df=arr([p.Df for p in problems]), J=arr(Js), K=arr(Ks))
    npair = np.array([len(p.info) for p in problems], np.int32)
    nbf = np.array([p.nbf for p in problems], np.int32)
    p0 = problems[0]
    for X in range(len(p0.pcs)):
        for Y in range(X + 1):
            bra, ket0, cnt, rowmol = [], [], [], []
            for m, p in enumerate(problems):
                r = p.rows(X, Y)
                if r is None:
                    continue
                b, k, st = r
                bra.append(b); ket0.append(k); cnt.append(np.diff(st)); rowmol.append(np.full(len(b), m, np.int32))
            if not bra:
                continue
            bra, ket0, rowmol = np.concatenate(bra), np.concatenate(ket0), np.concatenate(rowmol)
            start = np.concatenate([[0], np.cumsum(np.concatenate(cnt))]).astype(np.int64)
            rc = lib.emu_jk_batched(X, Y, prec, nmol, npair.ctypes.data_as(C.c_void_p), ptrs["info"], ptrs["A"],
                                    ptrs["B"], ptrs["pp"], ptrs["pp2"], ptrs["ppf"], ptrs["ppf2"], ptrs["D"],
                                    ptrs["Df"], ptrs["J"], ptrs["K"], nbf.ctypes.data_as(C.c_void_p), len(bra),
                                    start.ctypes.data_as(C.c_void_p), bra.ctypes.data_as(C.c_void_p),
                                    ket0.ctypes.data_as(C.c_void_p), rowmol.ctypes.data_as(C.c_void_p),
                                    p0.boys.ctypes.data_as(C.c_void_p), p0.boysf.ctypes.data_as(C.c_void_p),
                                    C.c_float(tsmall))
            assert rc == 0
    return [J + J.T for J in Js], [K + K.T for K in Ks]
