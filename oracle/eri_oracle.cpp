// CPU oracle for the four-centre electron repulsion integrals and their J/K
// contraction.  TEST INFRASTRUCTURE ONLY: tests, the package smoke check and
// the benchmark's CPU-baseline leg call it; the GPU library never does.
//
// Plain, slow and obviously correct FP64 code.  It shares nothing with the
// GPU path: the GPU evaluates integrals with McMurchie-Davidson Hermite
// expansions and a tabulated Boys function; this file uses the Obara-Saika
// vertical recurrence with the Head-Gordon-Pople horizontal recurrence (the
// recurrence family the paper describes in Sec. 2.2, "HRR + VRR down to
// [00|00]") and evaluates the Boys function by its power series.
//
// Definitions followed (the paper gives only the structure, Eq. 1 and Eq. 2
// "contraction"; the formulas are the textbook ones):
//   * primitive g = N x_A^lx y_A^ly z_A^lz exp(-alpha r_A^2), with
//     N(alpha,l) = (2 alpha/pi)^(3/4) (4 alpha)^(l/2) / sqrt((2l-1)!!); the
//     contracted axial component x^l is rescaled to unit norm;
//   * Cartesian components ordered lx descending, then ly descending;
//   * (ab|cd) = sum_klmn c_k c_l c_m c_n [a_k b_l | c_m d_n]  (Eq. 2);
//   * J_mn = sum_ls (mn|ls) D_ls,  K_mn = sum_ls (ml|ns) D_ls;
//   * E = tr(D J)/2 - tr(D K)/4;
//   * Schwarz: a shell quartet is kept iff Q_ab Q_cd >= thresh with
//     Q_ab = sqrt(max_i |(ab|ab)_ii|).
#include <cmath>
#include <cstring>
#include <vector>
#include <algorithm>
#include <cstdint>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {
typedef struct {
    int natom;
    const double* xyz;       // [natom*3]
    int nshell;
    const int* atom;         // [nshell]
    const int* l;            // [nshell]
    const int* nprim;        // [nshell]
    const int* off;          // [nshell] first primitive
    const double* exps;      // [nprim_total]
    const double* coefs;     // [nprim_total] normalised (see orc_normalize)
} orc_mol;
}

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr long double kPiL = 3.14159265358979323846264338327950288L;
constexpr int kLmax = 8;  // per shell, gradients included (l <= 3 shells + 1, with margin)

inline int ncart(int l) { return (l + 1) * (l + 2) / 2; }
inline int cumoff(int l) { return l * (l + 1) * (l + 2) / 6; }  // # Cartesian fns with total l' < l
inline int cidx(int lx, int ly, int lz) {
    int r = ly + lz;  // = l - lx
    return r * (r + 1) / 2 + lz;
}

struct Comp { int x[3]; };

const std::vector<std::vector<Comp>>& comps() {
    static std::vector<std::vector<Comp>> t = [] {
        std::vector<std::vector<Comp>> c(2 * kLmax + 2);
        for (int l = 0; l < (int)c.size(); ++l)
            for (int lx = l; lx >= 0; --lx)
                for (int ly = l - lx; ly >= 0; --ly) c[l].push_back(Comp{{lx, ly, l - lx - ly}});
        return c;
    }();
    return t;
}

inline int gidx(const int* x) { return cumoff(x[0] + x[1] + x[2]) + cidx(x[0], x[1], x[2]); }

// Boys function F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt for m = 0..mmax.
// T < 30: the convergent power series
//   F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)),
// evaluated separately for every m (all terms positive, no cancellation).
// T >= 30: F_0 = sqrt(pi/T) erf(sqrt(T)) / 2 and the upward recursion
// F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T), stable for large T.
template <class R>
void boys(int mmax, R T, R* F) {
    if (T < R(30)) {
        const R eT = std::exp(-T);
        for (int m = 0; m <= mmax; ++m) {
            // the terms are positive; their sum is compensated (Kahan) so that
            // the ~100 terms needed near T = 30 do not add up ~100 roundings
            R term = R(1) / (2 * m + 1), sum = term, comp = R(0);
            for (int k = 1; k < 400; ++k) {
                term *= R(2) * T / (2 * m + 2 * k + 1);
                const R y = term - comp;
                const R t = sum + y;
                comp = (t - sum) - y;
                sum = t;
                if (term < sum * R(sizeof(R) > sizeof(double) ? 1e-22 : 1e-18)) break;
            }
            F[m] = eT * sum;
        }
    } else {
        const R eT = std::exp(-T);
        F[0] = R(0.5) * std::sqrt(R(kPiL) / T) * std::erf(std::sqrt(T));
        for (int m = 0; m < mmax; ++m) F[m + 1] = ((2 * m + 1) * F[m] - eT) / (R(2) * T);
    }
}

struct Shell {
    int l;
    const double* R;
    int k;
    const double* e;
    const double* c;
};

// Horizontal recurrence (Head-Gordon & Pople):
//   (a, b + 1_i | = (a + 1_i, b | + (A - B)_i (a, b |
// in: G[iE][x] for e-shells of total angular momentum la..la+lb (global index
// minus cumoff(la)); out: H[ia][ib][x].
template <class R>
void hrr(int la, int lb, const R* AB, const R* G, int X, R* H) {
    const auto& C = comps();
    const int base = cumoff(la);
    const int nE = cumoff(la + lb + 1) - base;
    if (lb == 0) {
        std::memcpy(H, G, sizeof(R) * ncart(la) * X);
        return;
    }
    // level tables: T_j[(a global - base) * ncart(j) + ib][x], a over l in [la, la+lb-j]
    std::vector<R> prev(G, G + (size_t)nE * X), cur;
    for (int j = 1; j <= lb; ++j) {
        const int nbj = ncart(j), nbm = ncart(j - 1);
        const int amax = la + lb - j;
        const int na_all = cumoff(amax + 1) - base;
        cur.assign((size_t)na_all * nbj * X, R(0));
        for (int ib = 0; ib < nbj; ++ib) {
            const Comp& b = C[j][ib];
            int d = b.x[0] > 0 ? 0 : (b.x[1] > 0 ? 1 : 2);
            int bm[3] = {b.x[0], b.x[1], b.x[2]};
            bm[d] -= 1;
            const int ibm = cidx(bm[0], bm[1], bm[2]);
            for (int l = la; l <= amax; ++l) {
                for (const Comp& a : C[l]) {
                    int ap[3] = {a.x[0], a.x[1], a.x[2]};
                    ap[d] += 1;
                    const int ia = gidx(a.x) - base, iap = gidx(ap) - base;
                    R* dst = &cur[((size_t)ia * nbj + ib) * X];
                    const R* s1 = &prev[((size_t)iap * nbm + ibm) * X];
                    const R* s2 = &prev[((size_t)ia * nbm + ibm) * X];
                    for (int x = 0; x < X; ++x) dst[x] = s1[x] + AB[d] * s2[x];
                }
            }
        }
        prev.swap(cur);
    }
    // rows with l == la are the first ncart(la) a-entries
    std::memcpy(H, prev.data(), sizeof(R) * ncart(la) * ncart(lb) * X);
}

template <class R>
struct WorkT {
    std::vector<R> V, G, H, T, K;
};
using Work = WorkT<double>;

// Contracted shell quartet (ab|cd), out[ia][ib][ic][id].
// R is the arithmetic type (double, or long double for the extended-precision
// reference); the shell data are read as given and converted once.
template <class R>
void eri_quartet(const Shell& a, const Shell& b, const Shell& c, const Shell& d, R* out, WorkT<R>& w) {
    const auto& C = comps();
    const int Emax = a.l + b.l, Fmax = c.l + d.l, L = Emax + Fmax;
    const int NI = cumoff(Emax + 1), NJ = cumoff(Fmax + 1);
    const int e0 = cumoff(a.l), ne = NI - e0;
    const int f0 = cumoff(c.l), nf = NJ - f0;
    w.V.resize((size_t)(L + 1) * NI * NJ);
    w.G.assign((size_t)ne * nf, R(0));
    R* V = w.V.data();
    auto at = [&](int m, int i, int j) -> R& { return V[((size_t)m * NI + i) * NJ + j]; };
    R AB[3], CD[3];
    for (int i = 0; i < 3; ++i) { AB[i] = R(a.R[i]) - R(b.R[i]); CD[i] = R(c.R[i]) - R(d.R[i]); }
    const R AB2 = AB[0] * AB[0] + AB[1] * AB[1] + AB[2] * AB[2];
    const R CD2 = CD[0] * CD[0] + CD[1] * CD[1] + CD[2] * CD[2];
    R F[2 * (2 * kLmax) + 2];
    for (int ka = 0; ka < a.k; ++ka)
    for (int kb = 0; kb < b.k; ++kb) {
        const R al = a.e[ka], be = b.e[kb], p = al + be;
        const R Kab = std::exp(-al * be / p * AB2);
        R P[3], PA[3];
        for (int i = 0; i < 3; ++i) { P[i] = (al * R(a.R[i]) + be * R(b.R[i])) / p; PA[i] = P[i] - R(a.R[i]); }
        for (int kc = 0; kc < c.k; ++kc)
        for (int kd = 0; kd < d.k; ++kd) {
            const R ga = c.e[kc], de = d.e[kd], q = ga + de;
            const R Kcd = std::exp(-ga * de / q * CD2);
            R Q[3], QC[3], W[3], WP[3], WQ[3], PQ2 = 0;
            for (int i = 0; i < 3; ++i) {
                Q[i] = (ga * R(c.R[i]) + de * R(d.R[i])) / q;
                QC[i] = Q[i] - R(c.R[i]);
                W[i] = (p * P[i] + q * Q[i]) / (p + q);
                WP[i] = W[i] - P[i];
                WQ[i] = W[i] - Q[i];
                PQ2 += (P[i] - Q[i]) * (P[i] - Q[i]);
            }
            const R rho = p * q / (p + q);
            boys<R>(L, rho * PQ2, F);
            const R pref = R(2) * std::pow(R(kPiL), R(2.5)) / (p * q * std::sqrt(p + q)) * Kab * Kcd;
            for (int m = 0; m <= L; ++m) at(m, 0, 0) = pref * F[m];
            // electron 1: [e 0|0 0]^(m)
            for (int le = 1; le <= Emax; ++le)
                for (const Comp& e : C[le]) {
                    const int dd = e.x[0] > 0 ? 0 : (e.x[1] > 0 ? 1 : 2);
                    int e1[3] = {e.x[0], e.x[1], e.x[2]}; e1[dd] -= 1;
                    const int ie = gidx(e.x), ie1 = gidx(e1);
                    const int n1 = e1[dd];
                    int ie2 = -1;
                    if (n1 > 0) { int e2[3] = {e1[0], e1[1], e1[2]}; e2[dd] -= 1; ie2 = gidx(e2); }
                    for (int m = 0; m <= L - le; ++m) {
                        R v = PA[dd] * at(m, ie1, 0) + WP[dd] * at(m + 1, ie1, 0);
                        if (n1 > 0) v += R(n1) / (R(2) * p) * (at(m, ie2, 0) - rho / p * at(m + 1, ie2, 0));
                        at(m, ie, 0) = v;
                    }
                }
            // electron 2 (transfer form): [e 0|f 0]^(m)
            for (int lf = 1; lf <= Fmax; ++lf)
                for (const Comp& f : C[lf]) {
                    const int dd = f.x[0] > 0 ? 0 : (f.x[1] > 0 ? 1 : 2);
                    int f1[3] = {f.x[0], f.x[1], f.x[2]}; f1[dd] -= 1;
                    const int jf = gidx(f.x), jf1 = gidx(f1);
                    const int n1 = f1[dd];
                    int jf2 = -1;
                    if (n1 > 0) { int f2[3] = {f1[0], f1[1], f1[2]}; f2[dd] -= 1; jf2 = gidx(f2); }
                    for (int le = 0; le <= Emax; ++le)
                        for (const Comp& e : C[le]) {
                            const int ie = gidx(e.x);
                            const int ne1 = e.x[dd];
                            int ie1 = -1;
                            if (ne1 > 0) { int e1[3] = {e.x[0], e.x[1], e.x[2]}; e1[dd] -= 1; ie1 = gidx(e1); }
                            for (int m = 0; m <= L - le - lf; ++m) {
                                R v = QC[dd] * at(m, ie, jf1) + WQ[dd] * at(m + 1, ie, jf1);
                                if (n1 > 0) v += R(n1) / (R(2) * q) * (at(m, ie, jf2) - rho / q * at(m + 1, ie, jf2));
                                if (ne1 > 0) v += R(ne1) / (R(2) * (p + q)) * at(m + 1, ie1, jf1);
                                at(m, ie, jf) = v;
                            }
                        }
                }
            const R cc = R(a.c[ka]) * R(b.c[kb]) * R(c.c[kc]) * R(d.c[kd]);
            for (int i = 0; i < ne; ++i)
                for (int j = 0; j < nf; ++j) w.G[(size_t)i * nf + j] += cc * at(0, e0 + i, f0 + j);
        }
    }
    // bra HRR: G[e][f] -> H[ab][f]
    const int na = ncart(a.l), nb = ncart(b.l), nc = ncart(c.l), nd = ncart(d.l);
    w.H.resize((size_t)na * nb * nf);
    hrr(a.l, b.l, AB, w.G.data(), nf, w.H.data());
    // ket HRR on the transposed block: T[f][ab] -> out'[cd][ab]
    w.T.resize((size_t)nf * na * nb);
    for (int i = 0; i < na * nb; ++i)
        for (int j = 0; j < nf; ++j) w.T[(size_t)j * na * nb + i] = w.H[(size_t)i * nf + j];
    std::vector<R>& ket = w.K;
    ket.resize((size_t)nc * nd * na * nb);
    hrr(c.l, d.l, CD, w.T.data(), na * nb, ket.data());
    for (int i = 0; i < na * nb; ++i)
        for (int j = 0; j < nc * nd; ++j) out[(size_t)i * nc * nd + j] = ket[(size_t)j * na * nb + i];
}

Shell shell_of(const orc_mol& m, int s) {
    return Shell{m.l[s], m.xyz + 3 * m.atom[s], m.nprim[s], m.exps + m.off[s], m.coefs + m.off[s]};
}

std::vector<int> bf_offsets(const orc_mol& m) {
    std::vector<int> o(m.nshell + 1, 0);
    for (int s = 0; s < m.nshell; ++s) o[s + 1] = o[s] + ncart(m.l[s]);
    return o;
}

// Neumaier-compensated accumulator array.
template <class R>
struct CompArrT {
    std::vector<R> s, c;
    explicit CompArrT(size_t n = 0) : s(n, R(0)), c(n, R(0)) {}
    inline void add(size_t i, R v) {
        R t = s[i] + v;
        if (std::fabs(s[i]) >= std::fabs(v)) c[i] += (s[i] - t) + v;
        else c[i] += (v - t) + s[i];
        s[i] = t;
    }
    R get(size_t i) const { return s[i] + c[i]; }
};
using CompArr = CompArrT<double>;

void schwarz_table(const orc_mol& m, std::vector<double>& Q) {
    const int S = m.nshell;
    Q.assign((size_t)S * S, 0.0);
#pragma omp parallel
    {
        Work w;
        std::vector<double> blk;
#pragma omp for schedule(dynamic)
        for (int a = 0; a < S; ++a)
            for (int b = 0; b <= a; ++b) {
                Shell A = shell_of(m, a), B = shell_of(m, b);
                const int na = ncart(A.l), nb = ncart(B.l), n = na * nb;
                blk.resize((size_t)n * n);
                eri_quartet(A, B, A, B, blk.data(), w);
                double mx = 0.0;
                for (int i = 0; i < n; ++i) mx = std::max(mx, std::fabs(blk[(size_t)i * n + i]));
                Q[(size_t)a * S + b] = Q[(size_t)b * S + a] = std::sqrt(mx);
            }
    }
}

template <class R>
int jk_rows_impl(const orc_mol* m, const double* D, double thresh, int nrows, const int* rows,
                 double* Jr, double* Kr) {
    const auto o = bf_offsets(*m);
    const int S = m->nshell, N = o[S];
    std::vector<double> Q;
    if (thresh > 0) schwarz_table(*m, Q);
    int r0 = 0;
    for (int r = 0; r < nrows; ++r) {
        const int a = rows[r];
        if (a < 0 || a >= S) return -1;
        const int na = ncart(m->l[a]);
        CompArrT<R> Jt((size_t)na * N), Kt((size_t)na * N);
#pragma omp parallel
        {
            WorkT<R> w;
            std::vector<R> blk;
            CompArrT<R> Jl((size_t)na * N), Kl((size_t)na * N);
#pragma omp for schedule(dynamic)
            for (int b = 0; b < S; ++b)
                for (int c = 0; c < S; ++c)
                    for (int d = 0; d < S; ++d) {
                        if (thresh > 0 && Q[(size_t)a * S + b] * Q[(size_t)c * S + d] < thresh) continue;
                        Shell A = shell_of(*m, a), B = shell_of(*m, b), C = shell_of(*m, c), Dd = shell_of(*m, d);
                        const int nb = ncart(B.l), nc = ncart(C.l), nd = ncart(Dd.l);
                        blk.resize((size_t)na * nb * nc * nd);
                        eri_quartet(A, B, C, Dd, blk.data(), w);
                        for (int i = 0; i < na; ++i) for (int j = 0; j < nb; ++j)
                        for (int k = 0; k < nc; ++k) for (int l = 0; l < nd; ++l) {
                            const R v = blk[((i * nb + j) * nc + k) * nd + l];
                            Jl.add((size_t)i * N + o[b] + j, v * R(D[(size_t)(o[c] + k) * N + o[d] + l]));
                            Kl.add((size_t)i * N + o[c] + k, v * R(D[(size_t)(o[b] + j) * N + o[d] + l]));
                        }
                    }
#pragma omp critical
            for (size_t i = 0; i < (size_t)na * N; ++i) {
                Jt.add(i, Jl.s[i]); Jt.add(i, Jl.c[i]);
                Kt.add(i, Kl.s[i]); Kt.add(i, Kl.c[i]);
            }
        }
        for (int i = 0; i < na; ++i)
            for (int j = 0; j < N; ++j) {
                Jr[(size_t)(r0 + i) * N + j] = (double)Jt.get((size_t)i * N + j);
                Kr[(size_t)(r0 + i) * N + j] = (double)Kt.get((size_t)i * N + j);
            }
        r0 += na;
    }
    return 0;
}

// J and K over the screened quartets (mode 0 all, mode 1 unique with images),
// in arithmetic type R; see orc_jk.
template <class R>
long long jk_impl(const orc_mol* m, const double* D, double thresh, int mode, double* J, double* K) {
    const auto o = bf_offsets(*m);
    const int S = m->nshell, N = o[S];
    std::vector<double> Q;
    if (thresh > 0) schwarz_table(*m, Q);
    CompArrT<R> Jt((size_t)N * N), Kt((size_t)N * N);
    long long kept = 0;
#pragma omp parallel reduction(+ : kept)
    {
        WorkT<R> w;
        std::vector<R> blk;
        CompArrT<R> Jl((size_t)N * N), Kl((size_t)N * N);
#pragma omp for schedule(dynamic)
        for (int a = 0; a < S; ++a)
            for (int b = 0; b < S; ++b) {
                if (mode == 1 && b > a) continue;
                for (int c = 0; c < S; ++c)
                    for (int d = 0; d < S; ++d) {
                        if (mode == 1) {
                            if (d > c) continue;
                            const long ab = (long)a * (a + 1) / 2 + b, cd = (long)c * (c + 1) / 2 + d;
                            if (cd > ab) continue;
                        }
                        if (thresh > 0 && Q[(size_t)a * S + b] * Q[(size_t)c * S + d] < thresh) continue;
                        ++kept;
                        Shell A = shell_of(*m, a), B = shell_of(*m, b), C = shell_of(*m, c), Dd = shell_of(*m, d);
                        const int na = ncart(A.l), nb = ncart(B.l), nc = ncart(C.l), nd = ncart(Dd.l);
                        blk.resize((size_t)na * nb * nc * nd);
                        eri_quartet(A, B, C, Dd, blk.data(), w);
                        if (mode == 0) {
                            for (int i = 0; i < na; ++i) for (int j = 0; j < nb; ++j)
                            for (int k = 0; k < nc; ++k) for (int l = 0; l < nd; ++l) {
                                const R v = blk[((i * nb + j) * nc + k) * nd + l];
                                const int mu = o[a] + i, nu = o[b] + j, la = o[c] + k, si = o[d] + l;
                                Jl.add((size_t)mu * N + nu, v * R(D[(size_t)la * N + si]));
                                Kl.add((size_t)mu * N + la, v * R(D[(size_t)nu * N + si]));
                            }
                        } else {
                            const long ab = (long)a * (a + 1) / 2 + b, cd = (long)c * (c + 1) / 2 + d;
                            R s = 1;
                            if (a == b) s *= 0.5;
                            if (c == d) s *= 0.5;
                            if (ab == cd) s *= 0.5;
                            for (int i = 0; i < na; ++i) for (int j = 0; j < nb; ++j)
                            for (int k = 0; k < nc; ++k) for (int l = 0; l < nd; ++l) {
                                const R v = s * blk[((i * nb + j) * nc + k) * nd + l];
                                const int p = o[a] + i, q = o[b] + j, r = o[c] + k, t = o[d] + l;
                                // the eight images (pq|rt) (qp|rt) (pq|tr) (qp|tr) (rt|pq) (tr|pq) (rt|qp) (tr|qp)
                                const int img[8][4] = {{p, q, r, t}, {q, p, r, t}, {p, q, t, r}, {q, p, t, r},
                                                       {r, t, p, q}, {t, r, p, q}, {r, t, q, p}, {t, r, q, p}};
                                for (int g = 0; g < 8; ++g) {
                                    const int* x = img[g];
                                    Jl.add((size_t)x[0] * N + x[1], v * R(D[(size_t)x[2] * N + x[3]]));
                                    Kl.add((size_t)x[0] * N + x[2], v * R(D[(size_t)x[1] * N + x[3]]));
                                }
                            }
                        }
                    }
            }
#pragma omp critical
        for (size_t i = 0; i < (size_t)N * N; ++i) {
            Jt.add(i, Jl.s[i]); Jt.add(i, Jl.c[i]);
            Kt.add(i, Kl.s[i]); Kt.add(i, Kl.c[i]);
        }
    }
    for (size_t i = 0; i < (size_t)N * N; ++i) { J[i] = (double)Jt.get(i); K[i] = (double)Kt.get(i); }
    return kept;
}

}  // namespace

extern "C" {

void orc_boys(int mmax, double T, double* F) { boys(mmax, T, F); }

// Normalise contraction coefficients (see the header comment): c_out[i] = c[i] N(alpha_i, l) / sqrt(S).
void orc_normalize(int nshell, const int* l, const int* nprim, const int* off, const double* exps,
                   const double* coefs, double* out) {
    for (int s = 0; s < nshell; ++s) {
        const int L = l[s], k = nprim[s], o = off[s];
        double dfact = 1.0;  // (2L-1)!!
        for (int i = 2 * L - 1; i > 1; i -= 2) dfact *= i;
        for (int i = 0; i < k; ++i) {
            const double a = exps[o + i];
            out[o + i] = coefs[o + i] * std::pow(2.0 * a / kPi, 0.75) * std::pow(4.0 * a, 0.5 * L) / std::sqrt(dfact);
        }
        double S = 0.0;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                const double p = exps[o + i] + exps[o + j];
                S += out[o + i] * out[o + j] * std::pow(kPi / p, 1.5) * dfact / std::pow(2.0 * p, L);
            }
        const double f = 1.0 / std::sqrt(S);
        for (int i = 0; i < k; ++i) out[o + i] *= f;
    }
}

// One contracted quartet with explicit shells: out[na*nb*nc*nd].
int orc_eri_quartet(const double* RA, int la, int ka, const double* ea, const double* ca,
                    const double* RB, int lb, int kb, const double* eb, const double* cb,
                    const double* RC, int lc, int kc, const double* ec, const double* cc,
                    const double* RD, int ld, int kd, const double* ed, const double* cd, double* out) {
    if (la < 0 || lb < 0 || lc < 0 || ld < 0 || la > kLmax || lb > kLmax || lc > kLmax || ld > kLmax) return -1;
    Work w;
    eri_quartet(Shell{la, RA, ka, ea, ca}, Shell{lb, RB, kb, eb, cb}, Shell{lc, RC, kc, ec, cc},
                Shell{ld, RD, kd, ed, cd}, out, w);
    return 0;
}

// Every integral of a (small) molecule: out[nbf^4], (mn|ls) at ((m*nbf+n)*nbf+l)*nbf+s.
int orc_eri_full(const orc_mol* m, double* out) {
    const auto o = bf_offsets(*m);
    const int S = m->nshell, N = o[S];
#pragma omp parallel
    {
        Work w;
        std::vector<double> blk;
#pragma omp for schedule(dynamic) collapse(2)
        for (int a = 0; a < S; ++a)
            for (int b = 0; b < S; ++b)
                for (int c = 0; c < S; ++c)
                    for (int d = 0; d < S; ++d) {
                        Shell A = shell_of(*m, a), B = shell_of(*m, b), C = shell_of(*m, c), D = shell_of(*m, d);
                        const int na = ncart(A.l), nb = ncart(B.l), nc = ncart(C.l), nd = ncart(D.l);
                        blk.resize((size_t)na * nb * nc * nd);
                        eri_quartet(A, B, C, D, blk.data(), w);
                        for (int i = 0; i < na; ++i) for (int j = 0; j < nb; ++j)
                        for (int k = 0; k < nc; ++k) for (int l = 0; l < nd; ++l)
                            out[(((size_t)(o[a] + i) * N + o[b] + j) * N + o[c] + k) * N + o[d] + l] =
                                blk[((i * nb + j) * nc + k) * nd + l];
                    }
    }
    return 0;
}

// Schwarz factors Q[nshell*nshell].
void orc_schwarz(const orc_mol* m, double* Q) {
    std::vector<double> q;
    schwarz_table(*m, q);
    std::memcpy(Q, q.data(), sizeof(double) * q.size());
}

// J and K.  mode 0: every shell quartet (S^4, the plain definition);
// mode 1: unique quartets a>=b, c>=d, ab>=cd, each added to all of its
// permutational images.  thresh <= 0 disables screening.  Returns the number
// of unique shell quartets kept (mode 1) or of all quartets kept (mode 0).
long long orc_jk(const orc_mol* m, const double* D, double thresh, int mode, double* J, double* K) {
    return jk_impl<double>(m, D, thresh, mode, J, K);
}

// The same J and K with every integral and sum in long double (x86: 64-bit
// significand): an extended-precision reference for the FP64 result (the
// Schwarz screening, from the FP64 Q, is the same).
long long orc_jk_ld(const orc_mol* m, const double* D, double thresh, int mode, double* J, double* K) {
    return jk_impl<long double>(m, D, thresh, mode, J, K);
}

// J/K contributions of an explicit list of unique shell quartets
// quartets[4*i..4*i+3] = (a, b, c, d) with a >= b, c >= d, ab >= cd, each added
// to all of its permutational images (used to time a bounded sample of a
// workload).  Returns the number processed, or -1 for a malformed entry.
long long orc_jk_quartets(const orc_mol* m, const double* D, long long nq, const int* quartets, double* J, double* K) {
    const auto o = bf_offsets(*m);
    const int S = m->nshell, N = o[S];
    for (long long i = 0; i < nq; ++i) {
        const int* q = quartets + 4 * i;
        for (int k = 0; k < 4; ++k) if (q[k] < 0 || q[k] >= S) return -1;
        const long ab = (long)q[0] * (q[0] + 1) / 2 + q[1], cd = (long)q[2] * (q[2] + 1) / 2 + q[3];
        if (q[1] > q[0] || q[3] > q[2] || cd > ab) return -1;
    }
    CompArr Jt((size_t)N * N), Kt((size_t)N * N);
#pragma omp parallel
    {
        Work w;
        std::vector<double> blk;
        CompArr Jl((size_t)N * N), Kl((size_t)N * N);
#pragma omp for schedule(dynamic, 16)
        for (long long i = 0; i < nq; ++i) {
            const int a = quartets[4 * i], b = quartets[4 * i + 1], c = quartets[4 * i + 2], d = quartets[4 * i + 3];
            Shell A = shell_of(*m, a), B = shell_of(*m, b), C = shell_of(*m, c), Dd = shell_of(*m, d);
            const int na = ncart(A.l), nb = ncart(B.l), nc = ncart(C.l), nd = ncart(Dd.l);
            blk.resize((size_t)na * nb * nc * nd);
            eri_quartet(A, B, C, Dd, blk.data(), w);
            const long ab = (long)a * (a + 1) / 2 + b, cd = (long)c * (c + 1) / 2 + d;
            double s = 1.0;
            if (a == b) s *= 0.5;
            if (c == d) s *= 0.5;
            if (ab == cd) s *= 0.5;
            for (int ii = 0; ii < na; ++ii) for (int j = 0; j < nb; ++j)
            for (int k = 0; k < nc; ++k) for (int l = 0; l < nd; ++l) {
                const double v = s * blk[((ii * nb + j) * nc + k) * nd + l];
                const int p = o[a] + ii, q = o[b] + j, r = o[c] + k, t = o[d] + l;
                const int img[8][4] = {{p, q, r, t}, {q, p, r, t}, {p, q, t, r}, {q, p, t, r},
                                       {r, t, p, q}, {t, r, p, q}, {r, t, q, p}, {t, r, q, p}};
                for (int g = 0; g < 8; ++g) {
                    const int* x = img[g];
                    Jl.add((size_t)x[0] * N + x[1], v * D[(size_t)x[2] * N + x[3]]);
                    Kl.add((size_t)x[0] * N + x[2], v * D[(size_t)x[1] * N + x[3]]);
                }
            }
        }
#pragma omp critical
        for (size_t i = 0; i < (size_t)N * N; ++i) {
            Jt.add(i, Jl.s[i]); Jt.add(i, Jl.c[i]);
            Kt.add(i, Kl.s[i]); Kt.add(i, Kl.c[i]);
        }
    }
    for (size_t i = 0; i < (size_t)N * N; ++i) { J[i] = Jt.get(i); K[i] = Kt.get(i); }
    return nq;
}

// Rows of J and K: for every shell in rows[], J[mu,:] and K[mu,:] for all mu
// of that shell, over the full (screened) quartet list.  Jr/Kr are
// [sum ncart(rows) x nbf].
int orc_jk_rows(const orc_mol* m, const double* D, double thresh, int nrows, const int* rows,
                double* Jr, double* Kr) {
    return jk_rows_impl<double>(m, D, thresh, nrows, rows, Jr, Kr);
}

// The same rows with every integral and sum in long double (x86: 64-bit
// significand): an extended-precision reference for the FP64 rows (the
// Schwarz screening, from the FP64 Q, is the same).
int orc_jk_rows_ld(const orc_mol* m, const double* D, double thresh, int nrows, const int* rows,
                   double* Jr, double* Kr) {
    return jk_rows_impl<long double>(m, D, thresh, nrows, rows, Jr, Kr);
}

// E = tr(D J)/2 - tr(D K)/4 with a compensated sum.
double orc_energy(int n, const double* D, const double* J, const double* K) {
    CompArr acc(1);
    for (size_t i = 0; i < (size_t)n * n; ++i) {
        acc.add(0, 0.5 * D[i] * J[i]);
        acc.add(0, -0.25 * D[i] * K[i]);
    }
    return acc.get(0);
}

// Nuclear gradient of E = tr(DJ)/2 - tr(DK)/4 for a fixed density D:
//   dE/dR = sum_{abcd} d(ab|cd)/dR * Gamma_abcd,
//   Gamma_abcd = D_ab D_cd / 2 - D_ac D_bd / 4.
// Derivative integrals by the shift rule on each of the four centres:
//   d phi_a / dA_i = 2 alpha phi_{a+1_i} - a_i phi_{a-1_i};
// all four centres are differentiated explicitly, so translational
// invariance (sum over atoms = 0) is a check, not an assumption.
// mode 0: every quartet; mode 1: unique quartets with the symmetrised weight
//   s * (4 D_ab D_cd - D_ac D_bd - D_ad D_bc).
int orc_grad(const orc_mol* m, const double* D, double thresh, int mode, double* grad) {
    const auto o = bf_offsets(*m);
    const int S = m->nshell, N = o[S];
    std::vector<double> Q;
    if (thresh > 0) schwarz_table(*m, Q);
    // per-shell shifted coefficient sets: 2 alpha c (for l+1) and c (for l-1)
    int ptot = 0;
    for (int s = 0; s < S; ++s) ptot = std::max(ptot, m->off[s] + m->nprim[s]);
    std::vector<double> c2a(ptot);
    for (int i = 0; i < ptot; ++i) c2a[i] = 2.0 * m->exps[i] * m->coefs[i];
    CompArr G((size_t)m->natom * 3);
#pragma omp parallel
    {
        Work w;
        std::vector<double> Ip, Im;
        CompArr Gl((size_t)m->natom * 3);
        const auto& C = comps();
#pragma omp for schedule(dynamic)
        for (int a = 0; a < S; ++a)
            for (int b = 0; b < S; ++b) {
                if (mode == 1 && b > a) continue;
                for (int c = 0; c < S; ++c)
                    for (int d = 0; d < S; ++d) {
                        double s = 1.0;
                        if (mode == 1) {
                            if (d > c) continue;
                            const long ab = (long)a * (a + 1) / 2 + b, cd = (long)c * (c + 1) / 2 + d;
                            if (cd > ab) continue;
                            if (a == b) s *= 0.5;
                            if (c == d) s *= 0.5;
                            if (ab == cd) s *= 0.5;
                        }
                        if (thresh > 0 && Q[(size_t)a * S + b] * Q[(size_t)c * S + d] < thresh) continue;
                        Shell sh[4] = {shell_of(*m, a), shell_of(*m, b), shell_of(*m, c), shell_of(*m, d)};
                        const int idx[4] = {a, b, c, d};
                        const int n[4] = {ncart(sh[0].l), ncart(sh[1].l), ncart(sh[2].l), ncart(sh[3].l)};
                        // weight of every component quartet
                        std::vector<double> gam((size_t)n[0] * n[1] * n[2] * n[3]);
                        for (int i = 0; i < n[0]; ++i) for (int j = 0; j < n[1]; ++j)
                        for (int k = 0; k < n[2]; ++k) for (int l = 0; l < n[3]; ++l) {
                            const size_t mu = o[a] + i, nu = o[b] + j, la = o[c] + k, si = o[d] + l;
                            double g;
                            if (mode == 0) g = 0.5 * D[mu * N + nu] * D[la * N + si] - 0.25 * D[mu * N + la] * D[nu * N + si];
                            else g = s * (4.0 * D[mu * N + nu] * D[la * N + si] - D[mu * N + la] * D[nu * N + si]
                                          - D[mu * N + si] * D[nu * N + la]);
                            gam[((i * n[1] + j) * n[2] + k) * n[3] + l] = g;
                        }
                        for (int centre = 0; centre < 4; ++centre) {
                            const Shell& X = sh[centre];
                            const int sidx = idx[centre];
                            Shell plus{X.l + 1, X.R, X.k, X.e, c2a.data() + m->off[sidx]};
                            Shell minus{X.l - 1, X.R, X.k, X.e, X.c};
                            Shell qp[4] = {sh[0], sh[1], sh[2], sh[3]};
                            qp[centre] = plus;
                            int np[4] = {n[0], n[1], n[2], n[3]};
                            np[centre] = ncart(X.l + 1);
                            Ip.resize((size_t)np[0] * np[1] * np[2] * np[3]);
                            eri_quartet(qp[0], qp[1], qp[2], qp[3], Ip.data(), w);
                            int nm[4] = {n[0], n[1], n[2], n[3]};
                            if (X.l > 0) {
                                Shell qm[4] = {sh[0], sh[1], sh[2], sh[3]};
                                qm[centre] = minus;
                                nm[centre] = ncart(X.l - 1);
                                Im.resize((size_t)nm[0] * nm[1] * nm[2] * nm[3]);
                                eri_quartet(qm[0], qm[1], qm[2], qm[3], Im.data(), w);
                            }
                            double acc[3] = {0, 0, 0};
                            for (int i = 0; i < n[0]; ++i) for (int j = 0; j < n[1]; ++j)
                            for (int k = 0; k < n[2]; ++k) for (int l = 0; l < n[3]; ++l) {
                                const double g = gam[((i * n[1] + j) * n[2] + k) * n[3] + l];
                                if (g == 0.0) continue;
                                int cmp[4] = {i, j, k, l};
                                const Comp& x = C[X.l][cmp[centre]];
                                for (int dir = 0; dir < 3; ++dir) {
                                    int up[3] = {x.x[0], x.x[1], x.x[2]}; up[dir] += 1;
                                    int cp[4] = {i, j, k, l};
                                    cp[centre] = cidx(up[0], up[1], up[2]);
                                    double v = Ip[((cp[0] * np[1] + cp[1]) * np[2] + cp[2]) * np[3] + cp[3]];
                                    if (x.x[dir] > 0) {
                                        int dn[3] = {x.x[0], x.x[1], x.x[2]}; dn[dir] -= 1;
                                        int cm[4] = {i, j, k, l};
                                        cm[centre] = cidx(dn[0], dn[1], dn[2]);
                                        v -= x.x[dir] * Im[((cm[0] * nm[1] + cm[1]) * nm[2] + cm[2]) * nm[3] + cm[3]];
                                    }
                                    acc[dir] += g * v;
                                }
                            }
                            const int at = m->atom[sidx];
                            for (int dir = 0; dir < 3; ++dir) Gl.add((size_t)at * 3 + dir, acc[dir]);
                        }
                    }
            }
#pragma omp critical
        for (size_t i = 0; i < (size_t)m->natom * 3; ++i) { G.add(i, Gl.s[i]); G.add(i, Gl.c[i]); }
    }
    for (size_t i = 0; i < (size_t)m->natom * 3; ++i) grad[i] = G.get(i);
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
