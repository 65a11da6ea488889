// Device-side building blocks shared by the generated per-class ERI kernels
// and the host runtime: argument structures, the tabulated Boys function, the
// quartet-row lookup and the fused J/K digestion.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <type_traits>

namespace gb {

// ------------------------------------------------------------------ double-float
// A value carried as an unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2),
// about 44 significant bits, with every operation on the FP32 pipe: the
// mixed build's largest-bound quartets run in it instead of FP64 (the GB300's
// FP64 rate is 1/64 of its FP32 rate).  Sums use Knuth's two-sum on the high
// parts, products the FMA-exact product of the high parts (Dekker/Knuth
// error-free transformations); the low parts are added without their own
// error terms, which bounds every operation's error by ~2^-44 of its operands.
struct dfl {
    float hi, lo;
    __host__ __device__ constexpr dfl(float h = 0.f, float l = 0.f) : hi(h), lo(l) {}
    __host__ __device__ constexpr dfl(int v) : hi((float)v), lo(0.f) {}
    dfl(double) = delete;  // a double would lose its low bits silently: split it with df_const
    explicit __host__ __device__ operator double() const { return (double)hi + (double)lo; }
};

// hi + lo split of a double (compile-time constants and host / setup code)
__host__ __device__ constexpr dfl df_const(double x) { return dfl((float)x, (float)(x - (double)(float)x)); }

// the global fma overloads stay visible next to the double-float one below
using ::fma;
using ::fmaf;

__device__ __forceinline__ dfl df_norm(float s, float e) {  // fast two-sum, |s| >= |e|
    const float h = s + e;
    return dfl(h, e - (h - s));
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb) + (a.lo + b.lo);
    return df_norm(s, e);
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return df_norm(p, e);
}
__device__ __forceinline__ dfl operator*(dfl a, float b) {
    const float p = a.hi * b;
    return df_norm(p, fmaf(a.lo, b, fmaf(a.hi, b, -p)));
}
__device__ __forceinline__ dfl operator*(float a, dfl b) { return b * a; }
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { a = a + b; return a; }
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) { a = a * b; return a; }
__device__ __forceinline__ dfl& operator*=(dfl& a, float b) { a = a * b; return a; }
__device__ __forceinline__ bool operator==(dfl a, float b) { return a.hi == b && a.lo == 0.f; }
__device__ __forceinline__ dfl fma(dfl a, dfl b, dfl c) { return a * b + c; }
__device__ __forceinline__ dfl df_rsqrt(dfl x) {
    // rsqrtf of the high part, then one Newton step in double-float
    const dfl r(rsqrtf(x.hi));
    return r + r * (dfl(0.5f) - (x * (r * r)) * 0.5f);
}
template <class T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }
__device__ __forceinline__ dfl ldg(const dfl* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return dfl(v.x, v.y);
}

constexpr int kLmaxShell = 3;
constexpr int kLmaxBoys = 4 * kLmaxShell + 1;  // highest F_m needed (gradients of (ff|ff))
constexpr int kBoysTaylor = 8;                  // Taylor terms j = 0..7 around each grid point
constexpr int kBoysPerUnit = 16;                // grid step 1/16
constexpr int kBoysNgrid = 80 * kBoysPerUnit + 1;  // T_k = k/16 on [0, 80]
constexpr double kBoysTmax = 80.0;
constexpr int kBoysRows = kLmaxBoys + 2;        // rows m = 0..kLmaxBoys, then exp(-T)
constexpr int kBoysRowLen = kBoysTaylor;        // coefficients per (k, row)

// Table layout: tab[(k * kBoysRows + m) * kBoysTaylor + j] = F_{m+j}(T_k) / j!
// for m = 0..kLmaxBoys, and row kLmaxBoys+1 holds exp(-T_k) / j!.
// F_L(T) = sum_j tab[k][L][j] (T_k - T)^j (Taylor expansion of F_L, using
// dF_m/dT = -F_{m+1}).  Lower orders follow from the downward recursion
// F_m = (2T F_{m+1} + exp(-T)) / (2m + 1).  For T >= 80 the asymptotic form
// F_0 = sqrt(pi/T)/2, F_{m+1} = (2m+1) F_m / (2T) is exact to double
// precision for every m <= kLmaxBoys (exp(-T) is below 1e-17 F_m there).

struct PairsView {
    int npair;
    const int4* info;      // per pair: fa, fb (first basis functions of shells a, b), nprim pairs, first prim pair
    const double4* A;      // per pair: centre of a (xyz), w = Q_ab (Schwarz factor)
    const double4* B;      // per pair: centre of b (xyz), w = unused
    const double4* pp;     // per primitive pair: P (xyz), p
    const double2* pp2;    // per primitive pair: kappa = sqrt(2 pi^(5/2)) K_AB c_a c_b / p, 1/(2p)
    // FP32 kernels see only centre differences, each formed in FP64 and then
    // rounded once, so that no FP32 subtraction of two absolute coordinates
    // (|R| ~ 10 bohr) loses the digits of a short distance:
    const float4* ppf;     // per primitive pair: P - A (xyz), p
    const float4* ppf2;    // per primitive pair: P - B (xyz), kappa
    const double* alpha;   // per primitive pair: exponent of the shell-a primitive (gradients)
    // per pair: centre of a split into two floats per coordinate, [2i] = hi =
    // (float)A, [2i + 1] = lo = (float)(A - hi): FP32 kernels form A - C as
    // (hi_A - hi_C) + (lo_A - lo_C) without an FP64 operation
    const float4* Ahl;
    // per primitive pair, double-float kernels: 5 float4 = (P-A)x,(P-A)y | (P-A)z,(P-B)x |
    // (P-B)y,(P-B)z | p, kappa | 1/(2p), - (each value as hi, lo; differences formed in FP64)
    const float4* ppd;
    // per primitive pair: its Schwarz factor sqrt(max_i |(pp|pp)_ii|) (contraction
    // coefficients included), the primitive pairs of every pair sorted by it,
    // largest first, so that |(p|q)| <= pq[p] pq[q] for every primitive quartet
    // and the primitive quartets above a cut form a prefix of every ket loop
    const float* pq;
};

struct RowsView {
    int nrows;
    const long long* start;  // [nrows + 1], exclusive prefix of the per-row work items
    const int* bra;          // bra pair of every row
    const int* ket0;         // first ket pair of every row (kets are contiguous) ...
    const long long* kofs;   // ... or, if klist is set, the row's first entry in klist
    const int* klist;        // explicit ket pairs (rows of a mixed build's FP64 / demoted lists)
    // per klist entry (primitive split of a mixed build's FP64 list): the cut
    // on pq[p] pq[q] that separates the quartet's large primitive quartets (FP64
    // tier) from the rest (FP32), tau_p / max|D| of the quartet's D blocks
    const float* kthr;
};

// One molecule of a batched launch.
struct BatchMol {
    PairsView pairs;
    const double* D;
    float* Df;                // FP32 copy of D (mixed builds; written by the max|D| pass)
    dfl* Ddf;                 // double-float copy of D (mixed builds)
    float* Dsh;               // mixed builds: max |D| per shell block [nshell^2]
    const int* bf_shell;      // shell of every basis function
    const int2* psh;          // shells a, b of every kept pair
    int nshell;
    double* J;
    double* K;
    double* Jlo;              // compensated accumulation of FP64 builds (nullptr: plain atomics)
    double* Klo;
    int nbf;
};

struct JKArgs {
    PairsView pairs;
    RowsView rows;            // quartets of this launch: rows.start[rows.nrows] (read on the device)
    const double* boys;       // FP64 Boys table
    const float* boysf;       // FP32 Boys table
    float tsmall;             // mixed kernels: FP64 Boys below this T
    const double* D;
    const float* Df;          // FP32 copy of D (mixed builds: digestion of the FP32 quartets)
    const dfl* Ddf;           // double-float copy of D (mixed builds: digestion of the double-float quartets)
    const float2* boysd;      // double-float Boys table (hi, lo of the FP64 table)
    double* J;                // accumulates J' (J = J' + J'^T afterwards)
    double* K;                // accumulates K'
    double* Jlo;              // FP64 builds: remainders of the split accumulation (see jk_add);
    double* Klo;              // nullptr: plain FP64 atomics (mixed builds)
    int nbf;
    const BatchMol* mols;     // batched launches: per-molecule data (nullptr: single molecule above)
    const int* row_mol;       // batched launches: molecule of every row
    // primitive quartets a work item evaluates: 0 all; 1 those with
    // pq[p] pq[q] >= rows.kthr[entry] (FP64 / double-float tier); 2 the others
    // (their FP32 complement, launched over the same list)
    int pmode;
};

// Work items of one shell quartet whose bra pair has z primitive pairs, in a
// class whose quartets spread over at most P threads: the largest divisor of z
// not above P, so that every item of the quartet loops over the same number of
// bra primitive pairs (the lanes of a warp, items of the same quartets, stay
// in step).
__host__ __device__ __forceinline__ int item_split(int P, int z) {
    int d = P < z ? P : z;
    while (d > 1 && z % d != 0) --d;
    return d < 1 ? 1 : d;
}

// The ket primitive pairs [j0, j1) that one bra primitive pair `ip` of a work
// item evaluates under primitive mode `mode` (see JKArgs::pmode).  The kets'
// factors are sorted descending, so pq[ip] pq[k0 + j] >= thr holds on a prefix;
// both tiers take the decision with the same FP32 product, so every primitive
// quartet is evaluated exactly once.
__device__ __forceinline__ void prim_range(const float* __restrict__ pq, int ip, int k0, int nk, float thr, int mode,
                                           int& j0, int& j1) {
    const float qb = __ldg(pq + ip);
    int n = 0;
    while (n < nk && __fmul_rn(qb, __ldg(pq + k0 + n)) >= thr) ++n;
    j0 = mode == 1 ? 0 : n;
    j1 = mode == 1 ? n : nk;
}

struct GradArgs {
    PairsView pairs;
    RowsView rows;            // work items of the launch: rows.start[0] .. rows.start[nrows] - 1 (device)
    const double* boys;
    const float* boysf;       // FP32 Boys table (FP32 derivative kernels)
    float tsmall;             // FP32 kernels: FP64 Boys below this T
    const double* D;
    int nbf;
    const int2* atoms;        // per pair: atoms of shells a and b
    double* grad;             // [natom * 3], accumulated
    int pmode;                // primitive split of a mixed gradient's FP64 list (as JKArgs::pmode)
};

// Schwarz kernels spread the bra primitive pairs of a pair over up to this
// many threads, each writing its partial diagonal (ab|ab)_ii.
constexpr int kSchwarzSplit = 8;

struct SchwarzArgs {
    PairsView pairs;
    int first, count;         // pair range (one angular class)
    const double* boys;
    double* diag;             // [count][kSchwarzSplit][NAB] partial diagonals, zeroed by the caller
    double* Q;                // out: Q for pairs first..first+count-1
};


// ------------------------------------------------------------------ Boys
template <int L>
__device__ __forceinline__ void boys_f64(double T, double* F, const double* __restrict__ tab) {
    if (T < kBoysTmax) {
        const int k = __double2int_rn(T * kBoysPerUnit);
        const double d = k * (1.0 / kBoysPerUnit) - T;
        const double* c = tab + ((size_t)k * kBoysRows + L) * kBoysTaylor;
        double f = __ldg(c + kBoysTaylor - 1);
#pragma unroll
        for (int j = kBoysTaylor - 2; j >= 0; --j) f = fma(f, d, __ldg(c + j));
        F[L] = f;
        if (L > 0) {
            const double* e = tab + ((size_t)k * kBoysRows + kLmaxBoys + 1) * kBoysTaylor;
            double eT = __ldg(e + kBoysTaylor - 1);
#pragma unroll
            for (int j = kBoysTaylor - 2; j >= 0; --j) eT = fma(eT, d, __ldg(e + j));
            const double t2 = 2.0 * T;
#pragma unroll
            for (int m = L - 1; m >= 0; --m) F[m] = fma(t2, F[m + 1], eT) * (1.0 / (2 * m + 1));
        }
    } else {
        const double r = rsqrt(T);
        F[0] = 0.88622692545275801365 * r;  // sqrt(pi)/2 / sqrt(T)
        const double h = 0.5 * r * r;       // 1 / (2T)
#pragma unroll
        for (int m = 0; m < L; ++m) F[m + 1] = F[m] * ((2 * m + 1) * h);
    }
}

// 1/(2m+1) as hi + lo floats (the downward recursions of boys_f32 and boys_df).
// The FP32 roundings of these reciprocals are too large for 12 of the 13
// m >= 1 (by up to 5e-8 relative): multiplying by them alone would bias F_m
// of every FP32 quartet the same way, an error that adds up over quartets
// instead of cancelling.
static __constant__ dfl kInvOddDf[kLmaxBoys + 1] = {
    df_const(1.0), df_const(1.0 / 3), df_const(1.0 / 5), df_const(1.0 / 7), df_const(1.0 / 9),
    df_const(1.0 / 11), df_const(1.0 / 13), df_const(1.0 / 15), df_const(1.0 / 17), df_const(1.0 / 19),
    df_const(1.0 / 21), df_const(1.0 / 23), df_const(1.0 / 25), df_const(1.0 / 27)};

// Slot of a Taylor row of the FP32 table that holds the low part of the row's
// leading coefficient (FP32 evaluation uses terms 0..4 only): the series is
// summed smallest terms first and the leading term's hi part added last, so
// the one rounding of F_m(T_k) to FP32 is not shared by every T of a bin.
constexpr int kBoysLoSlot = 5;

template <int L>
__device__ __forceinline__ void boys_f32(float T, float* F, const float* __restrict__ tab) {
    if (T < (float)kBoysTmax) {
        const int k = __float2int_rn(T * kBoysPerUnit);
        const float d = k * (1.0f / kBoysPerUnit) - T;
        const float* c = tab + ((size_t)k * kBoysRows + L) * kBoysTaylor;
        // |d| <= 1/32: five terms reach FP32 rounding
        float f = __ldg(c + 4);
#pragma unroll
        for (int j = 3; j >= 1; --j) f = fmaf(f, d, __ldg(c + j));
        F[L] = __ldg(c) + fmaf(f, d, __ldg(c + kBoysLoSlot));
        if (L > 0) {
            const float* e = tab + ((size_t)k * kBoysRows + kLmaxBoys + 1) * kBoysTaylor;
            float eT = __ldg(e + 4);
#pragma unroll
            for (int j = 3; j >= 1; --j) eT = fmaf(eT, d, __ldg(e + j));
            eT = __ldg(e) + fmaf(eT, d, __ldg(e + kBoysLoSlot));
            const float t2 = 2.0f * T;
#pragma unroll
            for (int m = L - 1; m >= 0; --m) {
                const float y = fmaf(t2, F[m + 1], eT);
                F[m] = m == 0 ? y : fmaf(y, kInvOddDf[m].hi, y * kInvOddDf[m].lo);  // one rounding of y (hi + lo)
            }
        }
    } else {
        // rsqrtf refined by one Newton step, sqrt(pi)/2 as hi + lo
        const float r0 = rsqrtf(T);
        const float r = fmaf(0.5f * r0, fmaf(-T * r0, r0, 1.0f), r0);
        F[0] = fmaf(r, 0.886226952f, r * -2.66231996e-08f);
        const float h = 0.5f * r * r;
#pragma unroll
        for (int m = 0; m < L; ++m) F[m + 1] = F[m] * ((2 * m + 1) * h);
    }
}

// Double-float evaluation (the double-float quartets of a mixed build): the
// FP64 table's values split into hi + lo, the same Taylor series, downward
// recursion and asymptotic form, every operation on the FP32 pipe.
template <int L>
__device__ __forceinline__ void boys_df(dfl T, dfl* F, const float2* __restrict__ tab) {
    if (T.hi < (float)kBoysTmax) {
        const int k = __float2int_rn(T.hi * kBoysPerUnit);
        const dfl d = dfl(k * (1.0f / kBoysPerUnit)) - T;  // the grid point is exact in FP32
        const float2* c = tab + ((size_t)k * kBoysRows + L) * kBoysTaylor;
        float2 cv = __ldg(c + kBoysTaylor - 1);
        dfl f(cv.x, cv.y);
#pragma unroll
        for (int j = kBoysTaylor - 2; j >= 0; --j) { cv = __ldg(c + j); f = fma(f, d, dfl(cv.x, cv.y)); }
        F[L] = f;
        if (L > 0) {
            const float2* e = tab + ((size_t)k * kBoysRows + kLmaxBoys + 1) * kBoysTaylor;
            cv = __ldg(e + kBoysTaylor - 1);
            dfl eT(cv.x, cv.y);
#pragma unroll
            for (int j = kBoysTaylor - 2; j >= 0; --j) { cv = __ldg(e + j); eT = fma(eT, d, dfl(cv.x, cv.y)); }
            const dfl t2 = T + T;
#pragma unroll
            for (int m = L - 1; m >= 0; --m) F[m] = fma(t2, F[m + 1], eT) * kInvOddDf[m];
        }
    } else {
        const dfl r = df_rsqrt(T);
        F[0] = r * dfl(0.886226952f, -2.66231996e-08f);  // sqrt(pi)/2 / sqrt(T), hi + lo
        const dfl h = (r * r) * 0.5f;                 // 1 / (2T)
#pragma unroll
        for (int m = 0; m < L; ++m) F[m + 1] = F[m] * (h * (float)(2 * m + 1));
    }
}

// Mixed precision: FP64 evaluation below tsmall, FP32 above.
template <int L>
__device__ __forceinline__ void boys_mixed(float T, float* F, const double* __restrict__ tab,
                                           const float* __restrict__ tabf, float tsmall) {
    if (T < tsmall) {
        double Fd[L + 1];
        boys_f64<L>((double)T, Fd, tab);
#pragma unroll
        for (int m = 0; m <= L; ++m) F[m] = (float)Fd[m];
    } else {
        boys_f32<L>(T, F, tabf);
    }
}

// ------------------------------------------------------------------ rows
// Row r of work item t (the largest r with start[r] <= t < start[nrows]) and
// the item's offset li = t - start[r] inside the row.
__device__ __forceinline__ void locate_row(const RowsView& rv, long long t, int& row, long long& li) {
    int lo = 0, hi = rv.nrows;  // invariant: start[lo] <= t < start[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(rv.start + mid) <= t) lo = mid; else hi = mid;
    }
    row = lo;
    li = t - __ldg(rv.start + lo);
}

// ------------------------------------------------------------------ digestion
// One J'/K' update.  FP64 builds pass lo arrays and accumulate with
// compensation: the value is split into vh, a multiple of 2^-32 (round to
// nearest through v + C - C with C = 1.5 * 2^20), and the exact remainder
// v - vh (|v - vh| <= 2^-33).  The multiples add up in X without rounding as
// long as every partial sum stays below 2^21 in magnitude; the remainders add
// up in lo with a rounding error below 1e-25 per update.  X + lo is then the
// sum of the updates to about 1e-20, whatever order the atomics land in
// (plain FP64 atomics round every update to the element's ulp, and 1e6 updates
// of an element of size 4 can drift by 1e-10).  Mixed builds (lo null) and
// FP32 quartets add plainly.
constexpr double kSplitC = 1572864.0;  // 1.5 * 2^20: ulp 2^-32

template <class R>
__device__ __forceinline__ void jk_add(double* X, double* lo, size_t i, double v) {
    if constexpr (std::is_same<R, double>::value) {
        if (lo) {
            const double vh = __dsub_rn(__dadd_rn(v, kSplitC), kSplitC);
            atomicAdd(X + i, vh);
            atomicAdd(lo + i, __dsub_rn(v, vh));
            return;
        }
    }
    atomicAdd(X + i, v);
}

// Warp-level pre-reduction of the digestion (FP32 kernels).  The lanes of a
// warp hold consecutive work items: the items of one row share the bra pair
// (its J'_ab targets), and the items of one shell quartet split over bra
// primitive pairs share all of its targets.  Both form contiguous runs of
// lanes; a run's sum is formed with shuffles and added to J or K by its first
// lane -- one atomic (and one FP32 -> FP64 conversion) per run instead of one
// per lane.  Lanes past the end of the work (the last iteration) take part
// with zero values and keys of their own, and add nothing.
#ifndef GB_WARP_SIZE
#define GB_WARP_SIZE 32
#endif
struct WarpSeg {
    unsigned rmask, qmask;  // bit o set: lane + o is in this lane's row / quartet run
    bool rhead, qhead;      // this lane is the first of its run
    bool act;               // this lane holds a real work item
};

__device__ __forceinline__ WarpSeg warp_seg(unsigned rkey, unsigned qkey, bool act) {
    WarpSeg w;
    const unsigned lane = threadIdx.x & (GB_WARP_SIZE - 1);
    w.rmask = 0;
    w.qmask = 0;
    w.act = act;
#pragma unroll
    for (int o = 1; o < GB_WARP_SIZE; o <<= 1) {
        const unsigned r2 = __shfl_down_sync(0xffffffffu, rkey, o);
        const unsigned q2 = __shfl_down_sync(0xffffffffu, qkey, o);
        if (lane + o < GB_WARP_SIZE) {
            if (r2 == rkey) w.rmask |= o;
            if (q2 == qkey) w.qmask |= o;
        }
    }
    const unsigned rp = __shfl_up_sync(0xffffffffu, rkey, 1), qp = __shfl_up_sync(0xffffffffu, qkey, 1);
    w.rhead = lane == 0 || rp != rkey;
    w.qhead = lane == 0 || qp != qkey;
    return w;
}

// Sum of v over this lane's run (complete at the run's first lane): tree
// steps 1, 2, 4, ... add the partial of lane + o while it is in the same run.
template <class T>
__device__ __forceinline__ T run_sum(T v, unsigned mask) {
#pragma unroll
    for (int o = 1; o < GB_WARP_SIZE; o <<= 1) {
        const T u = __shfl_down_sync(0xffffffffu, v, o);
        if (mask & o) v += u;
    }
    return v;
}

// One digestion target: reduced over the row run (row) or the quartet run
// when W is set, then added by the run's first lane.
template <class R, bool W>
__device__ __forceinline__ void jk_put(double* X, double* lo, size_t i, R v, const WarpSeg& ws, bool row) {
    if constexpr (W) {
        v = run_sum(v, row ? ws.rmask : ws.qmask);
        if (!ws.act || !(row ? ws.rhead : ws.qhead)) return;
    }
    jk_add<R>(X, lo, i, (double)v);
}

// Fused J/K update of one unique shell quartet (ab|cd), acc[((a*NB+b)*NC+c)*ND+d],
// already scaled by the degeneracy factor s.  With the eight permutational
// images and a symmetric D,
//   J'_ab += 2 sum_cd I D_cd,   J'_cd += 2 sum_ab I D_ab,
//   K'_ac += sum_bd I D_bd,     K'_ad += sum_bc I D_bc,
//   K'_bc += sum_ad I D_ad,     K'_bd += sum_ac I D_ac,
// and J = J' + J'^T, K = K' + K'^T afterwards.
// R is the arithmetic type of the block and of the density copy (double for
// FP64 quartets; float for FP32 quartets, whose sums are added to J and K
// in FP64 by the atomics).
template <int NA, int NB, int NC, int ND, class R, bool WR = false, bool WQ = false>
__device__ __forceinline__ void digest(const R* acc, int fa, int fb, int fc, int fd,
                                       const R* __restrict__ D, double* J, double* K, double* Jlo,
                                       double* Klo, int n,
                                       const WarpSeg& ws = WarpSeg()) {
    // J'_ab
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            R v = 0;
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int d = 0; d < ND; ++d)
                    v = fma(acc[((a * NB + b) * NC + c) * ND + d], ldg(D + (size_t)(fc + c) * n + fd + d), v);
            jk_put<R, WR>(J, Jlo, (size_t)(fa + a) * n + fb + b, v + v, ws, true);
        }
    // J'_cd
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            R v = 0;
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int b = 0; b < NB; ++b)
                    v = fma(acc[((a * NB + b) * NC + c) * ND + d], ldg(D + (size_t)(fa + a) * n + fb + b), v);
            jk_put<R, WQ>(J, Jlo, (size_t)(fc + c) * n + fd + d, v + v, ws, false);
        }
    // K'_ac and K'_ad
#pragma unroll
    for (int a = 0; a < NA; ++a) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            R v = 0;
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int d = 0; d < ND; ++d)
                    v = fma(acc[((a * NB + b) * NC + c) * ND + d], ldg(D + (size_t)(fb + b) * n + fd + d), v);
            jk_put<R, WQ>(K, Klo, (size_t)(fa + a) * n + fc + c, v, ws, false);
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            R v = 0;
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    v = fma(acc[((a * NB + b) * NC + c) * ND + d], ldg(D + (size_t)(fb + b) * n + fc + c), v);
            jk_put<R, WQ>(K, Klo, (size_t)(fa + a) * n + fd + d, v, ws, false);
        }
    }
    // K'_bc and K'_bd
#pragma unroll
    for (int b = 0; b < NB; ++b) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            R v = 0;
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int d = 0; d < ND; ++d)
                    v = fma(acc[((a * NB + b) * NC + c) * ND + d], ldg(D + (size_t)(fa + a) * n + fd + d), v);
            jk_put<R, WQ>(K, Klo, (size_t)(fb + b) * n + fc + c, v, ws, false);
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            R v = 0;
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    v = fma(acc[((a * NB + b) * NC + c) * ND + d], ldg(D + (size_t)(fa + a) * n + fc + c), v);
            jk_put<R, WQ>(K, Klo, (size_t)(fb + b) * n + fd + d, v, ws, false);
        }
    }
}

// The update of `digest` restricted to the ket components c in [C0, C1) of a
// quartet: acc[(ab * NCR + (c - C0)) * ND + d], NCR = C1 - C0 (the FP32
// kernels of the large classes compute a quartet's block one c range per
// launch; the ranges' updates add up to the full one).
template <int NA, int NB, int NC, int ND, int C0, int C1, class R, bool WR = false, bool WQ = false>
__device__ __forceinline__ void digest_crange(const R* acc, int fa, int fb, int fc, int fd,
                                              const R* __restrict__ D, double* J, double* K, double* Jlo,
                                       double* Klo, int n,
                                       const WarpSeg& ws = WarpSeg()) {
    constexpr int NCR = C1 - C0;
#define GB_ACC(a, b, c, d) acc[(((a) * NB + (b)) * NCR + ((c) - C0)) * ND + (d)]
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) {  // J'_ab
            R v = 0;
#pragma unroll
            for (int c = C0; c < C1; ++c)
#pragma unroll
                for (int d = 0; d < ND; ++d) v = fma(GB_ACC(a, b, c, d), ldg(D + (size_t)(fc + c) * n + fd + d), v);
            jk_put<R, WR>(J, Jlo, (size_t)(fa + a) * n + fb + b, v + v, ws, true);
        }
#pragma unroll
    for (int c = C0; c < C1; ++c)
#pragma unroll
        for (int d = 0; d < ND; ++d) {  // J'_cd
            R v = 0;
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int b = 0; b < NB; ++b) v = fma(GB_ACC(a, b, c, d), ldg(D + (size_t)(fa + a) * n + fb + b), v);
            jk_put<R, WQ>(J, Jlo, (size_t)(fc + c) * n + fd + d, v + v, ws, false);
        }
#pragma unroll
    for (int a = 0; a < NA; ++a) {
#pragma unroll
        for (int c = C0; c < C1; ++c) {  // K'_ac
            R v = 0;
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int d = 0; d < ND; ++d) v = fma(GB_ACC(a, b, c, d), ldg(D + (size_t)(fb + b) * n + fd + d), v);
            jk_put<R, WQ>(K, Klo, (size_t)(fa + a) * n + fc + c, v, ws, false);
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) {  // K'_ad
            R v = 0;
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int c = C0; c < C1; ++c) v = fma(GB_ACC(a, b, c, d), ldg(D + (size_t)(fb + b) * n + fc + c), v);
            jk_put<R, WQ>(K, Klo, (size_t)(fa + a) * n + fd + d, v, ws, false);
        }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
#pragma unroll
        for (int c = C0; c < C1; ++c) {  // K'_bc
            R v = 0;
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int d = 0; d < ND; ++d) v = fma(GB_ACC(a, b, c, d), ldg(D + (size_t)(fa + a) * n + fd + d), v);
            jk_put<R, WQ>(K, Klo, (size_t)(fb + b) * n + fc + c, v, ws, false);
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) {  // K'_bd
            R v = 0;
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int c = C0; c < C1; ++c) v = fma(GB_ACC(a, b, c, d), ldg(D + (size_t)(fa + a) * n + fc + c), v);
            jk_put<R, WQ>(K, Klo, (size_t)(fb + b) * n + fd + d, v, ws, false);
        }
    }
#undef GB_ACC
}


// Same update with rolled loops (large classes: bounded code size; the block
// lives in local memory there anyway).
template <int NA, int NB, int NC, int ND, class R>
__device__ __forceinline__ void digest_loop(const R* acc, int fa, int fb, int fc, int fd,
                                            const R* __restrict__ D, double* J, double* K, double* Jlo,
                                       double* Klo, int n) {
#pragma unroll 1
    for (int ab = 0; ab < NA * NB; ++ab) {
        const int a = ab / NB, b = ab % NB;
        R v = 0;
        for (int cd = 0; cd < NC * ND; ++cd)
            v = fma(acc[ab * NC * ND + cd], ldg(D + (size_t)(fc + cd / ND) * n + fd + cd % ND), v);
        jk_add<R>(J, Jlo, (size_t)(fa + a) * n + fb + b, (double)(v + v));
    }
#pragma unroll 1
    for (int cd = 0; cd < NC * ND; ++cd) {
        const int c = cd / ND, d = cd % ND;
        R v = 0;
        for (int ab = 0; ab < NA * NB; ++ab)
            v = fma(acc[ab * NC * ND + cd], ldg(D + (size_t)(fa + ab / NB) * n + fb + ab % NB), v);
        jk_add<R>(J, Jlo, (size_t)(fc + c) * n + fd + d, (double)(v + v));
    }
#pragma unroll 1
    for (int a = 0; a < NA; ++a)
#pragma unroll 1
        for (int c = 0; c < NC; ++c) {
            R vac = 0;
            for (int b = 0; b < NB; ++b)
                for (int d = 0; d < ND; ++d)
                    vac = fma(acc[((a * NB + b) * NC + c) * ND + d], ldg(D + (size_t)(fb + b) * n + fd + d), vac);
            jk_add<R>(K, Klo, (size_t)(fa + a) * n + fc + c, (double)vac);
        }
#pragma unroll 1
    for (int a = 0; a < NA; ++a)
#pragma unroll 1
        for (int d = 0; d < ND; ++d) {
            R v = 0;
            for (int b = 0; b < NB; ++b)
                for (int c = 0; c < NC; ++c)
                    v = fma(acc[((a * NB + b) * NC + c) * ND + d], ldg(D + (size_t)(fb + b) * n + fc + c), v);
            jk_add<R>(K, Klo, (size_t)(fa + a) * n + fd + d, (double)v);
        }
#pragma unroll 1
    for (int b = 0; b < NB; ++b)
#pragma unroll 1
        for (int c = 0; c < NC; ++c) {
            R v = 0;
            for (int a = 0; a < NA; ++a)
                for (int d = 0; d < ND; ++d)
                    v = fma(acc[((a * NB + b) * NC + c) * ND + d], ldg(D + (size_t)(fa + a) * n + fd + d), v);
            jk_add<R>(K, Klo, (size_t)(fb + b) * n + fc + c, (double)v);
        }
#pragma unroll 1
    for (int b = 0; b < NB; ++b)
#pragma unroll 1
        for (int d = 0; d < ND; ++d) {
            R v = 0;
            for (int a = 0; a < NA; ++a)
                for (int c = 0; c < NC; ++c)
                    v = fma(acc[((a * NB + b) * NC + c) * ND + d], ldg(D + (size_t)(fa + a) * n + fc + c), v);
            jk_add<R>(K, Klo, (size_t)(fb + b) * n + fd + d, (double)v);
        }
}

// J/K update of the part of one unique shell quartet that has ket component
// c = ci (classes computed one ket-component chunk per thread):
// acc[(a*NB+b)*ND+d] = s (ab|ci d).  The same six updates as `digest`,
// restricted to that c; the chunks of a quartet add up to the full update.
template <int NA, int NB, int NC, int ND, class R>
__device__ __forceinline__ void digest_chunk(const R* acc, int ci, int fa, int fb, int fc, int fd,
                                             const R* __restrict__ D, double* J, double* K, double* Jlo,
                                       double* Klo, int n) {
    const int c = fc + ci;
#pragma unroll 1
    for (int ab = 0; ab < NA * NB; ++ab) {  // J'_ab
        const int a = ab / NB, b = ab % NB;
        R v = 0;
        for (int d = 0; d < ND; ++d) v = fma(acc[ab * ND + d], ldg(D + (size_t)c * n + fd + d), v);
        jk_add<R>(J, Jlo, (size_t)(fa + a) * n + fb + b, (double)(v + v));
    }
#pragma unroll 1
    for (int d = 0; d < ND; ++d) {  // J'_cd
        R v = 0;
        for (int ab = 0; ab < NA * NB; ++ab)
            v = fma(acc[ab * ND + d], ldg(D + (size_t)(fa + ab / NB) * n + fb + ab % NB), v);
        jk_add<R>(J, Jlo, (size_t)c * n + fd + d, (double)(v + v));
    }
#pragma unroll 1
    for (int a = 0; a < NA; ++a) {
        R vac = 0;  // K'_ac
        for (int b = 0; b < NB; ++b)
            for (int d = 0; d < ND; ++d)
                vac = fma(acc[(a * NB + b) * ND + d], ldg(D + (size_t)(fb + b) * n + fd + d), vac);
        jk_add<R>(K, Klo, (size_t)(fa + a) * n + c, (double)vac);
        for (int d = 0; d < ND; ++d) {  // K'_ad
            R v = 0;
            for (int b = 0; b < NB; ++b) v = fma(acc[(a * NB + b) * ND + d], ldg(D + (size_t)(fb + b) * n + c), v);
            jk_add<R>(K, Klo, (size_t)(fa + a) * n + fd + d, (double)v);
        }
    }
#pragma unroll 1
    for (int b = 0; b < NB; ++b) {
        R vbc = 0;  // K'_bc
        for (int a = 0; a < NA; ++a)
            for (int d = 0; d < ND; ++d)
                vbc = fma(acc[(a * NB + b) * ND + d], ldg(D + (size_t)(fa + a) * n + fd + d), vbc);
        jk_add<R>(K, Klo, (size_t)(fb + b) * n + c, (double)vbc);
        for (int d = 0; d < ND; ++d) {  // K'_bd
            R v = 0;
            for (int a = 0; a < NA; ++a) v = fma(acc[(a * NB + b) * ND + d], ldg(D + (size_t)(fa + a) * n + c), v);
            jk_add<R>(K, Klo, (size_t)(fb + b) * n + fd + d, (double)v);
        }
    }
}


}  // namespace gb
