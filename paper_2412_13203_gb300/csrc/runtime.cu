// Host runtime and C ABI of the screened-ERI / J-K library (include/gb300_eri.h).
//
// Everything on the data path runs in the kernels of this file, of the
// headers it includes (split_kernels.cuh: the mixed-precision split and
// density screening; sph_transform.cuh: the Cartesian <-> pure transform;
// one_electron.cuh: S, T, V) and of the generated per-class ERI and
// derivative kernels: coefficient normalisation, primitive Gaussian
// products, Schwarz factors, the pair sort, the quartet-row enumeration, J/K
// digestion, symmetrisation and the energy reduction.  The host only
// validates arguments, sizes launches and reads back a few counts.
//
// Paper mapping (arXiv 2412.13203):
//   Block Constructor stage 1 (Sec. 4): every basis-function pair, sorted by
//     angular class, cut into class-uniform tiles  -> pair build + sort here,
//     the tile key additionally carries the primitive-pair count (bucketed)
//     and the Schwarz factor so every warp runs one class with uniform loops.
//   Block Constructor stage 2 (Sec. 4): pair tile x pair tile quartet blocks,
//     never stored as O(N^4) lists -> "rows" (bra pair, ket bucket prefix),
//     O(N^2) memory, one launch per (bra class, ket class).
//   Workload Allocator atomics (Sec. 6) -> fused J/K digestion with FP64
//     atomics in the generated kernels.
#include <cuda_runtime.h>
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "eri_device.cuh"
#include "gb300_eri.h"
#include "sph_transform.cuh"
#include "one_electron.cuh"

int gb_launch_jk(int bra_cls, int ket_cls, int prec, const gb::JKArgs& a, int grid, int block, cudaStream_t s);
int gb_launch_schwarz(int cls, const gb::SchwarzArgs& a, cudaStream_t s);
int gb_class_flops(int bra_cls, int ket_cls, int* per_primq, int* per_brap);
int gb_launch_grad(int bra_cls, int ket_cls, int prec, const gb::GradArgs& a, int grid, cudaStream_t s);
int gb_grad_threads(int bra_cls, int ket_cls);
int gb_grad_lmax();
int gb_class_threads(int bra_cls, int ket_cls, int prec);
int gb_class_split(int bra_cls, int ket_cls);
extern "C" int gb_num_pair_classes();
extern "C" int gb_sph_table(const double** coef, const int** off);

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

// Fault injection (JK_OPT_FAIL_ALLOC_AFTER): the number of device
// allocations that still succeed before one fails as if the device were out
// of memory; negative: off.
std::atomic<long long> g_fail_alloc{-1};

#define CK(x)                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess) return fail(JK_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CKL()                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = cudaGetLastError();                                                      \
        if (e_ != cudaSuccess) return fail(JK_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
    } while (0)

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    int alloc(size_t n) {
        if (n <= bytes && p) return 0;
        release();
        if (n == 0) n = 16;
        if (g_fail_alloc.load() >= 0 && g_fail_alloc.fetch_sub(1) <= 0) {
            g_fail_alloc.store(0);
            return fail(JK_ERR_NOMEM, "injected allocation failure (" + std::to_string(n) + " bytes)");
        }
        if (cudaMalloc(&p, n) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(JK_ERR_NOMEM, "cudaMalloc of " + std::to_string(n) + " bytes failed");
        }
        bytes = n;
        return 0;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

constexpr int kMaxClasses = 10;  // pair classes for l <= 3
constexpr int kSplitSlots = 8;   // per class: FP32 q, FP64 q, FP32/FP64/demoted item totals, list totals
constexpr int kNB = 128;         // primitive-pair-count buckets (exact count, 128+ share the last)

struct TuneCfg {
    int block = 128;  // threads per block (kernels are compiled for <= 128)
    int qpt = 1;      // quartets per thread
};

struct ClassRows {
    int bra_cls = 0, ket_cls = 0;
    int nrows = 0;
    long long total = 0;
    long long nprimq = 0;
    long long nbrap = 0;
    DevBuf start, bra, ket0;
    DevBuf istart;      // prefix of work items per row (a quartet splits into gb::item_split(P, K_ab) items)
    long long itotal = 0;
    // mixed-precision split (filled on the device by jk_build).  Per row: the
    // kets of the global-bound FP64 prefix are listed explicitly -- FP64 ones
    // (c64 quartets, w64 items, item prefix s64, list offsets l64) and demoted
    // ones (cdem, wdem, sdem, ldem) -- and the FP32 suffix stays contiguous
    // (c32, w32, s32, ket starts k32).
    DevBuf s64, s32, k32, c64, c32, w64, w32, scr;
    DevBuf cdem, wdem, sdem, l64, ldem;
    TuneCfg tune[2];  // per precision (0 FP64 kernels, 1 FP32 kernels)
};

// Boys tables (one set per device, built on first use).
struct BoysTables {
    DevBuf tab, tabf, tabd;  // FP64, FP32, double-float (hi, lo of FP64)
    bool ready = false;
};
std::mutex g_boys_mu;
BoysTables g_boys[64];

struct Options {
    double tau = 5e-3;  // with the primitive split: J, K and E of the 32-atom workload and of the batch
                        // molecules measured within 3e-7 Eh of the FP64 build
    double eps = 0.0;  // density screening of mixed builds (0: off)
    double tsmall = 0.0;  // FP32 Boys everywhere in FP32 quartets (the FP64 branch buys no accuracy)
    int check_sym = 0;
    int graph = 1;
    int profile = 0;
    int rpath = 1;     // FP32 kernels of the classes emitted twice: Algorithm 1's R recursion order
    int df_tier = 0;   // mixed builds: the FP64-selected quartets in double-float arithmetic (off: FP64 is
                       // faster once the primitive split leaves only their large primitive quartets)
    double grad_tau = 3e-4;  // mixed gradient: FP32 derivative integrals iff the quartet's bound is below this
    double ptau = 1e-4;  // mixed builds: primitive quartets of the FP64 list below this bound run in FP32 (0: off)
    double grad_ptau = 1e-6;  // mixed gradient: the same split of its FP64 list (0: off)
} g_opt;

struct ProfRec {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int bra = 0, ket = 0, prec = 0;
    long long total = 0;
};

}  // namespace

struct jk_pairs_s {
    unsigned long long serial = 0;                  // unique per handle ever built (never reused)
    int device = 0;
    int natom = 0, nshell = 0, nbf = 0;
    long long npair_all = 0, npair = 0, nprimpair = 0;
    double thresh = 0.0, Qmax = 0.0;
    DevBuf info, A, B, pp, pp2, ppf, ppf2;          // sorted, kept pairs
    DevBuf Ahl;                                     // float4 x 2 per pair: centre of a as hi + lo floats
    DevBuf ppd;                                     // float4 x 5 per primitive pair: double-float data
    DevBuf pq;                                      // float per primitive pair: primitive Schwarz factor
    DevBuf Ddf;                                     // double-float copy of the last mixed build's D
    DevBuf Df;                                      // FP32 copy of the last mixed build's D
    DevBuf alpha;                                   // per primitive pair: exponent of the a primitive
    DevBuf pair_atoms;                              // int2 per pair: atoms of shells a, b
    DevBuf pair_sh;                                 // int2 per pair: shells a, b (caller's order)
    DevBuf bf_shell;                                // int per basis function: its shell
    DevBuf Dsh;                                     // float [nshell^2]: max |D| per shell block (mixed)
    DevBuf Jlo, Klo;                                // FP64 builds: remainders of the compensated J'/K' sums
    int part_n = 0;                                 // row partition cached for part_n parts (partial builds)
    std::vector<std::vector<int>> part_rows;        // per class: part_n + 1 row bounds
    std::vector<std::vector<long long>> part_items; // per class: work-item prefix (istart) at those bounds
    std::vector<std::vector<double>> part_cost;     // per class: algorithmic cost of every part, then the
                                                    // largest single-row cost of the class
    DevBuf list64, listdem;                         // mixed: FP64 and demoted (FP32) ket lists
    DevBuf thr64;                                   // mixed, primitive split: per FP64 list entry, its primitive cut
    bool last_psplit = false;                       // the last mixed build split its FP64 list by primitives
    std::vector<long long> list_off64, list_offd;   // per class: first entry in list64 / listdem
    std::vector<int> last_r0, last_r1;              // per class: rows of the last mixed build (partial builds)
    DevBuf pair_lab;                                // int2 per pair: la, lb
    DevBuf xyz;                                     // atoms
    std::vector<int> cls_start;                     // [ncls + 1] pair ranges per class
    std::vector<int> bucket_start;                  // [ncls * (kNB + 1)] per class bucket ranges
    std::vector<ClassRows> rows;
    long long nquartets = 0, nprimq = 0;
    long long last_n32 = 0, last_n64 = 0;
    long long launches = 0;
    int nsm = 152;
    int last_prec = 0;
    int tuned[2] = {0, 0};
    DevBuf split_tot;                               // per class: FP32, FP64 quartets, FP32, FP64 items (last mixed build)
    DevBuf npre;                                    // exclusive prefix of primitive pairs over the kept pairs
    DevBuf scratch;                                 // small reductions
    DevBuf charges;                                 // nuclear charges of the last jk_one_electron
    std::vector<int> shell_l;                       // host copy of every shell's l (caller's order)
    int nsph = 0;                                   // basis size with pure d and f shells
    DevBuf sph_shell;                               // int4 per shell: l, first Cartesian, first pure index, table offset
    DevBuf sph_owner;                               // int per pure basis function: its shell
    DevBuf sph_coef;                                // Cartesian-to-pure coefficient tables
    bool sph_ready = false;
    std::vector<ProfRec> prof;
    // forked streams of a build's class launches (created on first use, on the handle's device)
    cudaStream_t side[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[3] = {nullptr, nullptr, nullptr};
    ~jk_pairs_s() {
        for (auto& r : prof) {
            if (r.e0) cudaEventDestroy(r.e0);
            if (r.e1) cudaEventDestroy(r.e1);
        }
        for (auto& x : side) if (x) { cudaStreamSynchronize(x); cudaStreamDestroy(x); }
        if (fork) cudaEventDestroy(fork);
        for (auto& e : join) if (e) cudaEventDestroy(e);
    }
};

namespace {

// ------------------------------------------------------------------ Boys table build
// F_m(T_k) by its power series  F_m(T) = exp(-T) sum_i (2T)^i / ((2m+1)(2m+3)...(2m+2i+1)),
// summed with compensation; every term is positive.
__global__ void k_boys_raw(double* raw, int nm) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= gb::kBoysNgrid * nm) return;
    const int k = idx / nm, m = idx % nm;
    const double T = (double)k / gb::kBoysPerUnit;
    double term = 1.0 / (2 * m + 1), sum = term, comp = 0.0;
    for (int i = 1; i < 2000; ++i) {
        term *= 2.0 * T / (2 * m + 2 * i + 1);
        const double y = term - comp;
        const double t = sum + y;
        comp = (t - sum) - y;
        sum = t;
        if (term < 1e-18 * sum) break;
    }
    raw[idx] = exp(-T) * sum;
}

__global__ void k_boys_fill(const double* raw, int nm, double* tab, float* tabf, float2* tabd) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int per = gb::kBoysRows * gb::kBoysTaylor;
    if (idx >= gb::kBoysNgrid * per) return;
    const int k = idx / per, r = (idx / gb::kBoysTaylor) % gb::kBoysRows, j = idx % gb::kBoysTaylor;
    double fact = 1.0;
    for (int i = 2; i <= j; ++i) fact *= i;
    double v;
    if (r <= gb::kLmaxBoys) {
        v = raw[k * nm + r + j] / fact;
    } else {
        v = exp(-(double)k / gb::kBoysPerUnit) / fact;
    }
    tab[idx] = v;
    tabf[idx] = (float)v;
    tabd[idx] = make_float2((float)v, (float)(v - (double)(float)v));
    if (j == gb::kBoysLoSlot) {  // FP32 table: the low part of the row's leading term (unused slot)
        const double v0 = r <= gb::kLmaxBoys ? raw[k * nm + r] : exp(-(double)k / gb::kBoysPerUnit);
        tabf[idx] = (float)(v0 - (double)(float)v0);
    }
}

int ensure_boys(int dev, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_boys_mu);
    if (dev < 0 || dev >= 64) return fail(JK_ERR_INVALID, "device index");
    BoysTables& b = g_boys[dev];
    if (b.ready) return 0;
    const int nm = gb::kLmaxBoys + gb::kBoysTaylor;
    DevBuf raw;
    int rc;
    if ((rc = raw.alloc(sizeof(double) * gb::kBoysNgrid * nm))) return rc;
    const size_t n = (size_t)gb::kBoysNgrid * gb::kBoysRows * gb::kBoysTaylor;
    if ((rc = b.tab.alloc(sizeof(double) * n))) return rc;
    if ((rc = b.tabf.alloc(sizeof(float) * n))) return rc;
    if ((rc = b.tabd.alloc(sizeof(float2) * n))) return rc;
    k_boys_raw<<<(gb::kBoysNgrid * nm + 127) / 128, 128, 0, st>>>(raw.as<double>(), nm);
    CKL();
    k_boys_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(raw.as<double>(), nm, b.tab.as<double>(), b.tabf.as<float>(),
                                                            b.tabd.as<float2>());
    CKL();
    CK(cudaStreamSynchronize(st));
    b.ready = true;
    return 0;
}

// ------------------------------------------------------------------ scans and sorts
// Exclusive prefix sum of n int64 values (in place allowed), total written to *total.
__global__ void k_scan_block(const long long* in, long long* out, long long* bsum, long long n) {
    __shared__ long long s[1024];
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    const long long v = (i < n) ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        long long t = (threadIdx.x >= (unsigned)off) ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = s[1023];
}

__global__ void k_scan_add(long long* out, const long long* boff, long long n) {
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    if (i < n) out[i] += boff[blockIdx.x];
}

__global__ void k_set_total(const long long* in, const long long* out, long long n, long long* total) {
    *total = (n > 0) ? out[n - 1] + in[n - 1] : 0;
}

// Kernel launches scan_exclusive issues for n elements.
long long scan_launches(long long n) {
    if (n <= 0) return 0;
    const long long nb = (n + 1023) / 1024;
    return 2 + (nb > 1 ? 1 + scan_launches(nb) : 0);
}

// in == out is not allowed for the last-element total; callers keep the counts.
// long longs of scratch scan_into needs for n elements.
long long scan_scratch_len(long long n) {
    if (n <= 1024) return 0;
    const long long nb = (n + 1023) / 1024;
    return 2 * nb + 1 + scan_scratch_len(nb);
}

// Exclusive scan with caller-provided scratch (no allocation, no host sync).
int scan_into(const long long* in, long long* out, long long n, long long* total_dev, long long* scratch,
              cudaStream_t st) {
    if (n <= 0) {
        CK(cudaMemsetAsync(total_dev, 0, sizeof(long long), st));
        return 0;
    }
    const long long nb = (n + 1023) / 1024;
    long long* bsum = scratch;
    long long* boff = scratch + nb;
    long long* btot = scratch + 2 * nb;
    if (nb == 1) {
        // single block: its block sum slot is unused, use the total slot directly
        k_scan_block<<<1, 1024, 0, st>>>(in, out, total_dev, n);
        CKL();
    } else {
        k_scan_block<<<(unsigned)nb, 1024, 0, st>>>(in, out, bsum, n);
        CKL();
        int rc;
        if ((rc = scan_into(bsum, boff, nb, btot, scratch + 2 * nb + 1, st))) return rc;
        k_scan_add<<<(unsigned)nb, 1024, 0, st>>>(out, boff, n);
        CKL();
    }
    k_set_total<<<1, 1, 0, st>>>(in, out, n, total_dev);
    CKL();
    return 0;
}

// Exclusive scan with temporary scratch (synchronises before freeing it).
int scan_exclusive(const long long* in, long long* out, long long n, long long* total_dev, cudaStream_t st) {
    DevBuf tmp;
    int rc;
    if ((rc = tmp.alloc(sizeof(long long) * (scan_scratch_len(n) + 1)))) return rc;
    if ((rc = scan_into(in, out, n, total_dev, tmp.as<long long>(), st))) return rc;
    CK(cudaStreamSynchronize(st));
    return 0;
}

// Bitonic sort of (key, val) pairs, n a power of two.
__global__ void k_bitonic(unsigned long long* key, int* val, long long n, long long j, long long k) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long l = i ^ j;
    if (l <= i) return;
    const bool up = (i & k) == 0;
    const unsigned long long a = key[i], b = key[l];
    if ((a > b) == up) {
        key[i] = b; key[l] = a;
        const int t = val[i]; val[i] = val[l]; val[l] = t;
    }
}

int sort_pairs(unsigned long long* key, int* val, long long n, cudaStream_t st) {
    for (long long k = 2; k <= n; k <<= 1)
        for (long long j = k >> 1; j > 0; j >>= 1) {
            k_bitonic<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(key, val, n, j, k);
            CKL();
        }
    return 0;
}

// ------------------------------------------------------------------ pair build kernels
__global__ void k_normalize(int nshell, const int* l, const int* nprim, const int* off, const double* e,
                            const double* c, double* out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nshell) return;
    const int L = l[s], k = nprim[s], o = off[s];
    double dfact = 1.0;
    for (int i = 2 * L - 1; i > 1; i -= 2) dfact *= i;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < k; ++i) {
        const double a = e[o + i];
        out[o + i] = c[o + i] * pow(2.0 * a / pi, 0.75) * pow(4.0 * a, 0.5 * L) / sqrt(dfact);
    }
    double S = 0.0;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            const double p = e[o + i] + e[o + j];
            S += out[o + i] * out[o + j] * pow(pi / p, 1.5) * dfact / pow(2.0 * p, L);
        }
    const double f = rsqrt(S);
    for (int i = 0; i < k; ++i) out[o + i] *= f;
}

struct ShellDev {
    const int *atom, *l, *nprim, *off, *bf;
    const double *e, *c, *xyz;
};

__device__ __forceinline__ void decode_pair(long long k, int& i, int& j) {
    long long ii = (long long)((sqrt(8.0 * (double)k + 1.0) - 1.0) * 0.5);
    while (ii * (ii + 1) / 2 > k) --ii;
    while ((ii + 1) * (ii + 2) / 2 <= k) ++ii;
    i = (int)ii;
    j = (int)(k - ii * (ii + 1) / 2);
}

__device__ __forceinline__ void canon(const ShellDev& S, int i, int j, int& a, int& b) {
    // a carries the larger angular momentum (ties: the larger shell index)
    if (S.l[j] > S.l[i]) { a = j; b = i; } else { a = i; b = j; }
}

__global__ void k_pair_count(ShellDev S, long long npair, long long* nprimpair, unsigned long long* key, int* val,
                             long long npad) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npad) return;
    if (k >= npair) {
        key[k] = ~0ull;
        val[k] = -1;
        return;
    }
    int i, j, a, b;
    decode_pair(k, i, j);
    canon(S, i, j, a, b);
    nprimpair[k] = (long long)S.nprim[a] * S.nprim[b];
    const int la = S.l[a], lb = S.l[b];
    const unsigned long long cls = (unsigned long long)(la * (la + 1) / 2 + lb);
    key[k] = (cls << 40) | (unsigned long long)k;
    val[k] = (int)k;
}

__global__ void k_pair_fill(ShellDev S, long long npair, const long long* poff, int4* info, double4* A, double4* B,
                            int2* atoms, int2* lab, double4* pp, double2* pp2, float4* ppf, float4* ppf2, float4* ppd,
                            double* alpha, int2* sh) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npair) return;
    int i, j, a, b;
    decode_pair(k, i, j);
    canon(S, i, j, a, b);
    const double* Ra = S.xyz + 3 * S.atom[a];
    const double* Rb = S.xyz + 3 * S.atom[b];
    const double ABx = Ra[0] - Rb[0], ABy = Ra[1] - Rb[1], ABz = Ra[2] - Rb[2];
    const double AB2 = ABx * ABx + ABy * ABy + ABz * ABz;
    const int ka = S.nprim[a], kb = S.nprim[b];
    const long long o = poff[k];
    info[k] = make_int4(S.bf[a], S.bf[b], ka * kb, (int)o);
    A[k] = make_double4(Ra[0], Ra[1], Ra[2], 0.0);
    B[k] = make_double4(Rb[0], Rb[1], Rb[2], 0.0);
    atoms[k] = make_int2(S.atom[a], S.atom[b]);
    lab[k] = make_int2(S.l[a], S.l[b]);
    sh[k] = make_int2(a, b);
    const double s2pi52 = 5.9149671727956128778;  // sqrt(2 pi^(5/2))
    int n = 0;
    for (int u = 0; u < ka; ++u)
        for (int v = 0; v < kb; ++v, ++n) {
            const double al = S.e[S.off[a] + u], be = S.e[S.off[b] + v];
            const double p = al + be, ip = 1.0 / p;
            const double Kab = exp(-al * be * ip * AB2);
            const double kap = s2pi52 * Kab * S.c[S.off[a] + u] * S.c[S.off[b] + v] * ip;
            pp[o + n] = make_double4((al * Ra[0] + be * Rb[0]) * ip, (al * Ra[1] + be * Rb[1]) * ip,
                                     (al * Ra[2] + be * Rb[2]) * ip, p);
            pp2[o + n] = make_double2(kap, 0.5 * ip);
            // FP32 data: P - A = -(beta/p)(A - B), P - B = (alpha/p)(A - B), each rounded once
            const double fa = -be * ip, fb = al * ip;
            ppf[o + n] = make_float4((float)(fa * ABx), (float)(fa * ABy), (float)(fa * ABz), (float)p);
            ppf2[o + n] = make_float4((float)(fb * ABx), (float)(fb * ABy), (float)(fb * ABz), (float)kap);
            // double-float data: every value as hi + lo floats (P - A, P - B, p, kappa, 1/2p)
            const double dv[9] = {fa * ABx, fa * ABy, fa * ABz, fb * ABx, fb * ABy, fb * ABz, p, kap, 0.5 * ip};
            float hl[20];
            for (int t = 0; t < 9; ++t) { hl[2 * t] = (float)dv[t]; hl[2 * t + 1] = (float)(dv[t] - (double)hl[2 * t]); }
            hl[18] = 0.f;
            hl[19] = 0.f;
            float4* dst = ppd + 5 * (o + n);
            for (int t = 0; t < 5; ++t) dst[t] = make_float4(hl[4 * t], hl[4 * t + 1], hl[4 * t + 2], hl[4 * t + 3]);
            alpha[o + n] = al;
        }
}

template <class T>
__global__ void k_gather(const T* src, const int* perm, T* dst, long long n) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dst[k] = src[perm[k]];
}

__global__ void k_class_bounds(const unsigned long long* key, long long n, int shift, int mask, int* start) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int c = (int)((key[k] >> shift) & mask);
    const int cp = (k == 0) ? -1 : (int)((key[k - 1] >> shift) & mask);
    if (c != cp) start[c] = (int)k;
}

// Q_i = sqrt(max_d |sum_p diag[i][p][d]|) from the Schwarz kernels' partial
// diagonals, the parts added in a fixed order (Q does not depend on scheduling).
__global__ void k_schwarz_finish(const double* diag, int nab, int count, double* Q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double m = 0.0;
    for (int d = 0; d < nab; ++d) {
        double v = 0.0;
        for (int p = 0; p < gb::kSchwarzSplit; ++p) v += diag[((size_t)i * gb::kSchwarzSplit + p) * nab + d];
        m = fmax(m, fabs(v));
    }
    Q[i] = sqrt(m);
}

// Q_ab into A.w; maximum Q via integer atomics on the (non-negative) bit pattern.
__global__ void k_store_q(const double* Q, int first, int count, double4* A, unsigned long long* qmax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double q = Q[i];
    A[first + i].w = q;
    atomicMax(qmax, (unsigned long long)__double_as_longlong(q));
}

// Exact primitive-pair count: kets of one bucket have the same trip count, so
// the lanes of a warp working on one quartet row loop in step.
__device__ __forceinline__ int bucket_of(int np) { return min(np, kNB) - 1; }

// Final key: class (4 bits) | bucket (7 bits) | descending Q (53 bits); Q quantised
// (10 low mantissa bits cleared) so that the stored Q and the sort order agree.
__global__ void k_final_key(const double4* A, const int4* info, const int2* lab, long long n, double thresh,
                            double qmax, unsigned long long* key, int* val, long long npad) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npad) return;
    if (k >= n) { key[k] = ~0ull; val[k] = -1; return; }
    const double q = A[k].w;
    const int2 l = lab[k];
    const unsigned long long cls = (unsigned long long)(l.x * (l.x + 1) / 2 + l.y);
    const unsigned long long bk = (unsigned long long)bucket_of(info[k].z);
    const unsigned long long qb = ((unsigned long long)__double_as_longlong(q)) >> 10;  // 53 bits (q > 0)
    if (thresh > 0.0 && q * qmax < thresh) { key[k] = ~0ull; val[k] = (int)k; return; }
    key[k] = (cls << 60) | (bk << 53) | ((~qb) & ((1ull << 53) - 1));
    val[k] = (int)k;
}

// Centre of a of every pair as two floats per coordinate (hi, lo = A - hi).
__global__ void k_centres_hl(const double4* A, long long n, float4* hl) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double4 a = A[k];
    const float hx = (float)a.x, hy = (float)a.y, hz = (float)a.z;
    hl[2 * k] = make_float4(hx, hy, hz, 0.f);
    hl[2 * k + 1] = make_float4((float)(a.x - hx), (float)(a.y - hy), (float)(a.z - hz), 0.f);
}

__global__ void k_quantise_q(double4* A, long long n) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const unsigned long long b = (unsigned long long)__double_as_longlong(A[k].w);
    A[k].w = __longlong_as_double((long long)((b >> 10) << 10));
}

__global__ void k_count_kept(const unsigned long long* key, long long n, unsigned long long* cnt) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n && key[k] != ~0ull) atomicAdd(cnt, 1ull);
}

__global__ void k_bucket_bounds(const unsigned long long* key, long long n, int* start) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int c = (int)(key[k] >> 53);  // class * kNB + bucket
    const int cp = (k == 0) ? -1 : (int)(key[k - 1] >> 53);
    if (c != cp) start[c] = (int)k;
}

// Rows of one (bra class X, ket class Y) block: row r = bucket slot * nX + (i - x0).
// Count = kets of the bucket with Q_j >= thresh / Q_i (kets sorted by Q descending),
// capped at j <= i when X == Y (unique quartets ab >= cd).
__global__ void k_rows_count(const double4* A, int x0, int nX, const int* bseg /* [nb][2] */, int nb, bool same,
                             double thresh, long long* cnt, int* rbra, int* rket0) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (long long)nX * nb) return;
    const int bi = (int)(r / nX);
    const int i = x0 + (int)(r % nX);
    const int s = bseg[2 * bi], e = bseg[2 * bi + 1];
    int n;
    if (thresh > 0.0) {
        const double qi = A[i].w;
        int lo = s, hi = e;  // first j with Q_i Q_j < thresh
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (qi * A[mid].w >= thresh) lo = mid + 1; else hi = mid;
        }
        n = lo - s;
    } else {
        n = e - s;
    }
    if (same) {
        if (i < s) n = 0;
        else n = min(n, i - s + 1);
    }
    cnt[r] = n;
    rbra[r] = i;
    rket0[r] = s;
}

// Primitive quartets and (quartet x bra primitive pair) units of a class's
// rows, summed per warp before one atomic per warp into acc[0], acc[1].
__global__ void k_rows_primq(const long long* cnt, const int* rbra, const int* rket0, int nrows, const int4* info,
                             const long long* npre, unsigned long long* acc) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long pq = 0, bp = 0;
    if (r < nrows) {
        const long long c = cnt[r];
        if (c > 0) {
            const long long kab = info[rbra[r]].z;
            pq = (unsigned long long)((npre[rket0[r] + c] - npre[rket0[r]]) * kab);
            bp = (unsigned long long)(c * kab);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        pq += __shfl_xor_sync(0xffffffffu, pq, o);
        bp += __shfl_xor_sync(0xffffffffu, bp, o);
    }
    if ((threadIdx.x & 31) == 0 && (pq | bp)) {
        atomicAdd(acc, pq);
        atomicAdd(acc + 1, bp);
    }
}

// Algorithmic cost of every row: the generator's operation count of its
// primitive quartets (fq each) and of its (quartet x bra primitive pair)
// units (fb each); the weight of the row partition of partial builds.
__global__ void k_row_cost(const long long* start, const int* rbra, const int* rket0, int nrows, const int4* info,
                           const long long* npre, long long fq, long long fb, double* cost) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const long long c = start[r + 1] - start[r];
    const long long kab = info[rbra[r]].z;
    const long long kp = c > 0 ? npre[rket0[r] + c] - npre[rket0[r]] : 0;
    cost[r] = (double)(fq * kp * kab + fb * c * kab);
}

__global__ void k_np_of(const int4* info, long long n, long long* np) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) np[k] = info[k].z;
}

// One entry per primitive pair of the kept pairs (entry npre[i] + k for the
// k-th primitive pair of pair i): a one-primitive-pair view of its pair, on
// which the class's Schwarz kernel gives the primitive Schwarz factor.
__global__ void k_prim_expand(const int4* info, const double4* A, const double4* B, const long long* npre, long long n,
                              int4* finfo, double4* fA, double4* fB) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 ib = info[i];
    const long long o = npre[i];
    for (int k = 0; k < ib.z; ++k) {
        finfo[o + k] = make_int4(ib.x, ib.y, 1, ib.w + k);
        fA[o + k] = A[i];
        fB[o + k] = B[i];
    }
}

// The primitive pairs of every kept pair, sorted by primitive Schwarz factor
// (largest first, ties in their previous order), gathered into compact
// arrays at npre[i]; info[i].w is moved to the new first index.
__global__ void k_prim_sort(int4* info, const long long* npre, long long n, const double* q, const double4* pp,
                            const double2* pp2, const float4* ppf, const float4* ppf2, const float4* ppd,
                            const double* alpha, double4* pp_o, double2* pp2_o, float4* ppf_o, float4* ppf2_o,
                            float4* ppd_o, double* alpha_o, float* pq_o) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 ib = info[i];
    const long long o = npre[i];
    for (int k = 0; k < ib.z; ++k) {
        const double qk = q[o + k];
        int rank = 0;
        for (int j = 0; j < ib.z; ++j) {
            const double qj = q[o + j];
            rank += (qj > qk || (qj == qk && j < k)) ? 1 : 0;
        }
        const long long src = (long long)ib.w + k, dst = o + rank;
        pp_o[dst] = pp[src];
        pp2_o[dst] = pp2[src];
        ppf_o[dst] = ppf[src];
        ppf2_o[dst] = ppf2[src];
        for (int c = 0; c < 5; ++c) ppd_o[5 * dst + c] = ppd[5 * src + c];
        alpha_o[dst] = alpha[src];
        pq_o[dst] = (float)qk;
    }
    info[i].w = (int)o;
}

// Max |D| over every shell block (non-negative floats order like their bits).
__global__ void k_dsh(const double* D, int n, const int* bf_shell, int nshell, unsigned int* dsh) {
    const long long n2 = (long long)n * n;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n2; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / n), j = (int)(k - (long long)i * n);
        const float v = (float)fabs(D[k]);
        atomicMax(dsh + (size_t)bf_shell[i] * nshell + bf_shell[j], __float_as_uint(v));
    }
}

#include "split_kernels.cuh"

// Primitive quartets and (quartet x bra primitive pair) units of list rows.
__global__ void k_list_primq(const long long* cnt, const long long* ofs, const int* klist, const int* rbra, int nrows,
                             const int4* info, unsigned long long* acc) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const long long c = cnt[r];
    if (c == 0) return;
    long long kp = 0;
    for (long long k = 0; k < c; ++k) kp += info[klist[ofs[r] + k]].z;
    atomicAdd(acc, (unsigned long long)(kp * info[rbra[r]].z));
    atomicAdd(acc + 1, (unsigned long long)(c * info[rbra[r]].z));
}

// k_list_primq over a primitively split FP64 list: the primitive quartets and
// bra primitive-pair units of each listed quartet on either side of its cut
// (the same FP32 products as gb::prim_range), FP64 tier into acc64, the FP32
// complement into acc32.
__global__ void k_list_primq_split(const long long* cnt, const long long* ofs, const int* klist, const float* thr,
                                   const int* rbra, int nrows, const int4* info, const float* pq,
                                   unsigned long long* acc32, unsigned long long* acc64) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const long long c = cnt[r];
    if (c == 0) return;
    const int4 ib = info[rbra[r]];
    unsigned long long p64 = 0, u64 = 0, p32 = 0, u32 = 0;
    for (long long k = 0; k < c; ++k) {
        const int4 ik = info[klist[ofs[r] + k]];
        const float t = thr[ofs[r] + k];
        for (int ip = 0; ip < ib.z; ++ip) {
            int j0, j1;
            gb::prim_range(pq, ib.w + ip, ik.w, ik.z, t, 1, j0, j1);
            p64 += j1;
            u64 += j1 > 0;
            p32 += ik.z - j1;
            u32 += j1 < ik.z;
        }
    }
    atomicAdd(acc64, p64);
    atomicAdd(acc64 + 1, u64);
    atomicAdd(acc32, p32);
    atomicAdd(acc32 + 1, u32);
}

// Work items of every row: quartets x gb::item_split(P, K_ab) (bra primitive pairs of the
// row's bra pair; batched rows look the pair up in their molecule).
__global__ void k_row_items(const long long* start, const int* rbra, int nrows, const int4* info,
                            const gb::BatchMol* bm, const int* rowmol, int P, long long* w) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const int4* inf = bm ? bm[rowmol[r]].pairs.info : info;
    w[r] = (start[r + 1] - start[r]) * (long long)gb::item_split(P, inf[rbra[r]].z);
}

// max |x| (as the bit pattern of a non-negative double) and, if xf is not
// null, the FP32 copy of x used by the digestion of FP32 quartets.
__global__ void k_absmax(const double* x, long long n, unsigned long long* out, float* xf, float2* xd = nullptr) {
    double m = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        m = fmax(m, fabs(v));
        if (xf) xf[i] = (float)v;
        if (xd) xd[i] = make_float2((float)v, (float)(v - (double)(float)v));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// max |x - x^T| (bits of a non-negative double); a NaN or infinite element
// makes it NaN (sticky: NaN - anything is NaN, and the NaN bit pattern is
// above every finite one for the integer maximum).
__global__ void k_asym(const double* x, int n, unsigned long long* out) {
    double m = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)n * n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        const double d = fabs(x[(size_t)i * n + j] - x[(size_t)j * n + i]);
        if (isnan(d) || d > m) m = d;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double d = __shfl_xor_sync(0xffffffffu, m, o);
        if (isnan(d) || d > m) m = d;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(fabs(m)));
}

// J = J' + J'^T in place (one thread per unordered index pair).
__global__ void k_symmetrize(double* X, int n) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)n * (n + 1) / 2;
    if (t >= tot) return;
    int i, j;
    decode_pair(t, i, j);  // i >= j
    const size_t a = (size_t)i * n + j, b = (size_t)j * n + i;
    if (i == j) { X[a] *= 2.0; return; }
    const double v = X[a] + X[b];
    X[a] = v;
    X[b] = v;
}

// J = J' + J'^T in place for a compensated build: J' is X + lo (the exact
// multiples and the remainders of jk_add); the multiples of both triangles are
// added first (exactly, for sums below 2^21), then the remainders.
__global__ void k_symmetrize_lo(double* X, const double* lo, int n) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)n * (n + 1) / 2;
    if (t >= tot) return;
    int i, j;
    decode_pair(t, i, j);
    const size_t a = (size_t)i * n + j, b = (size_t)j * n + i;
    if (i == j) { X[a] = 2.0 * X[a] + 2.0 * lo[a]; return; }
    const double v = (X[a] + X[b]) + (lo[a] + lo[b]);
    X[a] = v;
    X[b] = v;
}

// Compensated energy: E = sum D J / 2 - sum D K / 4.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__global__ void k_energy_partial(const double* D, const double* J, const double* K, long long n2, double2* part) {
    double s = 0.0, c = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
        double t, e;
        two_sum(s, 0.5 * D[i] * J[i], t, e);
        s = t; c += e;
        two_sum(s, -0.25 * D[i] * K[i], t, e);
        s = t; c += e;
        // the products themselves carry rounding: add their exact residuals
        c += fma(0.5 * D[i], J[i], -(0.5 * D[i] * J[i]));
        c += fma(-0.25 * D[i], K[i], -(-0.25 * D[i] * K[i]));
    }
    __shared__ double ss[256], sc[256];
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < (unsigned)o) {
            double t, e;
            two_sum(ss[threadIdx.x], ss[threadIdx.x + o], t, e);
            ss[threadIdx.x] = t;
            sc[threadIdx.x] += sc[threadIdx.x + o] + e;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(ss[0], sc[0]);
}

__global__ void k_energy_final(const double2* part, int nb, double* E) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0, c = 0.0;
    for (int i = 0; i < nb; ++i) {
        double t, e;
        two_sum(s, part[i].x, t, e);
        s = t;
        c += e + part[i].y;
    }
    *E = s + c;
}

unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ------------------------------------------------------------------ allocation-free energy
// Scratch of jk_energy_noalloc: one compensated partial (sum, error) per row of
// D plus one slot for the result.  It is a fixed file-scope array, so every
// GPU that loads this library holds these 256 KiB until the process exits,
// and every call shares (and overwrites) it.
constexpr int kNoAllocMaxRows = 16383;
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocMaxRows + 1];
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {nullptr};

// Row partials: one warp per row of D, compensated (two-sum) accumulation of
// D J / 2 - D K / 4 including the rounding residuals of the products.
__global__ void k_energy_rows(const double* D, const double* J, const double* K, int n, double2* part) {
    const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;  // whole warps leave together
    double s = 0.0, c = 0.0;
    const size_t base = (size_t)row * n;
    for (int j = lane; j < n; j += 32) {
        const double d = D[base + j], a = 0.5 * d * J[base + j], b = -0.25 * d * K[base + j];
        double t, e;
        two_sum(s, a, t, e);
        s = t; c += e;
        two_sum(s, b, t, e);
        s = t; c += e;
        c += fma(0.5 * d, J[base + j], -a) + fma(-0.25 * d, K[base + j], -b);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
        double t, e;
        two_sum(s, s2, t, e);
        s = t;
        c += c2 + e;
    }
    if (lane == 0) part[row] = make_double2(s, c);
}

// Sum of the row partials (single block), result in out[0].x.
__global__ void k_energy_rows_final(const double2* part, int n, double2* out) {
    __shared__ double ss[256], sc[256];
    double s = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double t, e;
        two_sum(s, part[i].x, t, e);
        s = t;
        c += e + part[i].y;
    }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < (unsigned)o) {
            double t, e;
            two_sum(ss[threadIdx.x], ss[threadIdx.x + o], t, e);
            ss[threadIdx.x] = t;
            sc[threadIdx.x] += sc[threadIdx.x + o] + e;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = make_double2(ss[0] + sc[0], 0.0);
}

// Device address of the scratch array on the current device, looked up once
// per device (the array's name is only a host-side stand-in in host code).
int noalloc_scratch(double2** out) {
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(JK_ERR_INVALID, "device index");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(JK_ERR_CUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = static_cast<double2*>(g_noalloc_ptr[dev]);
    return 0;
}

// Cartesian components n_a n_b of a pair class (classes ss ps pp ds dp dd fs fp fd ff).
int pair_ncart(int cls) {
    int la = 0;
    while ((la + 1) * (la + 2) / 2 <= cls) ++la;
    const int lb = cls - la * (la + 1) / 2;
    return (la + 1) * (la + 2) / 2 * ((lb + 1) * (lb + 2) / 2);
}

gb::PairsView view_of(const jk_pairs_s* h) {
    gb::PairsView v;
    v.npair = (int)h->npair;
    v.info = h->info.as<int4>();
    v.A = h->A.as<double4>();
    v.B = h->B.as<double4>();
    v.pp = h->pp.as<double4>();
    v.pp2 = h->pp2.as<double2>();
    v.ppf = h->ppf.as<float4>();
    v.ppf2 = h->ppf2.as<float4>();
    v.alpha = h->alpha.as<double>();
    v.Ahl = h->Ahl.as<float4>();
    v.ppd = h->ppd.as<float4>();
    v.pq = h->pq.as<float>();
    return v;
}

template <class T>
int upload(DevBuf& d, const T* h, size_t n, cudaStream_t st) {
    int rc = d.alloc(sizeof(T) * n);
    if (rc) return rc;
    CK(cudaMemcpyAsync(d.p, h, sizeof(T) * n, cudaMemcpyHostToDevice, st));
    return 0;
}

int build_impl(const jk_atoms* atoms, const jk_shells* shells, double thresh, jk_pairs_s* h, cudaStream_t st) {
    const int S = shells->nshell;
    // ---- host-side validation and basis offsets (before any CUDA call, so a
    // malformed basis is reported the same way with or without a device)
    std::vector<int> bf(S);
    int nbf = 0, nprim_tot = 0;
    for (int s = 0; s < S; ++s) {
        const int l = shells->l[s];
        if (l < 0) return fail(JK_ERR_INVALID, "negative angular momentum");
        if (l > JK_LMAX) return fail(JK_ERR_UNSUPPORTED, "angular momentum above f");
        if ((l + 1) * (l + 2) / 2 > gb_num_pair_classes())  // pair classes compiled: (lmax+1)(lmax+2)/2
            return fail(JK_ERR_UNSUPPORTED, "angular momentum " + std::to_string(l) + " not compiled into this build");
        if (shells->nprim[s] < 1) return fail(JK_ERR_INVALID, "shell without primitives");
        if (shells->atom[s] < 0 || shells->atom[s] >= atoms->natom) return fail(JK_ERR_INVALID, "shell atom out of range");
        if (shells->prim_offset[s] < 0) return fail(JK_ERR_INVALID, "negative primitive offset");
        nprim_tot = std::max(nprim_tot, shells->prim_offset[s] + shells->nprim[s]);
        bf[s] = nbf;
        nbf += (l + 1) * (l + 2) / 2;
    }
    for (int i = 0; i < nprim_tot; ++i)
        if (!(shells->exps[i] > 0.0) || !std::isfinite(shells->coefs[i]))
            return fail(JK_ERR_INVALID, "non-positive exponent or non-finite coefficient");
    for (int i = 0; i < 3 * atoms->natom; ++i)
        if (!std::isfinite(atoms->xyz[i])) return fail(JK_ERR_INVALID, "non-finite coordinate");
    CK(cudaGetDevice(&h->device));
    CK(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device));
    int rc;
    if ((rc = ensure_boys(h->device, st))) return rc;
    h->natom = atoms->natom;
    h->nshell = S;
    h->nbf = nbf;
    h->shell_l.assign(shells->l, shells->l + S);
    h->nsph = 0;
    for (int s = 0; s < S; ++s) h->nsph += shells->l[s] >= 2 ? 2 * shells->l[s] + 1 : (shells->l[s] + 1) * (shells->l[s] + 2) / 2;
    h->thresh = thresh;
    // ---- upload
    DevBuf d_atom, d_l, d_np, d_off, d_bf, d_e, d_c, d_cn;
    if ((rc = upload(h->xyz, atoms->xyz, 3 * (size_t)atoms->natom, st))) return rc;
    if ((rc = upload(d_atom, shells->atom, S, st))) return rc;
    if ((rc = upload(d_l, shells->l, S, st))) return rc;
    if ((rc = upload(d_np, shells->nprim, S, st))) return rc;
    if ((rc = upload(d_off, shells->prim_offset, S, st))) return rc;
    if ((rc = upload(d_bf, bf.data(), S, st))) return rc;
    {
        std::vector<int> bsh(nbf);
        for (int sh = 0; sh < S; ++sh)
            for (int k = 0; k < (shells->l[sh] + 1) * (shells->l[sh] + 2) / 2; ++k) bsh[bf[sh] + k] = sh;
        if ((rc = upload(h->bf_shell, bsh.data(), nbf, st))) return rc;
    }
    if ((rc = upload(d_e, shells->exps, nprim_tot, st))) return rc;
    if ((rc = upload(d_c, shells->coefs, nprim_tot, st))) return rc;
    if ((rc = d_cn.alloc(sizeof(double) * nprim_tot))) return rc;
    k_normalize<<<nblk(S, 128), 128, 0, st>>>(S, d_l.as<int>(), d_np.as<int>(), d_off.as<int>(), d_e.as<double>(),
                                               d_c.as<double>(), d_cn.as<double>());
    CKL();
    ShellDev SD{d_atom.as<int>(), d_l.as<int>(), d_np.as<int>(), d_off.as<int>(), d_bf.as<int>(),
                d_e.as<double>(), d_cn.as<double>(), h->xyz.as<double>()};
    // ---- every unique pair, primitive offsets
    const long long np = (long long)S * (S + 1) / 2;
    h->npair_all = np;
    long long npad = 1;
    while (npad < np) npad <<= 1;
    DevBuf d_npp, d_poff, d_tot, d_key, d_val;
    if ((rc = d_npp.alloc(sizeof(long long) * np))) return rc;
    if ((rc = d_poff.alloc(sizeof(long long) * np))) return rc;
    if ((rc = d_tot.alloc(sizeof(long long) * 4))) return rc;
    if ((rc = d_key.alloc(sizeof(unsigned long long) * npad))) return rc;
    if ((rc = d_val.alloc(sizeof(int) * npad))) return rc;
    k_pair_count<<<nblk(npad, 256), 256, 0, st>>>(SD, np, d_npp.as<long long>(), d_key.as<unsigned long long>(),
                                                   d_val.as<int>(), npad);
    CKL();
    if ((rc = scan_exclusive(d_npp.as<long long>(), d_poff.as<long long>(), np, d_tot.as<long long>(), st))) return rc;
    long long nprimpair = 0;
    CK(cudaMemcpyAsync(&nprimpair, d_tot.p, sizeof(long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (nprimpair > (long long)INT32_MAX) return fail(JK_ERR_UNSUPPORTED, "more than 2^31 primitive pairs");
    h->nprimpair = nprimpair;
    // unsorted pair arrays
    DevBuf u_info, u_A, u_B, u_atoms, u_lab, u_sh;
    if ((rc = u_info.alloc(sizeof(int4) * np))) return rc;
    if ((rc = u_A.alloc(sizeof(double4) * np))) return rc;
    if ((rc = u_B.alloc(sizeof(double4) * np))) return rc;
    if ((rc = u_atoms.alloc(sizeof(int2) * np))) return rc;
    if ((rc = u_sh.alloc(sizeof(int2) * np))) return rc;
    if ((rc = u_lab.alloc(sizeof(int2) * np))) return rc;
    if ((rc = h->pp.alloc(sizeof(double4) * nprimpair))) return rc;
    if ((rc = h->pp2.alloc(sizeof(double2) * nprimpair))) return rc;
    if ((rc = h->ppf.alloc(sizeof(float4) * nprimpair))) return rc;
    if ((rc = h->ppf2.alloc(sizeof(float4) * nprimpair))) return rc;
    if ((rc = h->ppd.alloc(sizeof(float4) * 5 * nprimpair))) return rc;
    if ((rc = h->alpha.alloc(sizeof(double) * nprimpair))) return rc;
    k_pair_fill<<<nblk(np, 128), 128, 0, st>>>(SD, np, d_poff.as<long long>(), u_info.as<int4>(), u_A.as<double4>(),
                                                u_B.as<double4>(), u_atoms.as<int2>(), u_lab.as<int2>(),
                                                h->pp.as<double4>(), h->pp2.as<double2>(), h->ppf.as<float4>(),
                                                h->ppf2.as<float4>(), h->ppd.as<float4>(), h->alpha.as<double>(),
                                                u_sh.as<int2>());
    CKL();
    // ---- sort 1: by class, then Schwarz per class
    if ((rc = sort_pairs(d_key.as<unsigned long long>(), d_val.as<int>(), npad, st))) return rc;
    DevBuf s_info, s_A, s_B, s_atoms, s_lab, s_sh;
    if ((rc = s_info.alloc(sizeof(int4) * np))) return rc;
    if ((rc = s_A.alloc(sizeof(double4) * np))) return rc;
    if ((rc = s_B.alloc(sizeof(double4) * np))) return rc;
    if ((rc = s_atoms.alloc(sizeof(int2) * np))) return rc;
    if ((rc = s_sh.alloc(sizeof(int2) * np))) return rc;
    if ((rc = s_lab.alloc(sizeof(int2) * np))) return rc;
    k_gather<int4><<<nblk(np, 256), 256, 0, st>>>(u_info.as<int4>(), d_val.as<int>(), s_info.as<int4>(), np);
    k_gather<double4><<<nblk(np, 256), 256, 0, st>>>(u_A.as<double4>(), d_val.as<int>(), s_A.as<double4>(), np);
    k_gather<double4><<<nblk(np, 256), 256, 0, st>>>(u_B.as<double4>(), d_val.as<int>(), s_B.as<double4>(), np);
    k_gather<int2><<<nblk(np, 256), 256, 0, st>>>(u_atoms.as<int2>(), d_val.as<int>(), s_atoms.as<int2>(), np);
    k_gather<int2><<<nblk(np, 256), 256, 0, st>>>(u_sh.as<int2>(), d_val.as<int>(), s_sh.as<int2>(), np);
    k_gather<int2><<<nblk(np, 256), 256, 0, st>>>(u_lab.as<int2>(), d_val.as<int>(), s_lab.as<int2>(), np);
    CKL();
    const int ncls = gb_num_pair_classes();
    DevBuf d_cstart;
    if ((rc = d_cstart.alloc(sizeof(int) * kMaxClasses))) return rc;
    std::vector<int> cst(kMaxClasses, -1);
    CK(cudaMemcpyAsync(d_cstart.p, cst.data(), sizeof(int) * kMaxClasses, cudaMemcpyHostToDevice, st));
    k_class_bounds<<<nblk(np, 256), 256, 0, st>>>(d_key.as<unsigned long long>(), np, 40, 0xF, d_cstart.as<int>());
    CKL();
    CK(cudaMemcpyAsync(cst.data(), d_cstart.p, sizeof(int) * kMaxClasses, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<int> cend(kMaxClasses, 0);
    {
        int next = (int)np;
        for (int c = kMaxClasses - 1; c >= 0; --c) {
            if (cst[c] >= 0) { cend[c] = next; next = cst[c]; } else { cst[c] = next; cend[c] = next; }
        }
    }
    DevBuf d_q, d_qmax;
    if ((rc = d_q.alloc(sizeof(double) * np))) return rc;
    if ((rc = d_qmax.alloc(sizeof(unsigned long long)))) return rc;
    CK(cudaMemsetAsync(d_qmax.p, 0, sizeof(unsigned long long), st));
    gb::PairsView pv;
    std::memset(&pv, 0, sizeof(pv));
    pv.npair = (int)np;
    pv.info = s_info.as<int4>();
    pv.A = s_A.as<double4>();
    pv.B = s_B.as<double4>();
    pv.pp = h->pp.as<double4>();
    pv.pp2 = h->pp2.as<double2>();
    const double* boys = g_boys[h->device].tab.as<double>();
    DevBuf d_diag;
    size_t diag_len = 1;
    for (int c = 0; c < ncls; ++c) diag_len = std::max(diag_len, (size_t)(cend[c] - cst[c]) * pair_ncart(c));
    if ((rc = d_diag.alloc(sizeof(double) * diag_len * gb::kSchwarzSplit))) return rc;
    for (int c = 0; c < ncls; ++c) {
        const int cnt = cend[c] - cst[c];
        if (cnt <= 0) continue;
        const int nab = pair_ncart(c);
        CK(cudaMemsetAsync(d_diag.p, 0, sizeof(double) * (size_t)cnt * nab * gb::kSchwarzSplit, st));
        gb::SchwarzArgs sa{pv, cst[c], cnt, boys, d_diag.as<double>(), d_q.as<double>() + cst[c]};
        if (gb_launch_schwarz(c, sa, st)) return fail(JK_ERR_CUDA, "Schwarz kernel launch failed");
        k_schwarz_finish<<<nblk(cnt, 256), 256, 0, st>>>(d_diag.as<double>(), nab, cnt, d_q.as<double>() + cst[c]);
        CKL();
        k_store_q<<<nblk(cnt, 256), 256, 0, st>>>(d_q.as<double>() + cst[c], cst[c], cnt, s_A.as<double4>(),
                                                  d_qmax.as<unsigned long long>());
        CKL();
    }
    unsigned long long qmb = 0;
    CK(cudaMemcpyAsync(&qmb, d_qmax.p, sizeof(qmb), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double qmax;
    std::memcpy(&qmax, &qmb, sizeof(double));
    h->Qmax = qmax;
    // ---- sort 2: (class, bucket, Q descending), drop pairs with Q * Qmax < thresh
    k_final_key<<<nblk(npad, 256), 256, 0, st>>>(s_A.as<double4>(), s_info.as<int4>(), s_lab.as<int2>(), np, thresh,
                                                  qmax, d_key.as<unsigned long long>(), d_val.as<int>(), npad);
    CKL();
    CK(cudaMemsetAsync(d_tot.p, 0, sizeof(long long), st));
    k_count_kept<<<nblk(np, 256), 256, 0, st>>>(d_key.as<unsigned long long>(), np, d_tot.as<unsigned long long>());
    CKL();
    if ((rc = sort_pairs(d_key.as<unsigned long long>(), d_val.as<int>(), npad, st))) return rc;
    long long kept = 0;
    CK(cudaMemcpyAsync(&kept, d_tot.p, sizeof(long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    h->npair = kept;
    const long long nk = std::max(1LL, kept);
    if ((rc = h->info.alloc(sizeof(int4) * nk))) return rc;
    if ((rc = h->A.alloc(sizeof(double4) * nk))) return rc;
    if ((rc = h->B.alloc(sizeof(double4) * nk))) return rc;
    if ((rc = h->pair_atoms.alloc(sizeof(int2) * nk))) return rc;
    if ((rc = h->pair_sh.alloc(sizeof(int2) * nk))) return rc;
    if ((rc = h->pair_lab.alloc(sizeof(int2) * nk))) return rc;
    if (kept > 0) {
        k_gather<int4><<<nblk(kept, 256), 256, 0, st>>>(s_info.as<int4>(), d_val.as<int>(), h->info.as<int4>(), kept);
        k_gather<double4><<<nblk(kept, 256), 256, 0, st>>>(s_A.as<double4>(), d_val.as<int>(), h->A.as<double4>(), kept);
        k_gather<double4><<<nblk(kept, 256), 256, 0, st>>>(s_B.as<double4>(), d_val.as<int>(), h->B.as<double4>(), kept);
        k_gather<int2><<<nblk(kept, 256), 256, 0, st>>>(s_atoms.as<int2>(), d_val.as<int>(), h->pair_atoms.as<int2>(), kept);
        k_gather<int2><<<nblk(kept, 256), 256, 0, st>>>(s_sh.as<int2>(), d_val.as<int>(), h->pair_sh.as<int2>(), kept);
        k_gather<int2><<<nblk(kept, 256), 256, 0, st>>>(s_lab.as<int2>(), d_val.as<int>(), h->pair_lab.as<int2>(), kept);
        CKL();
        k_quantise_q<<<nblk(kept, 256), 256, 0, st>>>(h->A.as<double4>(), kept);
        CKL();
    }
    if ((rc = h->Ahl.alloc(sizeof(float4) * 2 * nk))) return rc;
    if (kept > 0) {
        k_centres_hl<<<nblk(kept, 256), 256, 0, st>>>(h->A.as<double4>(), kept, h->Ahl.as<float4>());
        CKL();
    }
    // ---- class / bucket segments
    const int nseg = kMaxClasses * kNB;
    DevBuf d_bs;
    if ((rc = d_bs.alloc(sizeof(int) * nseg))) return rc;
    std::vector<int> bs(nseg, -1);
    CK(cudaMemcpyAsync(d_bs.p, bs.data(), sizeof(int) * nseg, cudaMemcpyHostToDevice, st));
    if (kept > 0) {
        k_bucket_bounds<<<nblk(kept, 256), 256, 0, st>>>(d_key.as<unsigned long long>(), kept, d_bs.as<int>());
        CKL();
    }
    CK(cudaMemcpyAsync(bs.data(), d_bs.p, sizeof(int) * nseg, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<int> be(nseg, 0);
    {
        int next = (int)kept;
        for (int c = nseg - 1; c >= 0; --c) {
            if (bs[c] >= 0) { be[c] = next; next = bs[c]; } else { bs[c] = next; be[c] = next; }
        }
    }
    h->cls_start.assign(ncls + 1, 0);
    for (int c = 0; c < ncls; ++c) h->cls_start[c] = bs[c * kNB];
    h->cls_start[ncls] = (int)kept;
    h->bucket_start = bs;
    // ---- quartet rows per (bra class X >= ket class Y)
    DevBuf d_npk;
    DevBuf& d_npre = h->npre;
    if ((rc = d_npk.alloc(sizeof(long long) * (nk + 1)))) return rc;
    if ((rc = d_npre.alloc(sizeof(long long) * (nk + 1)))) return rc;
    CK(cudaMemsetAsync(d_npk.p, 0, sizeof(long long) * (nk + 1), st));
    if (kept > 0) {
        k_np_of<<<nblk(kept, 256), 256, 0, st>>>(h->info.as<int4>(), kept, d_npk.as<long long>());
        CKL();
    }
    if ((rc = scan_exclusive(d_npk.as<long long>(), d_npre.as<long long>(), kept + 1, d_tot.as<long long>() + 1, st)))
        return rc;
    // ---- primitive Schwarz factors; primitive pairs of every kept pair sorted by
    // them (largest first) into compact arrays (the dropped pairs' primitive
    // pairs are released)
    {
        std::vector<long long> ncp(ncls + 1, 0);
        for (int c = 0; c <= ncls; ++c)
            CK(cudaMemcpyAsync(&ncp[c], d_npre.as<long long>() + h->cls_start[c], sizeof(long long),
                               cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const long long nkp = ncp[ncls];
        if (nkp > (long long)INT32_MAX) return fail(JK_ERR_UNSUPPORTED, "more than 2^31 primitive pairs");
        const long long nk1 = std::max(1LL, nkp);
        DevBuf f_info, f_A, f_B, f_q;
        if ((rc = f_info.alloc(sizeof(int4) * nk1))) return rc;
        if ((rc = f_A.alloc(sizeof(double4) * nk1))) return rc;
        if ((rc = f_B.alloc(sizeof(double4) * nk1))) return rc;
        if ((rc = f_q.alloc(sizeof(double) * nk1))) return rc;
        if (kept > 0) {
            k_prim_expand<<<nblk(kept, 256), 256, 0, st>>>(h->info.as<int4>(), h->A.as<double4>(), h->B.as<double4>(),
                                                            d_npre.as<long long>(), kept, f_info.as<int4>(),
                                                            f_A.as<double4>(), f_B.as<double4>());
            CKL();
        }
        gb::PairsView fv;
        std::memset(&fv, 0, sizeof(fv));
        fv.npair = (int)nkp;
        fv.info = f_info.as<int4>();
        fv.A = f_A.as<double4>();
        fv.B = f_B.as<double4>();
        fv.pp = h->pp.as<double4>();
        fv.pp2 = h->pp2.as<double2>();
        for (int c = 0; c < ncls; ++c) {
            const int nab = pair_ncart(c);
            const long long chunk = std::max<long long>(1, (long long)(diag_len / nab));
            for (long long e0 = ncp[c]; e0 < ncp[c + 1]; e0 += chunk) {
                const int cnt = (int)std::min(chunk, ncp[c + 1] - e0);
                CK(cudaMemsetAsync(d_diag.p, 0, sizeof(double) * (size_t)cnt * nab * gb::kSchwarzSplit, st));
                gb::SchwarzArgs sa{fv, (int)e0, cnt, boys, d_diag.as<double>(), f_q.as<double>() + e0};
                if (gb_launch_schwarz(c, sa, st)) return fail(JK_ERR_CUDA, "primitive Schwarz kernel launch failed");
                k_schwarz_finish<<<nblk(cnt, 256), 256, 0, st>>>(d_diag.as<double>(), nab, cnt, f_q.as<double>() + e0);
                CKL();
            }
        }
        DevBuf n_pp, n_pp2, n_ppf, n_ppf2, n_ppd, n_alpha;
        if ((rc = n_pp.alloc(sizeof(double4) * nk1))) return rc;
        if ((rc = n_pp2.alloc(sizeof(double2) * nk1))) return rc;
        if ((rc = n_ppf.alloc(sizeof(float4) * nk1))) return rc;
        if ((rc = n_ppf2.alloc(sizeof(float4) * nk1))) return rc;
        if ((rc = n_ppd.alloc(sizeof(float4) * 5 * nk1))) return rc;
        if ((rc = n_alpha.alloc(sizeof(double) * nk1))) return rc;
        if ((rc = h->pq.alloc(sizeof(float) * nk1))) return rc;
        if (kept > 0) {
            k_prim_sort<<<nblk(kept, 128), 128, 0, st>>>(
                h->info.as<int4>(), d_npre.as<long long>(), kept, f_q.as<double>(), h->pp.as<double4>(),
                h->pp2.as<double2>(), h->ppf.as<float4>(), h->ppf2.as<float4>(), h->ppd.as<float4>(),
                h->alpha.as<double>(), n_pp.as<double4>(), n_pp2.as<double2>(), n_ppf.as<float4>(),
                n_ppf2.as<float4>(), n_ppd.as<float4>(), n_alpha.as<double>(), h->pq.as<float>());
            CKL();
        }
        CK(cudaStreamSynchronize(st));  // the old arrays are released below
        h->pp = std::move(n_pp);
        h->pp2 = std::move(n_pp2);
        h->ppf = std::move(n_ppf);
        h->ppf2 = std::move(n_ppf2);
        h->ppd = std::move(n_ppd);
        h->alpha = std::move(n_alpha);
        h->nprimpair = nkp;
    }
    // Every class pair's rows are enumerated, scanned and counted in stream
    // order with shared scratch; the per-class totals land in one device array
    // that is read back with a single synchronisation at the end.
    h->rows.clear();
    h->rows.reserve(ncls * (ncls + 1) / 2);
    h->nquartets = 0;
    h->nprimq = 0;
    std::vector<int> seg_all, seg_off(ncls + 1, 0);
    for (int Y = 0; Y < ncls; ++Y) {
        for (int b = 0; b < kNB; ++b)
            if (be[Y * kNB + b] > bs[Y * kNB + b]) { seg_all.push_back(bs[Y * kNB + b]); seg_all.push_back(be[Y * kNB + b]); }
        seg_off[Y + 1] = (int)seg_all.size() / 2;
    }
    if (seg_all.empty()) seg_all.assign(2, 0);  // nothing kept: a placeholder keeps the upload non-empty
    long long max_rows = 0;
    for (int X = 0; X < ncls; ++X) {
        const int nX = be[X * kNB + kNB - 1] - bs[X * kNB];
        for (int Y = 0; Y <= X; ++Y) {
            const int nb = seg_off[Y + 1] - seg_off[Y];
            if (nX == 0 || nb == 0) continue;
            h->rows.emplace_back();
            ClassRows& cr = h->rows.back();
            cr.bra_cls = X;
            cr.ket_cls = Y;
            if ((long long)nX * nb > INT32_MAX) return fail(JK_ERR_UNSUPPORTED, "more than 2^31 quartet rows in a class");
            cr.nrows = nX * nb;
            max_rows = std::max<long long>(max_rows, cr.nrows);
        }
    }
    const int ncr = (int)h->rows.size();
    DevBuf d_seg, d_cnt, d_scr, d_ctot;
    if ((rc = upload(d_seg, seg_all.data(), std::max<size_t>(1, seg_all.size()), st))) return rc;
    if ((rc = d_cnt.alloc(sizeof(long long) * (max_rows + 1)))) return rc;
    if ((rc = d_scr.alloc(sizeof(long long) * (scan_scratch_len(max_rows + 1) + 1)))) return rc;
    if ((rc = d_ctot.alloc(sizeof(long long) * 4 * std::max(1, ncr)))) return rc;
    CK(cudaMemsetAsync(d_ctot.p, 0, sizeof(long long) * 4 * std::max(1, ncr), st));
    for (int k = 0; k < ncr; ++k) {
        ClassRows& cr = h->rows[k];
        const int X = cr.bra_cls, Y = cr.ket_cls;
        const int x0 = bs[X * kNB], nX = be[X * kNB + kNB - 1] - x0, nb = seg_off[Y + 1] - seg_off[Y];
        long long* ctot = d_ctot.as<long long>() + 4 * k;  // quartets, work items, primitive quartets, bra prim units
        if ((rc = cr.start.alloc(sizeof(long long) * (cr.nrows + 1)))) return rc;
        if ((rc = cr.bra.alloc(sizeof(int) * cr.nrows))) return rc;
        if ((rc = cr.ket0.alloc(sizeof(int) * cr.nrows))) return rc;
        if ((rc = cr.istart.alloc(sizeof(long long) * (cr.nrows + 1)))) return rc;
        k_rows_count<<<nblk(cr.nrows, 256), 256, 0, st>>>(h->A.as<double4>(), x0, nX, d_seg.as<int>() + 2 * seg_off[Y],
                                                          nb, X == Y, thresh, d_cnt.as<long long>(), cr.bra.as<int>(),
                                                          cr.ket0.as<int>());
        CKL();
        CK(cudaMemsetAsync(d_cnt.as<long long>() + cr.nrows, 0, sizeof(long long), st));
        if ((rc = scan_into(d_cnt.as<long long>(), cr.start.as<long long>(), cr.nrows + 1, ctot, d_scr.as<long long>(), st)))
            return rc;
        k_rows_primq<<<nblk(cr.nrows, 256), 256, 0, st>>>(d_cnt.as<long long>(), cr.bra.as<int>(), cr.ket0.as<int>(),
                                                          cr.nrows, h->info.as<int4>(), d_npre.as<long long>(),
                                                          reinterpret_cast<unsigned long long*>(ctot + 2));
        CKL();
        // work items of the FP64 launch (the counts buffer is reused once primq has read it)
        k_row_items<<<nblk(cr.nrows, 256), 256, 0, st>>>(cr.start.as<long long>(), cr.bra.as<int>(), cr.nrows,
                                                         h->info.as<int4>(), nullptr, nullptr, gb_class_split(X, Y),
                                                         d_cnt.as<long long>());
        CKL();
        if ((rc = scan_into(d_cnt.as<long long>(), cr.istart.as<long long>(), cr.nrows + 1, ctot + 1,
                            d_scr.as<long long>(), st)))
            return rc;
    }
    std::vector<long long> ctot(4 * std::max(1, ncr));
    CK(cudaMemcpyAsync(ctot.data(), d_ctot.p, sizeof(long long) * ctot.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int k = 0; k < ncr; ++k) {
        ClassRows& cr = h->rows[k];
        cr.total = ctot[4 * k];
        cr.itotal = ctot[4 * k + 1];
        cr.nprimq = ctot[4 * k + 2];
        cr.nbrap = ctot[4 * k + 3];
        h->nquartets += cr.total;
        h->nprimq += cr.nprimq;
    }
    return 0;
}

// Grid of a persistent class launch: `qpt` work items per thread (the Workload
// Allocator's unit of work, Algorithm 2 "Combine" doubles it), at least one
// wave of one block per SM, at most 64 blocks per SM.
int grid_for(long long total, int block, int qpt, int nsm) {
    long long g = (total + (long long)block * qpt - 1) / ((long long)block * qpt);
    g = std::max<long long>(g, 1);
    g = std::min<long long>(g, (long long)nsm * 64);
    return (int)g;
}

// One class kernel over the rows [r0, r0 + nrows) of a class (nrows < 0: to the
// end of the class); start / ket0 / kofs are the class's per-row arrays of this
// launch (indexed by row, offset here), klist its explicit ket list.  Jlo/Klo:
// compensated accumulation (FP64 builds) or nullptr.
int launch_class(jk_pairs_s* h, const ClassRows& cr, int prec, const long long* start, const int* ket0,
                 long long total_hint, const double* D, double* J, double* K, cudaStream_t st,
                 int nrows = -1, const long long* kofs = nullptr, const int* klist = nullptr, int r0 = 0,
                 double* Jlo = nullptr, double* Klo = nullptr, int pmode = 0, const float* kthr = nullptr) {
    if (total_hint <= 0) return 0;
    const int nr = nrows >= 0 ? nrows : cr.nrows - r0;
    if (nr <= 0) return 0;
    gb::JKArgs a;
    std::memset(&a, 0, sizeof(a));
    a.pairs = view_of(h);
    a.rows.nrows = nr;
    a.rows.start = start + r0;
    a.rows.bra = cr.bra.as<int>() + r0;
    a.rows.ket0 = ket0 ? ket0 + r0 : nullptr;
    a.rows.kofs = kofs ? kofs + r0 : nullptr;
    a.rows.klist = klist;
    a.rows.kthr = kthr;
    a.pmode = (klist && kthr) ? pmode : 0;
    a.Jlo = Jlo;
    a.Klo = Klo;
    a.boys = g_boys[h->device].tab.as<double>();
    a.boysf = g_boys[h->device].tabf.as<float>();
    a.tsmall = (float)g_opt.tsmall;
    a.D = D;
    a.Df = h->Df.as<float>();
    a.Ddf = h->Ddf.as<gb::dfl>();
    a.boysd = g_boys[h->device].tabd.as<float2>();
    a.J = J;
    a.K = K;
    a.nbf = h->nbf;
    const TuneCfg& tc = cr.tune[prec == 3 ? 0 : prec];
    const int grid = grid_for(total_hint * gb_class_threads(cr.bra_cls, cr.ket_cls, prec == 3 ? 0 : prec), tc.block, tc.qpt,
                              h->nsm);
    ProfRec* pr = nullptr;
    if (g_opt.profile) {
        h->prof.emplace_back();
        pr = &h->prof.back();
        CK(cudaEventCreate(&pr->e0));
        CK(cudaEventCreate(&pr->e1));
        pr->bra = cr.bra_cls;
        pr->ket = cr.ket_cls;
        pr->prec = a.pmode == 2 ? 4 : prec;  // 4: FP32 complement of a primitive split
        pr->total = total_hint;
        CK(cudaEventRecord(pr->e0, st));
    }
    const int e = gb_launch_jk(cr.bra_cls, cr.ket_cls, prec == 1 && g_opt.rpath ? 2 : prec, a, grid, tc.block, st);
    if (e) return fail(JK_ERR_CUDA, std::string("ERI kernel launch: ") + cudaGetErrorString((cudaError_t)e));
    h->launches += 1;
    if (pr) CK(cudaEventRecord(pr->e1, st));
    return 0;
}

// Mixed split of the rows [r0, r1) of one class, first phase (counts): per-row
// quartet and item counts of the FP64 list, the demoted list and the FP32
// suffix; the quartet totals are added into split_tot[0..1] (FP32 incl.
// demoted, FP64).  The per-row arrays are sized for the whole class and
// written at the rows' own indices (with a zero after row r1 - 1).
int split_count(jk_pairs_s* h, ClassRows& cr, int r0, int r1, const double* dmax, long long* split_tot,
                cudaStream_t st, double tau, double eps) {
    int rc;
    const long long n1 = cr.nrows + 1;
    for (DevBuf* b : {&cr.c64, &cr.c32, &cr.cdem, &cr.w64, &cr.w32, &cr.wdem, &cr.s64, &cr.s32, &cr.sdem, &cr.l64,
                      &cr.ldem})
        if ((rc = b->alloc(sizeof(long long) * n1))) return rc;
    if ((rc = cr.k32.alloc(sizeof(int) * cr.nrows))) return rc;
    if ((rc = cr.scr.alloc(sizeof(long long) * (scan_scratch_len(n1) + 1)))) return rc;
    const int nr = r1 - r0;
    k_rows_split<<<nblk(nr, 256), 256, 0, st>>>(
        cr.start.as<long long>() + r0, cr.bra.as<int>() + r0, cr.ket0.as<int>() + r0, nr, h->A.as<double4>(), dmax,
        tau, eps, h->info.as<int4>(), h->pair_sh.as<int2>(), h->Dsh.as<float>(), h->nshell,
        gb_class_split(cr.bra_cls, cr.ket_cls), cr.c64.as<long long>() + r0, cr.cdem.as<long long>() + r0,
        cr.c32.as<long long>() + r0, cr.k32.as<int>() + r0, cr.w64.as<long long>() + r0,
        cr.wdem.as<long long>() + r0, cr.w32.as<long long>() + r0, reinterpret_cast<unsigned long long*>(split_tot));
    CKL();
    for (DevBuf* b : {&cr.c64, &cr.c32, &cr.cdem, &cr.w64, &cr.w32, &cr.wdem})
        CK(cudaMemsetAsync(b->as<long long>() + r1, 0, 8, st));
    h->launches += 1;
    return 0;
}

// Second phase over the same rows: item prefixes (s64, sdem, s32; totals into
// split_tot[2..4]), list offsets (l64, ldem; totals into split_tot[5..6]) and
// the list fill.  The prefixes start at 0 at row r0.
int split_fill(jk_pairs_s* h, ClassRows& cr, int r0, int r1, long long* split_tot, int* list64, int* listdem,
               cudaStream_t st, double tau, double eps, float taup, float* thr64) {
    int rc;
    const long long n1 = r1 - r0 + 1;
    long long* scr = cr.scr.as<long long>();
    if ((rc = scan_into(cr.w32.as<long long>() + r0, cr.s32.as<long long>() + r0, n1, split_tot + 2, scr, st))) return rc;
    if ((rc = scan_into(cr.w64.as<long long>() + r0, cr.s64.as<long long>() + r0, n1, split_tot + 3, scr, st))) return rc;
    if ((rc = scan_into(cr.wdem.as<long long>() + r0, cr.sdem.as<long long>() + r0, n1, split_tot + 4, scr, st)))
        return rc;
    if ((rc = scan_into(cr.c64.as<long long>() + r0, cr.l64.as<long long>() + r0, n1, split_tot + 5, scr, st))) return rc;
    if ((rc = scan_into(cr.cdem.as<long long>() + r0, cr.ldem.as<long long>() + r0, n1, split_tot + 6, scr, st)))
        return rc;
    const int nr = r1 - r0;
    k_rows_fill<<<nblk(nr, 256), 256, 0, st>>>(cr.bra.as<int>() + r0, cr.ket0.as<int>() + r0, cr.k32.as<int>() + r0, nr,
                                               h->A.as<double4>(), tau, eps, h->pair_sh.as<int2>(),
                                               h->Dsh.as<float>(), h->nshell, cr.l64.as<long long>() + r0,
                                               cr.ldem.as<long long>() + r0, list64, listdem, taup, thr64);
    CKL();
    h->launches += 1 + 5 * scan_launches(n1);
    return 0;
}

// Host: cost-balanced split of n consecutive units into nparts contiguous
// ranges (bounds[0] = 0 <= ... <= bounds[nparts] = n): bounds[p] is the first
// unit at which the running cost reaches p/nparts of the total, so every part
// costs total/nparts within the cost of one unit.  Zero total: equal counts.
int partition_costs(long long n, const double* cost, int nparts, long long* bounds) {
    if (n < 0 || nparts < 1 || (n > 0 && !cost) || !bounds) return fail(JK_ERR_INVALID, "partition arguments");
    std::vector<double> pre((size_t)n + 1, 0.0);
    for (long long i = 0; i < n; ++i) {
        if (!(cost[i] >= 0.0) || !std::isfinite(cost[i])) return fail(JK_ERR_INVALID, "partition cost negative or not finite");
        pre[i + 1] = pre[i] + cost[i];
    }
    const double T = pre[n];
    bounds[0] = 0;
    bounds[nparts] = n;
    for (int p = 1; p < nparts; ++p) {
        if (T > 0.0) {
            const double t = T * ((double)p / nparts);
            bounds[p] = (long long)(std::lower_bound(pre.begin(), pre.end(), t) - pre.begin());
        } else {
            bounds[p] = (long long)((double)n * p / nparts);
        }
        bounds[p] = std::max(bounds[p], bounds[p - 1]);
    }
    return 0;
}

// Row partition of every class for `nparts` parts (cached on the handle): the
// rows of each class are cut by their algorithmic cost, so that every part
// holds the same share of every class.  One synchronisation per new nparts.
int ensure_partition(jk_pairs_s* h, int nparts, cudaStream_t st) {
    if (h->part_n == nparts) return 0;
    h->part_n = 0;
    h->part_rows.assign(h->rows.size(), {});
    h->part_items.assign(h->rows.size(), {});
    h->part_cost.assign(h->rows.size(), std::vector<double>(nparts + 1, 0.0));
    DevBuf d_cost;
    int rc;
    for (size_t k = 0; k < h->rows.size(); ++k) {
        const ClassRows& cr = h->rows[k];
        std::vector<int>& rb = h->part_rows[k];
        std::vector<long long>& ib = h->part_items[k];
        rb.assign(nparts + 1, 0);
        ib.assign(nparts + 1, 0);
        if (cr.nrows <= 0 || cr.total <= 0) {
            for (int p = 0; p <= nparts; ++p) rb[p] = p == nparts ? cr.nrows : 0;
            continue;
        }
        int fq = 0, fb = 0;
        gb_class_flops(cr.bra_cls, cr.ket_cls, &fq, &fb);
        if ((rc = d_cost.alloc(sizeof(double) * cr.nrows))) return rc;
        k_row_cost<<<nblk(cr.nrows, 256), 256, 0, st>>>(cr.start.as<long long>(), cr.bra.as<int>(), cr.ket0.as<int>(),
                                                        cr.nrows, h->info.as<int4>(), h->npre.as<long long>(), fq, fb,
                                                        d_cost.as<double>());
        CKL();
        std::vector<double> cost(cr.nrows);
        std::vector<long long> istart(cr.nrows + 1);
        CK(cudaMemcpyAsync(cost.data(), d_cost.p, sizeof(double) * cr.nrows, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(istart.data(), cr.istart.p, sizeof(long long) * (cr.nrows + 1), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        std::vector<long long> b(nparts + 1);
        if ((rc = partition_costs(cr.nrows, cost.data(), nparts, b.data()))) return rc;
        for (int p = 0; p <= nparts; ++p) {
            rb[p] = (int)b[p];
            ib[p] = istart[b[p]];
        }
        std::vector<double>& pc = h->part_cost[k];
        for (int p = 0; p < nparts; ++p)
            for (long long r = b[p]; r < b[p + 1]; ++r) pc[p] += cost[r];
        pc[nparts] = *std::max_element(cost.begin(), cost.end());
    }
    h->part_n = nparts;
    return 0;
}

// J and K of the rows of part `part` of `nparts` (nparts = 1: the whole build).
// The class launches of one build are spread over the caller's stream and three
// forked ones (launch tails of one class overlap the next class's work; J and
// K take atomic updates from all of them), then joined back into the caller's
// stream.  With JK_OPT_PROFILE set everything stays on the caller's stream, so
// that the per-launch event times do not overlap.
int fork_streams(jk_pairs_s* h, cudaStream_t st, std::vector<cudaStream_t>& out) {
    out.assign(1, st);
    if (g_opt.profile) return 0;
    if (!h->fork) {
        for (auto& x : h->side) CK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
        for (auto& e : h->join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(h->fork, st));
    for (auto& x : h->side) {
        CK(cudaStreamWaitEvent(x, h->fork, 0));
        out.push_back(x);
    }
    return 0;
}

int join_streams(jk_pairs_s* h, cudaStream_t st, const std::vector<cudaStream_t>& ss) {
    for (size_t i = 1; i < ss.size(); ++i) {
        CK(cudaEventRecord(h->join[i - 1], ss[i]));
        CK(cudaStreamWaitEvent(st, h->join[i - 1], 0));
    }
    return 0;
}

int jk_build_impl(jk_pairs_s* h, const double* D, double* J, double* K, jk_precision prec, cudaStream_t st,
                  int part = 0, int nparts = 1) {
    const int n = h->nbf;
    int rc;
    if ((rc = h->scratch.alloc(64))) return rc;
    if (g_opt.check_sym) {
        CK(cudaMemsetAsync(h->scratch.p, 0, 8, st));
        k_asym<<<152 * 4, 256, 0, st>>>(D, n, h->scratch.as<unsigned long long>());
        CKL();
        unsigned long long b = 0;
        CK(cudaMemcpyAsync(&b, h->scratch.p, 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double m;
        std::memcpy(&m, &b, 8);
        if (!(m == 0.0)) {
            if (std::isnan(m)) return fail(JK_ERR_INVALID, "D holds a non-finite element");
            return fail(JK_ERR_NOT_SYMMETRIC, "D is not symmetric (max |D - D^T| = " + std::to_string(m) + ")");
        }
    }
    if (nparts > 1 && (rc = ensure_partition(h, nparts, st))) return rc;
    auto range = [&](size_t k, int& r0, int& r1) {
        if (nparts > 1) { r0 = h->part_rows[k][part]; r1 = h->part_rows[k][part + 1]; }
        else { r0 = 0; r1 = h->rows[k].nrows; }
    };
    const size_t n2 = (size_t)n * n;
    CK(cudaMemsetAsync(J, 0, sizeof(double) * n2, st));
    CK(cudaMemsetAsync(K, 0, sizeof(double) * n2, st));
    for (auto& r : h->prof) {
        if (r.e0) cudaEventDestroy(r.e0);
        if (r.e1) cudaEventDestroy(r.e1);
    }
    h->prof.clear();
    h->launches = 0;
    h->last_prec = prec;
    double* Jlo = nullptr;
    double* Klo = nullptr;
    if (prec == JK_FP64) {
        if ((rc = h->Jlo.alloc(sizeof(double) * n2))) return rc;
        if ((rc = h->Klo.alloc(sizeof(double) * n2))) return rc;
        Jlo = h->Jlo.as<double>();
        Klo = h->Klo.as<double>();
        CK(cudaMemsetAsync(Jlo, 0, sizeof(double) * n2, st));
        CK(cudaMemsetAsync(Klo, 0, sizeof(double) * n2, st));
        std::vector<cudaStream_t> ss;
        if ((rc = fork_streams(h, st, ss))) return rc;
        int rcl = 0;
        for (size_t k = 0; k < h->rows.size() && rcl == 0; ++k) {
            const ClassRows& cr = h->rows[k];
            int r0, r1;
            range(k, r0, r1);
            const long long items = nparts > 1 ? h->part_items[k][part + 1] - h->part_items[k][part] : cr.itotal;
            rcl = launch_class(h, cr, 0, cr.istart.as<long long>(), cr.ket0.as<int>(), items, D, J, K,
                               ss[k % ss.size()], r1 - r0, nullptr, nullptr, r0, Jlo, Klo);
        }
        if ((rc = join_streams(h, st, ss))) return rc;
        if (rcl) return rcl;
    } else {
        const int ncr = (int)h->rows.size();
        const size_t nst = (size_t)kSplitSlots * std::max(1, ncr);
        if ((rc = h->split_tot.alloc(sizeof(long long) * nst))) return rc;
        CK(cudaMemsetAsync(h->split_tot.p, 0, sizeof(long long) * nst, st));
        if ((rc = h->Df.alloc(sizeof(float) * n2))) return rc;
        if (g_opt.df_tier && (rc = h->Ddf.alloc(sizeof(float2) * n2))) return rc;
        CK(cudaMemsetAsync(h->scratch.p, 0, 8, st));
        k_absmax<<<152 * 4, 256, 0, st>>>(D, (long long)n2, h->scratch.as<unsigned long long>(), h->Df.as<float>(),
                                          g_opt.df_tier ? h->Ddf.as<float2>() : nullptr);
        CKL();
        // max |D| per shell block, for the density-weighted FP64 selection
        const size_t ns2 = (size_t)h->nshell * h->nshell;
        if ((rc = h->Dsh.alloc(sizeof(float) * ns2))) return rc;
        CK(cudaMemsetAsync(h->Dsh.p, 0, sizeof(float) * ns2, st));
        k_dsh<<<152 * 4, 256, 0, st>>>(D, n, h->bf_shell.as<int>(), h->nshell, h->Dsh.as<unsigned int>());
        CKL();
        h->launches += 2;
        const double* dmax = reinterpret_cast<const double*>(h->scratch.p);
        std::vector<int> R0(ncr), R1(ncr);
        for (int k = 0; k < ncr; ++k) {
            range(k, R0[k], R1[k]);
            if (h->rows[k].total > 0 && R1[k] > R0[k] &&
                (rc = split_count(h, h->rows[k], R0[k], R1[k], dmax, h->split_tot.as<long long>() + kSplitSlots * k, st,
                                  g_opt.tau, g_opt.eps)))
                return rc;
        }
        // list sizes: one host synchronisation per mixed build
        std::vector<long long> cnt(nst);
        CK(cudaMemcpyAsync(cnt.data(), h->split_tot.p, sizeof(long long) * nst, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        std::vector<long long> off64(ncr + 1, 0), offd(ncr + 1, 0);
        for (int k = 0; k < ncr; ++k) {
            off64[k + 1] = off64[k] + cnt[kSplitSlots * k + 1];
            offd[k + 1] = offd[k] + cnt[kSplitSlots * k + 7];
        }
        if ((rc = h->list64.alloc(sizeof(int) * std::max(1LL, off64[ncr])))) return rc;
        if ((rc = h->listdem.alloc(sizeof(int) * std::max(1LL, offd[ncr])))) return rc;
        const bool psplit = g_opt.ptau > 0.0;
        if (psplit && (rc = h->thr64.alloc(sizeof(float) * std::max(1LL, off64[ncr])))) return rc;
        h->last_psplit = psplit;
        std::vector<cudaStream_t> ss;
        if ((rc = fork_streams(h, st, ss))) return rc;
        const cudaStream_t st0 = st;
        auto one_class = [&](int k) -> int {
            ClassRows& cr = h->rows[k];
            const int r0 = R0[k], r1 = R1[k];
            if (cr.total <= 0 || r1 <= r0) return 0;
            // this class's list fill and launches on one of the forked streams
            cudaStream_t st = ss[k % ss.size()];
            int* l64 = h->list64.as<int>() + off64[k];
            int* ldm = h->listdem.as<int>() + offd[k];
            float* t64 = psplit ? h->thr64.as<float>() + off64[k] : nullptr;
            if ((rc = split_fill(h, cr, r0, r1, h->split_tot.as<long long>() + kSplitSlots * k, l64, ldm, st, g_opt.tau,
                                 g_opt.eps, (float)g_opt.ptau, t64)))
                return rc;
            // the largest-bound quartets: FP64, or double-float on the FP32 pipe (JK_OPT_DF_TIER); with
            // the primitive split only their large primitive quartets, the rest in an FP32 launch over
            // the same list
            if ((rc = launch_class(h, cr, g_opt.df_tier ? 3 : 0, cr.s64.as<long long>(), nullptr, cr.itotal, D, J, K, st,
                                   r1 - r0, cr.l64.as<long long>(), l64, r0, nullptr, nullptr, 1, t64)))
                return rc;
            if (psplit && (rc = launch_class(h, cr, 1, cr.s64.as<long long>(), nullptr, cr.itotal, D, J, K, st, r1 - r0,
                                             cr.l64.as<long long>(), l64, r0, nullptr, nullptr, 2, t64)))
                return rc;
            if ((rc = launch_class(h, cr, 1, cr.s32.as<long long>(), cr.k32.as<int>(), cr.itotal, D, J, K, st, r1 - r0,
                                   nullptr, nullptr, r0)))
                return rc;
            if ((rc = launch_class(h, cr, 1, cr.sdem.as<long long>(), nullptr, cr.itotal, D, J, K, st, r1 - r0,
                                   cr.ldem.as<long long>(), ldm, r0)))
                return rc;
            return 0;
        };
        int rcl = 0;
        for (int k = 0; k < ncr && rcl == 0; ++k) rcl = one_class(k);
        // joined also after a failed launch, so that no forked work outlives the call's ordering
        if ((rc = join_streams(h, st0, ss))) return rc;
        if (rcl) return rcl;
        h->list_off64 = off64;
        h->list_offd = offd;
        h->last_r0 = R0;
        h->last_r1 = R1;
    }
    const long long tri = (long long)n * (n + 1) / 2;
    if (Jlo) {
        k_symmetrize_lo<<<nblk(tri, 256), 256, 0, st>>>(J, Jlo, n);
        k_symmetrize_lo<<<nblk(tri, 256), 256, 0, st>>>(K, Klo, n);
    } else {
        k_symmetrize<<<nblk(tri, 256), 256, 0, st>>>(J, n);
        k_symmetrize<<<nblk(tri, 256), 256, 0, st>>>(K, n);
    }
    CKL();
    h->launches += 2;
    return 0;
}


// ------------------------------------------------------------------ batched launches
// Many molecules in one launch per (bra class, ket class): the rows of every
// molecule are concatenated, each row carries its molecule index, and the
// kernels read that molecule's pairs / D / J / K from a device table.  The
// launch sequence (zeroing, a mixed build's scans and list fill, class
// launches on four forked streams, symmetrisation) is captured into a CUDA
// graph and replayed while the molecule list, the matrices and the options are
// unchanged; a mixed build's split counts come from a pre-pass before it.
struct BatchClass {
    int X = 0, Y = 0, nrows = 0;
    long long total = 0;
    DevBuf start, bra, ket0, rowmol;
    DevBuf istart, itot;  // work-item prefix of the FP64 launch, its total
    DevBuf s64, s32, k32, c64, c32, w64, w32, scr;
    DevBuf cdem, wdem, sdem, l64, ldem;  // density-weighted split (as ClassRows)
    long long cap64 = 0, capdem = 0;     // list capacities of this class
    long long off64 = 0, offdem = 0;     // its segments in the plan's lists
    TuneCfg tune[2];
};

struct BatchPlan {
    std::vector<jk_pairs> mols;
    std::vector<unsigned long long> serial;  // of every handle: a freed handle's address can come back
    std::vector<const double*> D;
    std::vector<double*> J, K;
    int prec = 0, device = 0, max_n = 0, graph = 0, rpath = 0, df = 0;
    double tau = 0.0, eps = 0.0, tsmall = 0.0, ptau = 0.0;
    long long nquartets = 0;
    DevBuf bm, dmax, split_tot;
    DevBuf list64, listdem;  // mixed: FP64 and demoted ket lists, one segment per class
    DevBuf thr64;            // mixed, primitive split: per FP64 list entry, its primitive cut
    std::vector<BatchClass> cls;
    cudaStream_t cs = nullptr, ps[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[3] = {nullptr, nullptr, nullptr}, done = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;        // kernels of the (captured) launch sequence
    long long launches_total = 0;  // plus the pre-pass of a mixed build
    ~BatchPlan() {
        if (cs) cudaStreamSynchronize(cs);  // the plan's last launch sequence ends on cs
        if (exec) cudaGraphExecDestroy(exec);
        for (auto& x : ps) if (x) cudaStreamDestroy(x);
        if (cs) cudaStreamDestroy(cs);
        if (fork) cudaEventDestroy(fork);
        for (auto& e : join) if (e) cudaEventDestroy(e);
        if (done) cudaEventDestroy(done);
    }
};
std::mutex g_batch_mu;
std::atomic<unsigned long long> g_serial{0};
std::unique_ptr<BatchPlan> g_plan;

// A cached batch plan copies its molecules' per-class launch configuration
// when it is built: a new tuning of any of its handles (or freeing one)
// retires it.
void drop_plan_of(const jk_pairs_s* h) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (g_plan && std::find(g_plan->mols.begin(), g_plan->mols.end(), h) != g_plan->mols.end()) g_plan.reset();
}

__global__ void k_offset_copy(const long long* src, int n, long long off, long long* dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] + off;
}
__global__ void k_fill_int(int* dst, int n, int v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = v;
}
__global__ void k_set_ll(long long* dst, long long v) { *dst = v; }

__global__ void k_zero_batched(const gb::BatchMol* bm) {
    const gb::BatchMol& m = bm[blockIdx.y];
    const long long n2 = (long long)m.nbf * m.nbf;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
        m.J[i] = 0.0;
        m.K[i] = 0.0;
        if (m.Jlo) { m.Jlo[i] = 0.0; m.Klo[i] = 0.0; }
    }
}

__global__ void k_sym_batched(const gb::BatchMol* bm) {
    const gb::BatchMol& m = bm[blockIdx.y];
    const int n = m.nbf;
    const long long tri = (long long)n * (n + 1) / 2;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < tri; t += (long long)gridDim.x * blockDim.x) {
        int i, j;
        decode_pair(t, i, j);
        const size_t a = (size_t)i * n + j, b = (size_t)j * n + i;
        if (m.Jlo) {  // compensated FP64 build: fold the remainders in (as k_symmetrize_lo)
            if (i == j) { m.J[a] = 2.0 * m.J[a] + 2.0 * m.Jlo[a]; m.K[a] = 2.0 * m.K[a] + 2.0 * m.Klo[a]; continue; }
            const double vj = (m.J[a] + m.J[b]) + (m.Jlo[a] + m.Jlo[b]);
            const double vk = (m.K[a] + m.K[b]) + (m.Klo[a] + m.Klo[b]);
            m.J[a] = vj; m.J[b] = vj; m.K[a] = vk; m.K[b] = vk;
            continue;
        }
        if (i == j) { m.J[a] *= 2.0; m.K[a] *= 2.0; continue; }
        const double vj = m.J[a] + m.J[b], vk = m.K[a] + m.K[b];
        m.J[a] = vj; m.J[b] = vj; m.K[a] = vk; m.K[b] = vk;
    }
}

__global__ void k_absmax_batched(const gb::BatchMol* bm, unsigned long long* out) {
    const gb::BatchMol& m = bm[blockIdx.y];
    const long long n2 = (long long)m.nbf * m.nbf;
    double v = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
        const double x = m.D[i];
        v = fmax(v, fabs(x));
        m.Df[i] = (float)x;  // FP32 copy for the digestion of FP32 quartets
        if (m.Ddf) m.Ddf[i] = gb::dfl((float)x, (float)(x - (double)(float)x));
    }
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + blockIdx.y, (unsigned long long)__double_as_longlong(v));
}

// Max |D| per shell block of every molecule (grid.y = molecule).
__global__ void k_dsh_batched(const gb::BatchMol* bm) {
    const gb::BatchMol& m = bm[blockIdx.y];
    const int n = m.nbf;
    const long long n2 = (long long)n * n;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n2; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / n), j = (int)(k - (long long)i * n);
        atomicMax(reinterpret_cast<unsigned int*>(m.Dsh) + (size_t)m.bf_shell[i] * m.nshell + m.bf_shell[j],
                  __float_as_uint((float)fabs(m.D[k])));
    }
}

int build_plan(BatchPlan& P, cudaStream_t st) {
    const int nmol = (int)P.mols.size();
    int rc;
    std::vector<gb::BatchMol> host(nmol);
    P.max_n = 0;
    P.nquartets = 0;
    for (int m = 0; m < nmol; ++m) {
        jk_pairs_s* h = P.mols[m];
        if (h->device != P.device) return fail(JK_ERR_INVALID, "batched molecules on different devices");
        host[m].pairs = view_of(h);
        host[m].D = P.D[m];
        if (P.prec == JK_MIXED && (rc = h->Df.alloc(sizeof(float) * (size_t)h->nbf * h->nbf))) return rc;
        if (P.prec == JK_MIXED && (rc = h->Dsh.alloc(sizeof(float) * (size_t)h->nshell * h->nshell))) return rc;
        if (P.prec == JK_MIXED && P.df && (rc = h->Ddf.alloc(sizeof(float2) * (size_t)h->nbf * h->nbf))) return rc;
        host[m].Df = h->Df.as<float>();
        host[m].Ddf = P.df ? h->Ddf.as<gb::dfl>() : nullptr;
        host[m].Dsh = h->Dsh.as<float>();
        host[m].bf_shell = h->bf_shell.as<int>();
        host[m].psh = h->pair_sh.as<int2>();
        host[m].nshell = h->nshell;
        host[m].J = P.J[m];
        host[m].K = P.K[m];
        if (P.prec == JK_FP64) {  // compensated accumulation, as jk_build
            const size_t n2 = (size_t)h->nbf * h->nbf;
            if ((rc = h->Jlo.alloc(sizeof(double) * n2))) return rc;
            if ((rc = h->Klo.alloc(sizeof(double) * n2))) return rc;
            host[m].Jlo = h->Jlo.as<double>();
            host[m].Klo = h->Klo.as<double>();
        }
        host[m].nbf = h->nbf;
        P.max_n = std::max(P.max_n, h->nbf);
        P.nquartets += h->nquartets;
    }
    if ((rc = upload(P.bm, host.data(), nmol, st))) return rc;
    if ((rc = P.dmax.alloc(sizeof(unsigned long long) * nmol))) return rc;
    const int ncls = gb_num_pair_classes();
    P.cls.clear();
    P.cls.reserve(ncls * (ncls + 1) / 2);
    for (int X = 0; X < ncls; ++X)
        for (int Y = 0; Y <= X; ++Y) {
            int nrows = 0;
            long long total = 0;
            const ClassRows* first = nullptr;
            for (int m = 0; m < nmol; ++m)
                for (const ClassRows& cr : P.mols[m]->rows)
                    if (cr.bra_cls == X && cr.ket_cls == Y && cr.total > 0) {
                        nrows += cr.nrows;
                        total += cr.total;
                        if (!first) first = &cr;
                    }
            if (total == 0) continue;
            P.cls.emplace_back();
            BatchClass& bc = P.cls.back();
            bc.X = X; bc.Y = Y; bc.nrows = nrows; bc.total = total;
            bc.tune[0] = first->tune[0];
            bc.tune[1] = first->tune[1];
            if ((rc = bc.start.alloc(sizeof(long long) * (nrows + 1)))) return rc;
            if ((rc = bc.bra.alloc(sizeof(int) * nrows))) return rc;
            if ((rc = bc.ket0.alloc(sizeof(int) * nrows))) return rc;
            if ((rc = bc.rowmol.alloc(sizeof(int) * nrows))) return rc;
            int roff = 0;
            long long qoff = 0;
            for (int m = 0; m < nmol; ++m)
                for (const ClassRows& cr : P.mols[m]->rows)
                    if (cr.bra_cls == X && cr.ket_cls == Y && cr.total > 0) {
                        CK(cudaMemcpyAsync(bc.bra.as<int>() + roff, cr.bra.p, sizeof(int) * cr.nrows,
                                           cudaMemcpyDeviceToDevice, st));
                        CK(cudaMemcpyAsync(bc.ket0.as<int>() + roff, cr.ket0.p, sizeof(int) * cr.nrows,
                                           cudaMemcpyDeviceToDevice, st));
                        k_offset_copy<<<nblk(cr.nrows, 256), 256, 0, st>>>(cr.start.as<long long>(), cr.nrows, qoff,
                                                                            bc.start.as<long long>() + roff);
                        k_fill_int<<<nblk(cr.nrows, 256), 256, 0, st>>>(bc.rowmol.as<int>() + roff, cr.nrows, m);
                        CKL();
                        roff += cr.nrows;
                        qoff += cr.total;
                    }
            k_set_ll<<<1, 1, 0, st>>>(bc.start.as<long long>() + nrows, total);
            CKL();
            {   // work items of the FP64 launch
                DevBuf w;
                if ((rc = w.alloc(sizeof(long long) * (nrows + 1)))) return rc;
                if ((rc = bc.istart.alloc(sizeof(long long) * (nrows + 1)))) return rc;
                if ((rc = bc.itot.alloc(sizeof(long long)))) return rc;
                CK(cudaMemsetAsync(w.as<long long>() + nrows, 0, sizeof(long long), st));
                k_row_items<<<nblk(nrows, 256), 256, 0, st>>>(bc.start.as<long long>(), bc.bra.as<int>(), nrows, nullptr,
                                                              P.bm.as<gb::BatchMol>(), bc.rowmol.as<int>(),
                                                              gb_class_split(X, Y), w.as<long long>());
                CKL();
                if ((rc = scan_exclusive(w.as<long long>(), bc.istart.as<long long>(), nrows + 1, bc.itot.as<long long>(),
                                         st)))
                    return rc;
            }
            if (P.prec == JK_MIXED) {
                const long long n1 = nrows + 1;
                if ((rc = bc.c64.alloc(sizeof(long long) * n1))) return rc;
                if ((rc = bc.c32.alloc(sizeof(long long) * n1))) return rc;
                if ((rc = bc.w64.alloc(sizeof(long long) * n1))) return rc;
                if ((rc = bc.w32.alloc(sizeof(long long) * n1))) return rc;
                for (DevBuf* b : {&bc.cdem, &bc.wdem, &bc.sdem, &bc.l64, &bc.ldem})
                    if ((rc = b->alloc(sizeof(long long) * n1))) return rc;
                if ((rc = bc.s64.alloc(sizeof(long long) * n1))) return rc;
                if ((rc = bc.s32.alloc(sizeof(long long) * n1))) return rc;
                if ((rc = bc.k32.alloc(sizeof(int) * nrows))) return rc;
                if ((rc = bc.scr.alloc(sizeof(long long) * (scan_scratch_len(n1) + 1)))) return rc;
            }
        }
    if ((rc = P.split_tot.alloc(sizeof(long long) * kSplitSlots * std::max<size_t>(1, P.cls.size())))) return rc;
    CK(cudaStreamSynchronize(st));
    CK(cudaStreamCreateWithFlags(&P.cs, cudaStreamNonBlocking));
    for (auto& x : P.ps) CK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming));
    for (auto& e : P.join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&P.done, cudaEventDisableTiming));
    return 0;
}

int launch_batch_class(BatchPlan& P, BatchClass& bc, int prec, const long long* start, const int* ket0,
                       cudaStream_t s, const long long* kofs = nullptr, const int* klist = nullptr, int pmode = 0,
                       const float* kthr = nullptr) {
    gb::JKArgs a;
    std::memset(&a, 0, sizeof(a));
    a.pairs = view_of(P.mols[0]);
    a.rows.nrows = bc.nrows;
    a.rows.start = start;
    a.rows.bra = bc.bra.as<int>();
    a.rows.ket0 = ket0;
    a.rows.kofs = kofs;
    a.rows.klist = klist;
    a.rows.kthr = kthr;
    a.pmode = (klist && kthr) ? pmode : 0;
    a.boys = g_boys[P.device].tab.as<double>();
    a.boysf = g_boys[P.device].tabf.as<float>();
    a.boysd = g_boys[P.device].tabd.as<float2>();
    a.tsmall = (float)P.tsmall;
    a.mols = P.bm.as<gb::BatchMol>();
    a.row_mol = bc.rowmol.as<int>();
    const TuneCfg& tc = bc.tune[prec == 3 ? 0 : prec];
    int nsm = P.mols[0]->nsm;
    const long long items = bc.total * gb_class_split(bc.X, bc.Y) * gb_class_threads(bc.X, bc.Y, prec == 3 ? 0 : prec);
    const int e = gb_launch_jk(bc.X, bc.Y, prec == 1 && P.rpath ? 2 : prec, a, grid_for(items, tc.block, tc.qpt, nsm),
                               tc.block, s);
    if (e) return fail(JK_ERR_CUDA, std::string("batched ERI launch: ") + cudaGetErrorString((cudaError_t)e));
    P.launches += 1;
    return 0;
}

// The launch sequence of one batched build, on stream cs (forking to ps[]).
int enqueue_batch(BatchPlan& P) {
    const int nmol = (int)P.mols.size();
    int rc;
    P.launches = 0;
    const gb::BatchMol* bm = P.bm.as<gb::BatchMol>();
    const long long n2max = (long long)P.max_n * P.max_n;
    k_zero_batched<<<dim3(nblk(n2max, 256), nmol), 256, 0, P.cs>>>(bm);
    CKL();
    P.launches += 1;
    CK(cudaEventRecord(P.fork, P.cs));
    for (auto& x : P.ps) CK(cudaStreamWaitEvent(x, P.fork, 0));
    for (size_t k = 0; k < P.cls.size(); ++k) {
        BatchClass& bc = P.cls[k];
        cudaStream_t s = (k % 4 == 0) ? P.cs : P.ps[k % 4 - 1];
        if (P.prec == JK_FP64) {
            if ((rc = launch_batch_class(P, bc, 0, bc.istart.as<long long>(), bc.ket0.as<int>(), s))) return rc;
        } else {
            // counts come from the pre-pass (batch_prepass); scans, list fill, launches
            const long long n1 = bc.nrows + 1;
            long long* tot = P.split_tot.as<long long>() + kSplitSlots * k;
            long long* scr = bc.scr.as<long long>();
            if ((rc = scan_into(bc.w32.as<long long>(), bc.s32.as<long long>(), n1, tot + 2, scr, s))) return rc;
            if ((rc = scan_into(bc.w64.as<long long>(), bc.s64.as<long long>(), n1, tot + 3, scr, s))) return rc;
            if ((rc = scan_into(bc.wdem.as<long long>(), bc.sdem.as<long long>(), n1, tot + 4, scr, s))) return rc;
            if ((rc = scan_into(bc.c64.as<long long>(), bc.l64.as<long long>(), n1, tot + 5, scr, s))) return rc;
            if ((rc = scan_into(bc.cdem.as<long long>(), bc.ldem.as<long long>(), n1, tot + 6, scr, s))) return rc;
            int* l64 = P.list64.as<int>() + bc.off64;
            int* ldm = P.listdem.as<int>() + bc.offdem;
            float* t64 = P.ptau > 0.0 ? P.thr64.as<float>() + bc.off64 : nullptr;
            k_rows_fill_batched<<<nblk(bc.nrows, 256), 256, 0, s>>>(bc.bra.as<int>(), bc.ket0.as<int>(), bc.k32.as<int>(),
                                                                    bc.rowmol.as<int>(), bc.nrows, bm, P.tau, P.eps,
                                                                    bc.l64.as<long long>(), bc.ldem.as<long long>(),
                                                                    l64, ldm, (float)P.ptau, t64);
            CKL();
            P.launches += 1 + 5 * scan_launches(n1);
            if ((rc = launch_batch_class(P, bc, P.df ? 3 : 0, bc.s64.as<long long>(), nullptr, s, bc.l64.as<long long>(),
                                         l64, 1, t64)))
                return rc;
            if (t64 && (rc = launch_batch_class(P, bc, 1, bc.s64.as<long long>(), nullptr, s, bc.l64.as<long long>(),
                                                l64, 2, t64)))
                return rc;
            if ((rc = launch_batch_class(P, bc, 1, bc.s32.as<long long>(), bc.k32.as<int>(), s))) return rc;
            if ((rc = launch_batch_class(P, bc, 1, bc.sdem.as<long long>(), nullptr, s, bc.ldem.as<long long>(), ldm)))
                return rc;
        }
    }
    for (int i = 0; i < 3; ++i) {
        CK(cudaEventRecord(P.join[i], P.ps[i]));
        CK(cudaStreamWaitEvent(P.cs, P.join[i], 0));
    }
    const long long trimax = (long long)P.max_n * (P.max_n + 1) / 2;
    k_sym_batched<<<dim3(nblk(trimax, 256), nmol), 256, 0, P.cs>>>(bm);
    CKL();
    P.launches += 1;
    return 0;
}

// Mixed batched builds, before the (captured) launch sequence: max|D| and the
// FP32 copy of D, the shell-block maxima of D, and the per-row split counts of
// every class; then one host synchronisation reads the list sizes.  If a
// class's lists outgrow their segments, the lists are re-laid out (*relaid) and
// a captured graph must be captured again.
int batch_prepass(BatchPlan& P, bool* relaid) {
    const int nmol = (int)P.mols.size();
    const gb::BatchMol* bm = P.bm.as<gb::BatchMol>();
    *relaid = false;
    const size_t nst = (size_t)kSplitSlots * std::max<size_t>(1, P.cls.size());
    CK(cudaMemsetAsync(P.dmax.p, 0, sizeof(unsigned long long) * nmol, P.cs));
    CK(cudaMemsetAsync(P.split_tot.p, 0, sizeof(long long) * nst, P.cs));
    k_absmax_batched<<<dim3(64, nmol), 256, 0, P.cs>>>(bm, P.dmax.as<unsigned long long>());
    CKL();
    for (jk_pairs h : P.mols) CK(cudaMemsetAsync(h->Dsh.p, 0, sizeof(float) * (size_t)h->nshell * h->nshell, P.cs));
    const long long n2max = (long long)P.max_n * P.max_n;
    k_dsh_batched<<<dim3((unsigned)std::min<long long>(nblk(n2max, 256), 1024), nmol), 256, 0, P.cs>>>(bm);
    CKL();
    for (size_t k = 0; k < P.cls.size(); ++k) {
        BatchClass& bc = P.cls[k];
        k_rows_split_batched<<<nblk(bc.nrows, 256), 256, 0, P.cs>>>(
            bc.start.as<long long>(), bc.bra.as<int>(), bc.ket0.as<int>(), bc.rowmol.as<int>(), bc.nrows, bm,
            P.dmax.as<unsigned long long>(), P.tau, P.eps, gb_class_split(bc.X, bc.Y), bc.c64.as<long long>(),
            bc.cdem.as<long long>(), bc.c32.as<long long>(), bc.k32.as<int>(), bc.w64.as<long long>(),
            bc.wdem.as<long long>(), bc.w32.as<long long>(),
            reinterpret_cast<unsigned long long*>(P.split_tot.as<long long>() + kSplitSlots * k));
        CKL();
        for (DevBuf* b : {&bc.c64, &bc.c32, &bc.cdem, &bc.w64, &bc.w32, &bc.wdem})
            CK(cudaMemsetAsync(b->as<long long>() + bc.nrows, 0, 8, P.cs));
    }
    std::vector<long long> cnt(nst);
    CK(cudaMemcpyAsync(cnt.data(), P.split_tot.p, sizeof(long long) * nst, cudaMemcpyDeviceToHost, P.cs));
    CK(cudaStreamSynchronize(P.cs));
    bool grow = false;
    for (size_t k = 0; k < P.cls.size(); ++k)
        grow = grow || cnt[kSplitSlots * k + 1] > P.cls[k].cap64 || cnt[kSplitSlots * k + 7] > P.cls[k].capdem;
    if (grow) {  // new segments with 25 % headroom
        long long o64 = 0, od = 0;
        for (size_t k = 0; k < P.cls.size(); ++k) {
            BatchClass& bc = P.cls[k];
            bc.cap64 = std::max(bc.cap64, cnt[kSplitSlots * k + 1] + cnt[kSplitSlots * k + 1] / 4 + 1024);
            bc.capdem = std::max(bc.capdem, cnt[kSplitSlots * k + 7] + cnt[kSplitSlots * k + 7] / 4 + 1024);
            bc.off64 = o64;
            bc.offdem = od;
            o64 += bc.cap64;
            od += bc.capdem;
        }
        int rc;
        if ((rc = P.list64.alloc(sizeof(int) * o64))) return rc;
        if ((rc = P.listdem.alloc(sizeof(int) * od))) return rc;
        if (P.ptau > 0.0 && (rc = P.thr64.alloc(sizeof(float) * o64))) return rc;
        *relaid = true;
    }
    return 0;
}

int capture_batch(BatchPlan& P) {
    if (P.exec) {
        cudaGraphExecDestroy(P.exec);
        P.exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(P.cs, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_batch(P);
    const cudaError_t ce = cudaStreamEndCapture(P.cs, &graph);
    if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (ce != cudaSuccess) return fail(JK_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(&P.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return fail(JK_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    return 0;
}

int batched_impl(int nmol, const jk_pairs* pairs, const double* const* D, double* const* J, double* const* K,
                 jk_precision prec, cudaStream_t st, long long* launches) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    int dev = -1;
    CK(cudaGetDevice(&dev));
    bool same = g_plan && g_plan->device == dev && (int)g_plan->mols.size() == nmol && g_plan->prec == (int)prec &&
                g_plan->tau == g_opt.tau && g_plan->eps == g_opt.eps && g_plan->tsmall == g_opt.tsmall && g_plan->graph == g_opt.graph &&
                g_plan->rpath == g_opt.rpath && g_plan->df == g_opt.df_tier && g_plan->ptau == g_opt.ptau;
    for (int m = 0; same && m < nmol; ++m)
        same = g_plan->mols[m] == pairs[m] && g_plan->serial[m] == pairs[m]->serial && g_plan->D[m] == D[m] &&
               g_plan->J[m] == J[m] && g_plan->K[m] == K[m];
    int rc;
    if (!same) {
        g_plan.reset(new BatchPlan());
        BatchPlan& P = *g_plan;
        P.mols.assign(pairs, pairs + nmol);
        for (int m = 0; m < nmol; ++m) P.serial.push_back(pairs[m]->serial);
        P.D.assign(D, D + nmol);
        P.J.assign(J, J + nmol);
        P.K.assign(K, K + nmol);
        P.prec = prec;
        P.device = dev;
        P.tau = g_opt.tau;
        P.eps = g_opt.eps;
        P.tsmall = g_opt.tsmall;
        P.graph = g_opt.graph;
        P.rpath = g_opt.rpath;
        P.df = g_opt.df_tier;
        P.ptau = g_opt.ptau;
        if ((rc = build_plan(P, st))) { g_plan.reset(); return rc; }
    }
    BatchPlan& P = *g_plan;
    // order the batch after the caller's prior work on st, and st after the batch
    CK(cudaEventRecord(P.done, st));
    CK(cudaStreamWaitEvent(P.cs, P.done, 0));
    bool relaid = false;
    if (P.prec == JK_MIXED && (rc = batch_prepass(P, &relaid))) { g_plan.reset(); return rc; }
    const long long pre = P.prec == JK_MIXED ? 3 + (long long)P.cls.size() : 0;  // pre-pass kernels
    if (P.graph) {
        if ((!P.exec || relaid) && (rc = capture_batch(P))) { g_plan.reset(); return rc; }
        CK(cudaGraphLaunch(P.exec, P.cs));
    } else {
        if ((rc = enqueue_batch(P))) return rc;
    }
    P.launches_total = P.launches + pre;
    CK(cudaEventRecord(P.done, P.cs));
    CK(cudaStreamWaitEvent(st, P.done, 0));
    if (launches) *launches = P.launches_total;
    return 0;
}

// ------------------------------------------------------------------ autotuner
// Algorithm 2 of the paper (Workload Allocator): start every class at one
// quartet per thread, then repeatedly try "Combine" (double the quartets per
// thread, i.e. halve the grid) and keep it only if the class got faster; stop
// when no class improves.  Timed on a prefix of each class's rows (about an
// eighth, at least 2^21 quartets) with CUDA events; J and K are scratch.
int autotune_impl(jk_pairs_s* h, const double* D, double* J, double* K, int prec, cudaStream_t st) {
    if (prec == 1) {  // the FP32 kernels digest with the FP32 copy of D
        int rc;
        const long long n2 = (long long)h->nbf * h->nbf;
        if ((rc = h->Df.alloc(sizeof(float) * n2))) return rc;
        if ((rc = h->scratch.alloc(64))) return rc;
        CK(cudaMemsetAsync(h->scratch.p, 0, 8, st));
        k_absmax<<<152 * 4, 256, 0, st>>>(D, n2, h->scratch.as<unsigned long long>(), h->Df.as<float>());
        CKL();
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    struct Item { ClassRows* cr; int nrows; long long total; };
    std::vector<Item> items;
    for (ClassRows& cr : h->rows) {
        if (cr.total <= 0) continue;
        std::vector<long long> start(cr.nrows + 1);
        CK(cudaMemcpy(start.data(), cr.istart.p, sizeof(long long) * (cr.nrows + 1), cudaMemcpyDeviceToHost));
        const long long target = std::max<long long>(cr.itotal / 8, 1LL << 21);
        int r = (int)(std::lower_bound(start.begin(), start.end(), target) - start.begin());
        r = std::min(std::max(r, 1), cr.nrows);
        items.push_back({&cr, r, start[r]});
        cr.tune[prec] = TuneCfg();
    }
    auto time_one = [&](const Item& it, float* ms) -> int {
        int rc;
        for (int rep = 0; rep < 2; ++rep) {  // first run warms caches and clocks
            CK(cudaEventRecord(e0, st));
            if ((rc = launch_class(h, *it.cr, prec, it.cr->istart.as<long long>(), it.cr->ket0.as<int>(), it.total, D,
                                   J, K, st, it.nrows)))
                return rc;
            CK(cudaEventRecord(e1, st));
        }
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(ms, e0, e1));
        return 0;
    };
    bool improved = true;
    int rounds = 0;
    while (improved && rounds < 8) {
        improved = false;
        ++rounds;
        for (Item& it : items) {
            TuneCfg& tc = it.cr->tune[prec];
            if (grid_for(it.total, tc.block, tc.qpt * 2, h->nsm) < h->nsm) continue;  // keep one wave
            float t1 = 0.f, t2 = 0.f;
            int rc;
            if ((rc = time_one(it, &t1))) return rc;
            tc.qpt *= 2;  // Combine
            if ((rc = time_one(it, &t2))) return rc;
            if (t2 < t1) improved = true;
            else tc.qpt /= 2;  // Revert
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->tuned[prec] = 1;
    drop_plan_of(h);
    return 0;
}

template <int L>
__global__ void k_boys_eval(int n, const double* T, double* F, int prec, const double* tab, const float* tabf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (prec == 0) {
        double f[L + 1];
        gb::boys_f64<L>(T[i], f, tab);
        for (int m = 0; m <= L; ++m) F[(size_t)i * (L + 1) + m] = f[m];
    } else {
        float f[L + 1];
        gb::boys_f32<L>((float)T[i], f, tabf);
        for (int m = 0; m <= L; ++m) F[(size_t)i * (L + 1) + m] = f[m];
    }
}

template <int L>
int boys_launch(int n, const double* T, double* F, int prec, int dev, cudaStream_t st) {
    k_boys_eval<L><<<nblk(n, 128), 128, 0, st>>>(n, T, F, prec, g_boys[dev].tab.as<double>(), g_boys[dev].tabf.as<float>());
    CKL();
    return 0;
}

// Dependent FMA chains: 8 independent accumulators per thread (enough to cover
// the pipe latency), `iters` rounds each.
template <class T>
__global__ void k_fma_peak(int iters, T* sink) {
    T a0 = (T)threadIdx.x * (T)1e-3, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
    T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
    const T m = (T)0.999999, c = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            a0 = a0 * m + c; a1 = a1 * m + c; a2 = a2 * m + c; a3 = a3 * m + c;
            a4 = a4 * m + c; a5 = a5 * m + c; a6 = a6 * m + c; a7 = a7 * m + c;
        }
    }
    const T r = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (r == (T)-12345) *sink = r;  // keeps the chains alive
}

// ------------------------------------------------------------------ pure shells
// Device data of the Cartesian <-> pure transform, uploaded on first use: per
// shell (l, first Cartesian index, first pure index), the owning shell of
// every pure basis function, and the coefficient tables of the generated
// sph_table.cu.  The Cartesian owners are the handle's bf_shell.
int sph_prepare(jk_pairs_s* h, cudaStream_t st) {
    if (h->sph_ready) return 0;
    const double* coef = nullptr;
    const int* off = nullptr;
    const int lmax = gb_sph_table(&coef, &off);
    if (lmax < gb::kSphLmax) return fail(JK_ERR_UNSUPPORTED, "pure-shell table stops below l = 3");
    std::vector<int4> sh(h->nshell);
    std::vector<int> owner(h->nsph);
    int c = 0, p = 0;
    for (int s = 0; s < h->nshell; ++s) {
        const int l = h->shell_l[s];
        const int np = l >= 2 ? 2 * l + 1 : (l + 1) * (l + 2) / 2;
        sh[s] = make_int4(l, c, p, off[l]);
        for (int k = 0; k < np; ++k) owner[p + k] = s;
        c += (l + 1) * (l + 2) / 2;
        p += np;
    }
    if (c != h->nbf || p != h->nsph) return fail(JK_ERR_INVALID, "pure-shell layout does not match the handle");
    int rc;
    if ((rc = upload(h->sph_shell, sh.data(), sh.size(), st))) return rc;
    if ((rc = upload(h->sph_owner, owner.data(), owner.size(), st))) return rc;
    if ((rc = upload(h->sph_coef, coef, (size_t)off[gb::kSphLmax + 1], st))) return rc;
    h->sph_ready = true;
    return 0;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* jk_last_error(void) { return g_err.c_str(); }

int shellpairs_build(const jk_atoms* atoms, const jk_shells* shells, double thresh, jk_pairs* out, void* cuda_stream) {
    g_err.clear();
    if (!atoms || !shells || !out) return fail(JK_ERR_INVALID, "null argument");
    *out = nullptr;
    if (atoms->natom <= 0 || !atoms->xyz) return fail(JK_ERR_INVALID, "no atoms");
    if (shells->nshell <= 0 || !shells->atom || !shells->l || !shells->nprim || !shells->prim_offset || !shells->exps ||
        !shells->coefs)
        return fail(JK_ERR_INVALID, "no shells");
    if (!std::isfinite(thresh)) return fail(JK_ERR_INVALID, "threshold not finite");
    jk_pairs_s* h = new (std::nothrow) jk_pairs_s();
    if (!h) return fail(JK_ERR_NOMEM, "host allocation");
    const int rc = build_impl(atoms, shells, thresh, h, static_cast<cudaStream_t>(cuda_stream));
    if (rc) {
        delete h;
        return rc;
    }
    h->serial = ++g_serial;
    *out = h;
    return JK_OK;
}

int shellpairs_info(jk_pairs h, int* nbf, int64_t* npairs, int64_t* nquartets, int64_t* nprimq) {
    if (!h) return fail(JK_ERR_INVALID, "null handle");
    if (nbf) *nbf = h->nbf;
    if (npairs) *npairs = h->npair;
    if (nquartets) *nquartets = h->nquartets;
    if (nprimq) *nprimq = h->nprimq;
    return JK_OK;
}

int jk_build(jk_pairs h, const double* D, double* J, double* K, jk_precision prec, void* cuda_stream) {
    g_err.clear();
    if (!h || !D || !J || !K) return fail(JK_ERR_INVALID, "null argument");
    if (prec != JK_FP64 && prec != JK_MIXED) return fail(JK_ERR_INVALID, "precision");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != h->device) return fail(JK_ERR_INVALID, "handle belongs to another device");
    return jk_build_impl(h, D, J, K, prec, static_cast<cudaStream_t>(cuda_stream));
}

int jk_energy(int nbf, const double* D, const double* J, const double* K, double* E, void* cuda_stream) {
    g_err.clear();
    if (nbf <= 0 || !D || !J || !K || !E) return fail(JK_ERR_INVALID, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int nb = 152 * 2;
    DevBuf part, out;
    int rc;
    if ((rc = part.alloc(sizeof(double2) * nb))) return rc;
    if ((rc = out.alloc(sizeof(double)))) return rc;
    k_energy_partial<<<nb, 256, 0, st>>>(D, J, K, (long long)nbf * nbf, part.as<double2>());
    CKL();
    k_energy_final<<<1, 32, 0, st>>>(part.as<double2>(), nb, out.as<double>());
    CKL();
    CK(cudaMemcpyAsync(E, out.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return JK_OK;
}

int jk_energy_noalloc(int nbf, const double* D, const double* J, const double* K, double* E, void* cuda_stream) {
    g_err.clear();
    if (nbf <= 0 || !D || !J || !K || !E) return fail(JK_ERR_INVALID, "bad argument");
    if (nbf > kNoAllocMaxRows)
        return fail(JK_ERR_INVALID, "jk_energy_noalloc: nbf = " + std::to_string(nbf) + " exceeds the fixed scratch (" +
                                        std::to_string(kNoAllocMaxRows) + " rows); use jk_energy");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double2* scratch = nullptr;
    int rc;
    if ((rc = noalloc_scratch(&scratch))) return rc;
    const int rows_per_block = 8;  // 256 threads = 8 warps = 8 rows
    k_energy_rows<<<nblk(nbf, rows_per_block), 256, 0, st>>>(D, J, K, nbf, scratch);
    CKL();
    k_energy_rows_final<<<1, 256, 0, st>>>(scratch, nbf, scratch + kNoAllocMaxRows);
    CKL();
    CK(cudaMemcpyAsync(E, scratch + kNoAllocMaxRows, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return JK_OK;
}

int jk_grad(jk_pairs h, const double* D, double* dEdR, jk_precision prec, void* cuda_stream) {
    return jk_grad_part(h, 0, 1, D, dEdR, prec, cuda_stream);
}

int jk_grad_part(jk_pairs h, int part, int nparts, const double* D, double* dEdR, jk_precision prec,
                 void* cuda_stream) {
    g_err.clear();
    if (!h || !D || !dEdR) return fail(JK_ERR_INVALID, "null argument");
    if (prec != JK_FP64 && prec != JK_MIXED) return fail(JK_ERR_INVALID, "precision");
    if (nparts < 1 || part < 0 || part >= nparts) return fail(JK_ERR_INVALID, "part outside [0, nparts)");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != h->device) return fail(JK_ERR_INVALID, "handle belongs to another device");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    {
        const int gl = gb_grad_lmax(), gcls = (gl + 1) * (gl + 2) / 2;
        for (const ClassRows& cr : h->rows)
            if (cr.total > 0 && cr.bra_cls >= gcls)
                return fail(JK_ERR_UNSUPPORTED, "gradients are compiled for shells up to l = " + std::to_string(gl));
    }
    int rc;
    if (nparts > 1 && (rc = ensure_partition(h, nparts, st))) return rc;
    const int ncr = (int)h->rows.size();
    std::vector<int> R0(ncr), R1(ncr);
    std::vector<long long> items(ncr);
    for (int k = 0; k < ncr; ++k) {
        R0[k] = nparts > 1 ? h->part_rows[k][part] : 0;
        R1[k] = nparts > 1 ? h->part_rows[k][part + 1] : h->rows[k].nrows;
        items[k] = nparts > 1 ? h->part_items[k][part + 1] - h->part_items[k][part] : h->rows[k].itotal;
    }
    CK(cudaMemsetAsync(dEdR, 0, sizeof(double) * 3 * h->natom, st));
    h->launches = 0;
    // one launch over rows [r0, r1) of a class: per-row item prefix `start`,
    // contiguous kets from ket0 or explicit ones (kofs/klist)
    auto launch = [&](int k, int kp, const long long* start, const int* ket0, const long long* kofs, const int* klist,
                      int pmode = 0, const float* kthr = nullptr) {
        const ClassRows& cr = h->rows[k];
        const int r0 = R0[k], nr = R1[k] - R0[k];
        gb::GradArgs a;
        std::memset(&a, 0, sizeof(a));
        a.pairs = view_of(h);
        a.rows.nrows = nr;
        a.rows.start = start + r0;
        a.rows.bra = cr.bra.as<int>() + r0;
        a.rows.ket0 = ket0 ? ket0 + r0 : nullptr;
        a.rows.kofs = kofs ? kofs + r0 : nullptr;
        a.rows.klist = klist;
        a.rows.kthr = kthr;
        a.pmode = (klist && kthr) ? pmode : 0;
        a.boys = g_boys[h->device].tab.as<double>();
        a.boysf = g_boys[h->device].tabf.as<float>();
        a.tsmall = (float)g_opt.tsmall;
        a.D = D;
        a.nbf = h->nbf;
        a.atoms = h->pair_atoms.as<int2>();
        a.grad = dEdR;
        const int grid = grid_for(items[k] * gb_grad_threads(cr.bra_cls, cr.ket_cls), 128, 1, h->nsm);
        const int e = gb_launch_grad(cr.bra_cls, cr.ket_cls, kp, a, grid, st);
        if (e) return fail(JK_ERR_CUDA, std::string("gradient kernel launch: ") + cudaGetErrorString((cudaError_t)e));
        h->launches += 1;
        return 0;
    };
    if (prec == JK_FP64) {
        for (int k = 0; k < ncr; ++k) {
            const ClassRows& cr = h->rows[k];
            if (cr.total <= 0 || R1[k] <= R0[k] || items[k] <= 0) continue;
            if ((rc = launch(k, 0, cr.istart.as<long long>(), cr.ket0.as<int>(), nullptr, nullptr))) return rc;
        }
        return JK_OK;
    }
    // mixed: the J/K kernels' split with the gradient's cutoff -- derivative
    // integrals of the quartets whose density-weighted bound is below grad_tau
    // in FP32 (accumulated per item, added to dE/dR in FP64), the others FP64
    const int n = h->nbf;
    const size_t nst = (size_t)kSplitSlots * std::max(1, ncr);
    if ((rc = h->scratch.alloc(64))) return rc;
    if ((rc = h->split_tot.alloc(sizeof(long long) * nst))) return rc;
    CK(cudaMemsetAsync(h->split_tot.p, 0, sizeof(long long) * nst, st));
    CK(cudaMemsetAsync(h->scratch.p, 0, 8, st));
    k_absmax<<<152 * 4, 256, 0, st>>>(D, (long long)n * n, h->scratch.as<unsigned long long>(), nullptr);
    CKL();
    const size_t ns2 = (size_t)h->nshell * h->nshell;
    if ((rc = h->Dsh.alloc(sizeof(float) * ns2))) return rc;
    CK(cudaMemsetAsync(h->Dsh.p, 0, sizeof(float) * ns2, st));
    k_dsh<<<152 * 4, 256, 0, st>>>(D, n, h->bf_shell.as<int>(), h->nshell, h->Dsh.as<unsigned int>());
    CKL();
    const double* dmax = reinterpret_cast<const double*>(h->scratch.p);
    for (int k = 0; k < ncr; ++k)
        if (h->rows[k].total > 0 && R1[k] > R0[k] &&
            (rc = split_count(h, h->rows[k], R0[k], R1[k], dmax, h->split_tot.as<long long>() + kSplitSlots * k, st,
                              g_opt.grad_tau, 0.0)))
            return rc;
    std::vector<long long> cnt(nst);
    CK(cudaMemcpyAsync(cnt.data(), h->split_tot.p, sizeof(long long) * nst, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<long long> off64(ncr + 1, 0), offd(ncr + 1, 0);
    for (int k = 0; k < ncr; ++k) {
        off64[k + 1] = off64[k] + cnt[kSplitSlots * k + 1];
        offd[k + 1] = offd[k] + cnt[kSplitSlots * k + 7];
    }
    if ((rc = h->list64.alloc(sizeof(int) * std::max(1LL, off64[ncr])))) return rc;
    if ((rc = h->listdem.alloc(sizeof(int) * std::max(1LL, offd[ncr])))) return rc;
    const bool psplit = g_opt.grad_ptau > 0.0;
    if (psplit && (rc = h->thr64.alloc(sizeof(float) * std::max(1LL, off64[ncr])))) return rc;
    for (int k = 0; k < ncr; ++k) {
        ClassRows& cr = h->rows[k];
        if (cr.total <= 0 || R1[k] <= R0[k]) continue;
        int* l64 = h->list64.as<int>() + off64[k];
        int* ldm = h->listdem.as<int>() + offd[k];
        float* t64 = psplit ? h->thr64.as<float>() + off64[k] : nullptr;
        if ((rc = split_fill(h, cr, R0[k], R1[k], h->split_tot.as<long long>() + kSplitSlots * k, l64, ldm, st,
                             g_opt.grad_tau, 0.0, (float)g_opt.grad_ptau, t64)))
            return rc;
        // the large-bound quartets in FP64 (with the primitive split: their large primitive
        // quartets, the rest by the FP32 derivative kernels over the same list)
        if ((rc = launch(k, 0, cr.s64.as<long long>(), nullptr, cr.l64.as<long long>(), l64, 1, t64))) return rc;
        if (psplit && (rc = launch(k, 1, cr.s64.as<long long>(), nullptr, cr.l64.as<long long>(), l64, 2, t64)))
            return rc;
        if ((rc = launch(k, 1, cr.s32.as<long long>(), cr.k32.as<int>(), nullptr, nullptr))) return rc;
        if ((rc = launch(k, 1, cr.sdem.as<long long>(), nullptr, cr.ldem.as<long long>(), ldm))) return rc;
    }
    // the split diagnostics (jk_last_split, jk_split_stats) now describe this gradient
    h->last_psplit = psplit;
    h->list_off64 = off64;
    h->list_offd = offd;
    h->last_r0 = R0;
    h->last_r1 = R1;
    h->last_prec = JK_MIXED;
    return JK_OK;
}

int jk_build_part(jk_pairs h, int part, int nparts, const double* D, double* J, double* K, jk_precision prec,
                  void* cuda_stream) {
    g_err.clear();
    if (!h || !D || !J || !K) return fail(JK_ERR_INVALID, "null argument");
    if (prec != JK_FP64 && prec != JK_MIXED) return fail(JK_ERR_INVALID, "precision");
    if (nparts < 1 || part < 0 || part >= nparts) return fail(JK_ERR_INVALID, "part outside [0, nparts)");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != h->device) return fail(JK_ERR_INVALID, "handle belongs to another device");
    return jk_build_impl(h, D, J, K, prec, static_cast<cudaStream_t>(cuda_stream), part, nparts);
}

int jk_partition(int64_t n, const double* cost, int nparts, int64_t* bounds) {
    g_err.clear();
    static_assert(sizeof(int64_t) == sizeof(long long), "int64_t is long long");
    return partition_costs((long long)n, cost, nparts, reinterpret_cast<long long*>(bounds));
}

int jk_part_rows(jk_pairs h, int nparts, int max_rows, int64_t* rows, int* nrows) {
    g_err.clear();
    if (!h || !nrows || nparts < 1 || (max_rows > 0 && !rows)) return fail(JK_ERR_INVALID, "bad argument");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != h->device) return fail(JK_ERR_INVALID, "handle belongs to another device");
    int rc;
    if ((rc = ensure_partition(h, nparts, nullptr))) return rc;
    int k = 0;
    for (size_t ci = 0; ci < h->rows.size(); ++ci) {
        const ClassRows& cr = h->rows[ci];
        if (cr.total <= 0) continue;
        for (int p = 0; p < nparts; ++p, ++k) {
            if (k >= max_rows) continue;
            int64_t* r = rows + 8 * k;
            r[0] = cr.bra_cls; r[1] = cr.ket_cls; r[2] = p;
            r[3] = h->part_rows[ci][p];
            r[4] = h->part_rows[ci][p + 1];
            r[5] = h->part_items[ci][p + 1] - h->part_items[ci][p];
            r[6] = (int64_t)h->part_cost[ci][p];
            r[7] = (int64_t)h->part_cost[ci][nparts];
        }
    }
    *nrows = k;
    return JK_OK;
}

int jk_build_batched(int nmol, const jk_pairs* pairs, const double* const* D, double* const* J, double* const* K,
                     jk_precision prec, void* cuda_stream) {
    g_err.clear();
    if (nmol < 0 || (nmol > 0 && (!pairs || !D || !J || !K))) return fail(JK_ERR_INVALID, "bad argument");
    if (prec != JK_FP64 && prec != JK_MIXED) return fail(JK_ERR_INVALID, "precision");
    if (nmol == 0) return JK_OK;
    for (int i = 0; i < nmol; ++i)
        if (!pairs[i] || !D[i] || !J[i] || !K[i]) return fail(JK_ERR_INVALID, "null molecule entry");
    long long launches = 0;
    const int rc = batched_impl(nmol, pairs, D, J, K, prec, static_cast<cudaStream_t>(cuda_stream), &launches);
    if (!rc) pairs[0]->launches = launches;
    return rc;
}

int jk_boys(int L, int n, const double* T, double* F, jk_precision prec, void* cuda_stream) {
    g_err.clear();
    if (L < 0 || L > gb::kLmaxBoys || n < 0 || (n > 0 && (!T || !F))) return fail(JK_ERR_INVALID, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, rc;
    CK(cudaGetDevice(&dev));
    if ((rc = ensure_boys(dev, st))) return rc;
    if (n == 0) return JK_OK;
    const int p = prec == JK_FP64 ? 0 : 1;
    switch (L) {
        case 0: return boys_launch<0>(n, T, F, p, dev, st);
        case 1: return boys_launch<1>(n, T, F, p, dev, st);
        case 2: return boys_launch<2>(n, T, F, p, dev, st);
        case 3: return boys_launch<3>(n, T, F, p, dev, st);
        case 4: return boys_launch<4>(n, T, F, p, dev, st);
        case 5: return boys_launch<5>(n, T, F, p, dev, st);
        case 6: return boys_launch<6>(n, T, F, p, dev, st);
        case 7: return boys_launch<7>(n, T, F, p, dev, st);
        case 8: return boys_launch<8>(n, T, F, p, dev, st);
        case 9: return boys_launch<9>(n, T, F, p, dev, st);
        case 10: return boys_launch<10>(n, T, F, p, dev, st);
        case 11: return boys_launch<11>(n, T, F, p, dev, st);
        case 12: return boys_launch<12>(n, T, F, p, dev, st);
        default: return boys_launch<13>(n, T, F, p, dev, st);
    }
}

int jk_set_option(jk_option opt, double v) {
    switch (opt) {
        case JK_OPT_MIXED_TAU: if (!(v >= 0)) return fail(JK_ERR_INVALID, "tau"); g_opt.tau = v; return JK_OK;
        case JK_OPT_MIXED_TSMALL: if (!(v >= 0)) return fail(JK_ERR_INVALID, "tsmall"); g_opt.tsmall = v; return JK_OK;
        case JK_OPT_CHECK_SYMMETRY: g_opt.check_sym = v != 0.0; return JK_OK;
        case JK_OPT_GRAPH: g_opt.graph = v != 0.0; return JK_OK;
        case JK_OPT_PROFILE: g_opt.profile = v != 0.0; return JK_OK;
        case JK_OPT_DENSITY_SCREEN:
            if (!(v >= 0) || !std::isfinite(v)) return fail(JK_ERR_INVALID, "density screening threshold");
            g_opt.eps = v;
            return JK_OK;
        case JK_OPT_RPATH: g_opt.rpath = v != 0.0; return JK_OK;
        case JK_OPT_FAIL_ALLOC_AFTER:
            if (!std::isfinite(v)) return fail(JK_ERR_INVALID, "allocation fault count");
            g_fail_alloc.store(v < 0 ? -1 : (long long)v);
            return JK_OK;
        case JK_OPT_GRAD_TAU:
            if (!(v >= 0) || !std::isfinite(v)) return fail(JK_ERR_INVALID, "gradient tau");
            g_opt.grad_tau = v;
            return JK_OK;
        case JK_OPT_DF_TIER: g_opt.df_tier = v != 0.0; return JK_OK;
        case JK_OPT_PRIM_TAU: if (!(v >= 0) || !std::isfinite(v)) return fail(JK_ERR_INVALID, "primitive tau"); g_opt.ptau = v; return JK_OK;
        case JK_OPT_GRAD_PRIM_TAU:
            if (!(v >= 0) || !std::isfinite(v)) return fail(JK_ERR_INVALID, "gradient primitive tau");
            g_opt.grad_ptau = v;
            return JK_OK;
    }
    return fail(JK_ERR_INVALID, "unknown option");
}

int jk_get_option(jk_option opt, double* v) {
    if (!v) return fail(JK_ERR_INVALID, "null");
    switch (opt) {
        case JK_OPT_MIXED_TAU: *v = g_opt.tau; return JK_OK;
        case JK_OPT_MIXED_TSMALL: *v = g_opt.tsmall; return JK_OK;
        case JK_OPT_CHECK_SYMMETRY: *v = g_opt.check_sym; return JK_OK;
        case JK_OPT_GRAPH: *v = g_opt.graph; return JK_OK;
        case JK_OPT_PROFILE: *v = g_opt.profile; return JK_OK;
        case JK_OPT_DENSITY_SCREEN: *v = g_opt.eps; return JK_OK;
        case JK_OPT_RPATH: *v = g_opt.rpath; return JK_OK;
        case JK_OPT_FAIL_ALLOC_AFTER: *v = (double)g_fail_alloc.load(); return JK_OK;
        case JK_OPT_GRAD_TAU: *v = g_opt.grad_tau; return JK_OK;
        case JK_OPT_DF_TIER: *v = g_opt.df_tier; return JK_OK;
        case JK_OPT_PRIM_TAU: *v = g_opt.ptau; return JK_OK;
        case JK_OPT_GRAD_PRIM_TAU: *v = g_opt.grad_ptau; return JK_OK;
    }
    return fail(JK_ERR_INVALID, "unknown option");
}

int jk_last_split(jk_pairs h, int64_t* n32, int64_t* n64) {
    if (!h) return fail(JK_ERR_INVALID, "null handle");
    long long a = 0, b = h->nquartets;
    if (h->last_prec == JK_MIXED && h->split_tot.p) {
        std::vector<long long> t(kSplitSlots * h->rows.size());
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(t.data(), h->split_tot.p, sizeof(long long) * t.size(), cudaMemcpyDeviceToHost));
        a = b = 0;
        for (size_t k = 0; k < h->rows.size(); ++k) {
            if (h->rows[k].total <= 0) continue;
            a += t[kSplitSlots * k];
            b += t[kSplitSlots * k + 1];
        }
    }
    if (n32) *n32 = a;
    if (n64) *n64 = b;
    return JK_OK;
}

int jk_autotune(jk_pairs h, const double* D, double* J, double* K, jk_precision prec, void* cuda_stream) {
    g_err.clear();
    if (!h || !D || !J || !K) return fail(JK_ERR_INVALID, "null argument");
    if (prec != JK_FP64 && prec != JK_MIXED) return fail(JK_ERR_INVALID, "precision");
    return autotune_impl(h, D, J, K, prec == JK_FP64 ? 0 : 1, static_cast<cudaStream_t>(cuda_stream));
}

int jk_tuning(jk_pairs h, int max_rows, int* rows, int* nrows) {
    if (!h || !nrows || (max_rows > 0 && !rows)) return fail(JK_ERR_INVALID, "bad argument");
    int k = 0;
    for (const ClassRows& cr : h->rows) {
        if (cr.total <= 0) continue;
        if (k < max_rows) {
            int* r = rows + 6 * k;
            r[0] = cr.bra_cls; r[1] = cr.ket_cls;
            r[2] = cr.tune[0].block; r[3] = cr.tune[0].qpt; r[4] = cr.tune[1].block; r[5] = cr.tune[1].qpt;
        }
        ++k;
    }
    *nrows = k;
    return JK_OK;
}

int jk_set_tuning(jk_pairs h, int nrows, const int* rows) {
    if (!h || nrows < 0 || (nrows > 0 && !rows)) return fail(JK_ERR_INVALID, "bad argument");
    // every entry is checked before any is applied: a corrupted configuration changes nothing
    const int ncls = gb_num_pair_classes();
    for (int k = 0; k < nrows; ++k) {
        const int* r = rows + 6 * k;
        if (r[0] < 0 || r[0] >= ncls || r[1] < 0 || r[1] > r[0])
            return fail(JK_ERR_INVALID, "tuning entry " + std::to_string(k) + ": class out of range");
        if (r[2] < 32 || r[2] > 128 || r[2] % 32 || r[4] < 32 || r[4] > 128 || r[4] % 32 || r[3] < 1 || r[5] < 1 ||
            r[3] > (1 << 20) || r[5] > (1 << 20))
            return fail(JK_ERR_INVALID, "tuning entry " + std::to_string(k) + " out of range");
    }
    for (int k = 0; k < nrows; ++k) {
        const int* r = rows + 6 * k;
        for (ClassRows& cr : h->rows)
            if (cr.bra_cls == r[0] && cr.ket_cls == r[1]) {
                cr.tune[0].block = r[2]; cr.tune[0].qpt = r[3];
                cr.tune[1].block = r[4]; cr.tune[1].qpt = r[5];
            }
    }
    drop_plan_of(h);
    return JK_OK;
}

int jk_last_launches(jk_pairs h, int64_t* n) {
    if (!h || !n) return fail(JK_ERR_INVALID, "bad argument");
    *n = h->launches;
    return JK_OK;
}

int jk_class_stats(jk_pairs h, int max_rows, int64_t* rows, int* nrows) {
    if (!h || !nrows || (max_rows > 0 && !rows)) return fail(JK_ERR_INVALID, "bad argument");
    int k = 0;
    for (const ClassRows& cr : h->rows) {
        if (cr.total <= 0) continue;
        if (k < max_rows) {
            int fq = 0, fb = 0;
            gb_class_flops(cr.bra_cls, cr.ket_cls, &fq, &fb);
            int64_t* r = rows + 6 * k;
            r[0] = cr.bra_cls; r[1] = cr.ket_cls; r[2] = cr.total; r[3] = cr.nprimq; r[4] = cr.nbrap;
            r[5] = (int64_t)fq * cr.nprimq + (int64_t)fb * cr.nbrap;
        }
        ++k;
    }
    *nrows = k;
    return JK_OK;
}

int jk_split_stats(jk_pairs h, int max_rows, int64_t* rows, int* nrows) {
    g_err.clear();
    if (!h || !nrows || (max_rows > 0 && !rows)) return fail(JK_ERR_INVALID, "bad argument");
    if (h->last_prec != JK_MIXED) return fail(JK_ERR_INVALID, "the last jk_build on this handle was not mixed");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != h->device) return fail(JK_ERR_INVALID, "handle belongs to another device");
    CK(cudaDeviceSynchronize());  // the build may have run on any stream
    DevBuf acc;
    int rc;
    if ((rc = acc.alloc(4 * sizeof(unsigned long long)))) return rc;
    int k = 0;
    for (size_t ri = 0; ri < h->rows.size(); ++ri) {
        const ClassRows& cr = h->rows[ri];
        if (cr.total <= 0) continue;
        if (k < max_rows) {
            // FP32: the contiguous suffix (c32 from k32) plus the demoted list;
            // FP64: the FP64 list (over the rows the build ran: all, or a part's)
            CK(cudaMemset(acc.p, 0, 4 * sizeof(unsigned long long)));
            const int r0 = ri < h->last_r0.size() ? h->last_r0[ri] : 0;
            const int nr = (ri < h->last_r1.size() ? h->last_r1[ri] : cr.nrows) - r0;
            if (nr > 0) {
                k_rows_primq<<<nblk(nr, 256), 256>>>(cr.c32.as<long long>() + r0, cr.bra.as<int>() + r0,
                                                     cr.k32.as<int>() + r0, nr, h->info.as<int4>(),
                                                     h->npre.as<long long>(), acc.as<unsigned long long>());
                k_list_primq<<<nblk(nr, 256), 256>>>(cr.cdem.as<long long>() + r0, cr.ldem.as<long long>() + r0,
                                                     h->listdem.as<int>() + h->list_offd[ri], cr.bra.as<int>() + r0,
                                                     nr, h->info.as<int4>(), acc.as<unsigned long long>());
                if (h->last_psplit)
                    k_list_primq_split<<<nblk(nr, 256), 256>>>(
                        cr.c64.as<long long>() + r0, cr.l64.as<long long>() + r0,
                        h->list64.as<int>() + h->list_off64[ri], h->thr64.as<float>() + h->list_off64[ri],
                        cr.bra.as<int>() + r0, nr, h->info.as<int4>(), h->pq.as<float>(), acc.as<unsigned long long>(),
                        acc.as<unsigned long long>() + 2);
                else
                    k_list_primq<<<nblk(nr, 256), 256>>>(cr.c64.as<long long>() + r0, cr.l64.as<long long>() + r0,
                                                         h->list64.as<int>() + h->list_off64[ri], cr.bra.as<int>() + r0,
                                                         nr, h->info.as<int4>(), acc.as<unsigned long long>() + 2);
                CKL();
            }
            unsigned long long v[4];
            long long q2[2];
            CK(cudaMemcpy(v, acc.p, sizeof(v), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(q2, h->split_tot.as<long long>() + kSplitSlots * ri, 2 * sizeof(long long),
                          cudaMemcpyDeviceToHost));
            int fq = 0, fb = 0;
            gb_class_flops(cr.bra_cls, cr.ket_cls, &fq, &fb);
            int64_t* r = rows + 8 * k;
            r[0] = cr.bra_cls; r[1] = cr.ket_cls;
            r[2] = q2[0]; r[3] = (int64_t)v[0]; r[4] = (int64_t)fq * (int64_t)v[0] + (int64_t)fb * (int64_t)v[1];
            r[5] = q2[1]; r[6] = (int64_t)v[2]; r[7] = (int64_t)fq * (int64_t)v[2] + (int64_t)fb * (int64_t)v[3];
        }
        ++k;
    }
    *nrows = k;
    return JK_OK;
}

int jk_profile(jk_pairs h, int max_rows, double* rows, int* nrows) {
    if (!h || !nrows || (max_rows > 0 && !rows)) return fail(JK_ERR_INVALID, "bad argument");
    int k = 0;
    for (const ProfRec& r : h->prof) {
        if (k < max_rows) {
            CK(cudaEventSynchronize(r.e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, r.e0, r.e1));
            double* o = rows + 5 * k;
            o[0] = r.bra; o[1] = r.ket; o[2] = r.prec; o[3] = (double)r.total; o[4] = ms;
        }
        ++k;
    }
    *nrows = k;
    return JK_OK;
}

int jk_fma_peak(jk_precision prec, int iters, double* flops, void* cuda_stream) {
    if (!flops || iters <= 0) return fail(JK_ERR_INVALID, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    DevBuf sink;
    int rc;
    if ((rc = sink.alloc(16))) return rc;
    const int blocks = nsm * 8, threads = 256;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // warm-up, then the timed launch
    for (int rep = 0; rep < 2; ++rep) {
        CK(cudaEventRecord(e0, st));
        if (prec == JK_FP64) k_fma_peak<double><<<blocks, threads, 0, st>>>(iters, sink.as<double>());
        else k_fma_peak<float><<<blocks, threads, 0, st>>>(iters, sink.as<float>());
        CKL();
        CK(cudaEventRecord(e1, st));
    }
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *flops = 2.0 * 8 * 16 * (double)iters * blocks * threads / (ms * 1e-3);
    return JK_OK;
}

int jk_one_electron(jk_pairs h, const double* charges, double* S, double* T, double* V, void* cuda_stream) {
    g_err.clear();
    if (!h || !charges || !S || !T || !V) return fail(JK_ERR_INVALID, "null argument");
    for (int i = 0; i < h->natom; ++i)
        if (!std::isfinite(charges[i])) return fail(JK_ERR_INVALID, "non-finite nuclear charge");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != h->device) return fail(JK_ERR_INVALID, "handle belongs to another device");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int rc;
    if ((rc = upload(h->charges, charges, (size_t)h->natom, st))) return rc;
    const size_t n2 = (size_t)h->nbf * h->nbf;
    CK(cudaMemsetAsync(S, 0, sizeof(double) * n2, st));
    CK(cudaMemsetAsync(T, 0, sizeof(double) * n2, st));
    CK(cudaMemsetAsync(V, 0, sizeof(double) * n2, st));
    if (h->npair > 0) {
        gb::OneElArgs a;
        std::memset(&a, 0, sizeof(a));
        a.pairs = view_of(h);
        a.lab = h->pair_lab.as<int2>();
        a.boys = g_boys[h->device].tab.as<double>();
        a.xyz = h->xyz.as<double>();
        a.Z = h->charges.as<double>();
        a.natom = h->natom;
        a.nbf = h->nbf;
        a.S = S;
        a.T = T;
        a.V = V;
        const unsigned grid = (unsigned)std::min<long long>(nblk(h->npair, 128), (long long)h->nsm * 16);
        gb::k_one_electron<<<grid, 128, 0, st>>>(a);
        CKL();
    }
    return JK_OK;
}

int jk_limits(int* lmax, int* grad_lmax) {
    if (!lmax || !grad_lmax) return fail(JK_ERR_INVALID, "null argument");
    int l = 0;
    while ((l + 2) * (l + 3) / 2 <= gb_num_pair_classes()) ++l;  // pair classes compiled: (lmax+1)(lmax+2)/2
    *lmax = l;
    *grad_lmax = gb_grad_lmax();
    return JK_OK;
}

int jk_sph_nbf(jk_pairs h, int* nsph) {
    if (!h || !nsph) return fail(JK_ERR_INVALID, "bad argument");
    *nsph = h->nsph;
    return JK_OK;
}

int jk_sph_transform(jk_pairs h, jk_sph_dir dir, const double* in, double* out, void* cuda_stream) {
    g_err.clear();
    if (!h || !in || !out) return fail(JK_ERR_INVALID, "null argument");
    if (dir != JK_SPH_TO_CART && dir != JK_CART_TO_SPH) return fail(JK_ERR_INVALID, "direction");
    const int n_in = dir == JK_SPH_TO_CART ? h->nsph : h->nbf;
    const int n_out = dir == JK_SPH_TO_CART ? h->nbf : h->nsph;
    const uintptr_t i0 = (uintptr_t)in, i1 = i0 + sizeof(double) * (size_t)n_in * n_in;
    const uintptr_t o0 = (uintptr_t)out, o1 = o0 + sizeof(double) * (size_t)n_out * n_out;
    if (i0 < o1 && o0 < i1) return fail(JK_ERR_INVALID, "in and out overlap");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != h->device) return fail(JK_ERR_INVALID, "handle belongs to another device");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int rc;
    if ((rc = sph_prepare(h, st))) return rc;
    gb::SphArgs a;
    std::memset(&a, 0, sizeof(a));
    a.in = in;
    a.out = out;
    a.n_in = n_in;
    a.n_out = n_out;
    a.dir = dir == JK_SPH_TO_CART ? 0 : 1;
    a.owner = dir == JK_SPH_TO_CART ? h->bf_shell.as<int>() : h->sph_owner.as<int>();
    a.shell = h->sph_shell.as<int4>();
    a.coef = h->sph_coef.as<double>();
    const long long total = (long long)n_out * n_out;
    const unsigned grid = (unsigned)std::min<long long>(nblk(total, 256), (long long)h->nsm * 8);
    gb::k_sph_transform<<<grid, 256, 0, st>>>(a);
    CKL();
    return JK_OK;
}

void shellpairs_free(jk_pairs h) {
    if (!h) return;
    drop_plan_of(h);  // a cached batch plan that reads this handle's device arrays goes with it
    delete h;
}

}  // extern "C"
