// Per-row precision split and density screening of the quartet rows of a
// mixed build (single-molecule and batched forms).  Included by the runtime
// inside its file-local namespace, after eri_device.cuh.
//
// A row holds the kets [s, s + c) of one bra pair, sorted by Schwarz factor
// Q descending.  With qi = Q_ab and the largest |D| element dmax, the global
// bound of ket j is qi Q_j dmax and its density-weighted bound qi Q_j max|D|
// over the six shell blocks its J and K updates read.  Because the global
// bound falls along the row:
//   * the kets with global bound >= eps form a prefix [s, kend); the rest of
//     the row is skipped (density screening; eps = 0 keeps every ket);
//   * the kets with global bound >= tau form a prefix [s, lo), lo <= kend;
//     there each ket is tested with its own D blocks: FP64 if the weighted
//     bound is >= tau, else demoted to FP32 if it is >= eps, else skipped;
//   * the kets [lo, kend) run in FP32 as a contiguous range.
// A skipped ket's weighted bound is below eps, so it changes no J or K
// element by more than eps times its number of components and degeneracy.

// The largest |D| block a quartet's J and K updates touch: D_ab and D_cd
// (Coulomb), D_ac, D_ad, D_bc, D_bd (exchange).
__device__ __forceinline__ float quartet_dmax(const float* dsh, int nshell, int2 ab, int2 cd) {
    const float* r_a = dsh + (size_t)ab.x * nshell;
    const float* r_b = dsh + (size_t)ab.y * nshell;
    float m = fmaxf(r_a[ab.y], dsh[(size_t)cd.x * nshell + cd.y]);
    m = fmaxf(m, fmaxf(r_a[cd.x], r_a[cd.y]));
    return fmaxf(m, fmaxf(r_b[cd.x], r_b[cd.y]));
}

// First ket in [s, s + c) whose global bound qg Q_j is below `cut` (kets
// sorted by Q descending).
__device__ __forceinline__ int split_search(const double4* A, int s, int c, double qg, double cut) {
    int lo = s, hi = s + c;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (qg * A[mid].w >= cut) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Counts of one row: FP64 and demoted kets of the prefix, FP32 range [lo, kend).
__device__ __forceinline__ void split_row(const double4* A, int i, int s, int c, double dmax, double tau, double eps,
                                          const int2* psh, const float* dsh, int nshell, long long& n64,
                                          long long& nd, long long& n32, int& lo) {
    const double qi = A[i].w;
    const double qg = qi * dmax;
    const int kend = split_search(A, s, c, qg, eps);
    lo = split_search(A, s, kend - s, qg, tau);
    const int2 ab = psh[i];
    n64 = 0;
    nd = 0;
    for (int j = s; j < lo; ++j) {
        const double b = qi * A[j].w * (double)quartet_dmax(dsh, nshell, ab, psh[j]);
        if (b >= tau) ++n64;
        else if (b >= eps) ++nd;
    }
    n32 = kend - lo;
}

// The prefix [s, lo) of one row into the FP64 and demoted lists.  With a
// primitive split (thr64 set), every FP64 entry also gets its primitive cut
// taup / max|D| of its D blocks: its primitive quartets with pq[p] pq[q] at or
// above the cut run in the FP64 tier, the others in FP32 (JKArgs::pmode).
__device__ __forceinline__ void fill_row(const double4* A, int i, int s, int lo, double tau, double eps,
                                         const int2* psh, const float* dsh, int nshell, int* list64, int* listdem,
                                         float taup, float* thr64) {
    const double qi = A[i].w;
    const int2 ab = psh[i];
    int o64 = 0, od = 0;
    for (int j = s; j < lo; ++j) {
        const float dq = quartet_dmax(dsh, nshell, ab, psh[j]);
        const double b = qi * A[j].w * (double)dq;
        if (b >= tau) {
            if (thr64) thr64[o64] = __fdiv_rn(taup, dq);
            list64[o64++] = j;
        } else if (b >= eps) {
            listdem[od++] = j;
        }
    }
}

// Writes per-row quartet and work-item counts of the three parts (P: most
// work items per quartet) and adds the FP32 (incl. demoted) / FP64 / demoted
// quartet totals to qtot[0], qtot[1], qtot[7].
__device__ __forceinline__ void store_split(int r, long long n64, long long nd, long long n32, int lo, long long m,
                                            long long* c64, long long* cdem, long long* c32, int* k32,
                                            long long* w64, long long* wdem, long long* w32, unsigned long long* qtot) {
    c64[r] = n64;
    cdem[r] = nd;
    c32[r] = n32;
    k32[r] = lo;
    w64[r] = n64 * m;
    wdem[r] = nd * m;
    w32[r] = n32 * m;
    atomicAdd(qtot, (unsigned long long)(n32 + nd));
    atomicAdd(qtot + 1, (unsigned long long)n64);
    atomicAdd(qtot + 7, (unsigned long long)nd);
}

__global__ void k_rows_split(const long long* start, const int* rbra, const int* rket0, int nrows, const double4* A,
                             const double* dmax, double tau, double eps, const int4* info, const int2* psh,
                             const float* dsh, int nshell, int P, long long* c64, long long* cdem, long long* c32,
                             int* k32, long long* w64, long long* wdem, long long* w32, unsigned long long* qtot) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const int i = rbra[r];
    long long n64, nd, n32;
    int lo;
    split_row(A, i, rket0[r], (int)(start[r + 1] - start[r]), *dmax, tau, eps, psh, dsh, nshell, n64, nd, n32, lo);
    store_split(r, n64, nd, n32, lo, gb::item_split(P, info[i].z), c64, cdem, c32, k32, w64, wdem, w32, qtot);
}

// Second pass: the kets of every row's prefix into the FP64 and demoted lists,
// at the row offsets l64 / ldem (exclusive prefixes of c64 / cdem).
__global__ void k_rows_fill(const int* rbra, const int* rket0, const int* k32, int nrows, const double4* A, double tau,
                            double eps, const int2* psh, const float* dsh, int nshell, const long long* l64,
                            const long long* ldem, int* list64, int* listdem, float taup, float* thr64) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    fill_row(A, rbra[r], rket0[r], k32[r], tau, eps, psh, dsh, nshell, list64 + l64[r], listdem + ldem[r], taup,
             thr64 ? thr64 + l64[r] : nullptr);
}

// k_rows_split for batched rows (each row's molecule from rowmol; dmax holds
// every molecule's max|D| as the bits of a double).
__global__ void k_rows_split_batched(const long long* start, const int* rbra, const int* rket0, const int* rowmol,
                                     int nrows, const gb::BatchMol* bm, const unsigned long long* dmax, double tau,
                                     double eps, int P, long long* c64, long long* cdem, long long* c32, int* k32,
                                     long long* w64, long long* wdem, long long* w32, unsigned long long* qtot) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const gb::BatchMol& mol = bm[rowmol[r]];
    const int i = rbra[r];
    long long n64, nd, n32;
    int lo;
    split_row(mol.pairs.A, i, rket0[r], (int)(start[r + 1] - start[r]),
              __longlong_as_double((long long)dmax[rowmol[r]]), tau, eps, mol.psh, mol.Dsh, mol.nshell, n64, nd, n32,
              lo);
    store_split(r, n64, nd, n32, lo, gb::item_split(P, mol.pairs.info[i].z), c64, cdem, c32, k32, w64, wdem, w32, qtot);
}

// k_rows_fill for batched rows.
__global__ void k_rows_fill_batched(const int* rbra, const int* rket0, const int* k32, const int* rowmol, int nrows,
                                    const gb::BatchMol* bm, double tau, double eps, const long long* l64,
                                    const long long* ldem, int* list64, int* listdem, float taup, float* thr64) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const gb::BatchMol& mol = bm[rowmol[r]];
    fill_row(mol.pairs.A, rbra[r], rket0[r], k32[r], tau, eps, mol.psh, mol.Dsh, mol.nshell, list64 + l64[r],
             listdem + ldem[r], taup, thr64 ? thr64 + l64[r] : nullptr);
}
