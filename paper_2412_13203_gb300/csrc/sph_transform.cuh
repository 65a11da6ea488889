// Cartesian <-> pure (real solid-harmonic) transform of a basis-indexed
// matrix, for basis sets with pure d and f shells.
//
// The ERI kernels work on Cartesian components (Sec. 2.2, Eq. 1).  With T the
// block-diagonal Cartesian-to-pure matrix (one ncart(l) x npure(l) block per
// shell, identity for s and p), a pure-basis build is
//     D_cart = T D_pure T^T  ->  J_cart, K_cart  ->  J_pure = T^T J_cart T
// (and the same for K): every (ij|kl) over pure functions is the Cartesian
// integral with each index contracted against T, and the density enters J/K
// linearly.  The transform is O(nbf^2 * ncart) work, negligible beside the
// O(nbf^4) integrals, so it runs as its own pass instead of inside digestion.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace gb {

constexpr int kSphLmax = 3;

struct SphArgs {
    const double* in;   // [n_in x n_in] row-major
    double* out;        // [n_out x n_out] row-major, must not overlap `in`
    int n_in, n_out;
    int dir;            // 0: pure -> Cartesian, out = T in T^T; 1: Cartesian -> pure, out = T^T in T
    const int* owner;   // [n_out]: shell of every output index
    const int4* shell;  // [nshell]: (l, first Cartesian index, first pure index, offset of T_l in coef)
    const double* coef; // per l: T_l, ncart(l) x npure(l) row-major
};

__device__ __forceinline__ int sph_ncart(int l) { return (l + 1) * (l + 2) / 2; }
__device__ __forceinline__ int sph_npure(int l) { return l >= 2 ? 2 * l + 1 : (l + 1) * (l + 2) / 2; }

// One thread per output element (grid-stride): the element's two shells fix
// the input block it reads (at most 10 x 10 values, shared with the other
// elements of the same output block through L1/L2).  Zero coefficients are
// skipped; a 1 x 1 or identity block (s, p) copies its input exactly.
__global__ void __launch_bounds__(256) k_sph_transform(SphArgs a) {
    const long long total = (long long)a.n_out * a.n_out;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int I = (int)(e / a.n_out);
        const int J = (int)(e - (long long)I * a.n_out);
        const int4 sI = a.shell[a.owner[I]];
        const int4 sJ = a.shell[a.owner[J]];
        const int npI = sph_npure(sI.x), npJ = sph_npure(sJ.x);
        const double* TI = a.coef + sI.w;
        const double* TJ = a.coef + sJ.w;
        double acc = 0.0;
        if (a.dir == 1) {
            // out[I][J] = sum_{p,q} T_I[p][i] in[cI + p][cJ + q] T_J[q][j]
            const int i = I - sI.z, j = J - sJ.z;
            const int ncI = sph_ncart(sI.x), ncJ = sph_ncart(sJ.x);
            for (int p = 0; p < ncI; ++p) {
                const double ti = TI[p * npI + i];
                if (ti == 0.0) continue;
                const double* row = a.in + (size_t)(sI.y + p) * a.n_in + sJ.y;
                double s = 0.0;
                for (int q = 0; q < ncJ; ++q) {
                    const double tj = TJ[q * npJ + j];
                    if (tj != 0.0) s = fma(tj, row[q], s);
                }
                acc = fma(ti, s, acc);
            }
        } else {
            // out[P][Q] = sum_{i,j} T_I[p][i] in[pI + i][pJ + j] T_J[q][j]
            const int p = I - sI.y, q = J - sJ.y;
            for (int i = 0; i < npI; ++i) {
                const double ti = TI[p * npI + i];
                if (ti == 0.0) continue;
                const double* row = a.in + (size_t)(sI.z + i) * a.n_in + sJ.z;
                double s = 0.0;
                for (int j = 0; j < npJ; ++j) {
                    const double tj = TJ[q * npJ + j];
                    if (tj != 0.0) s = fma(tj, row[j], s);
                }
                acc = fma(ti, s, acc);
            }
        }
        a.out[e] = acc;
    }
}

}  // namespace gb
