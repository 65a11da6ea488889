// One-electron integrals (overlap S, kinetic energy T, nuclear attraction V)
// over the kept shell pairs of a handle, for the SCF around the J/K build
// (Sec. 2.1: the Fock matrix is the one-electron part plus J - K/2).
// Included after eri_device.cuh.
//
// McMurchie-Davidson, one thread per shell pair (grid-stride), all component
// pairs of the pair at once:
//   E^{ij}_t per axis from E^{00}_0 = 1,
//     E^{i+1,j}_t = E^{ij}_{t-1}/2p + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1}  (same with X_PB for j+1);
//   S_ij(1-D) = E^{ij}_0 sqrt(pi/p),  S = K_AB c_a c_b Sx Sy Sz;
//   kinetic from the ket's second derivative,
//     T_ij(1-D) = -1/2 [ j(j-1) S_i(j-2) - 2b(2j+1) S_ij + 4b^2 S_i(j+2) ],  T = Tx Sy Sz + Sx Ty Sz + Sx Sy Tz;
//   V = -sum_C Z_C (2 pi / p) K_AB c_a c_b sum_tuv E_t E_u E_v R_tuv(p, P - C), with
//     R^{(n)}_000 = (-2p)^n F_n(p |P - C|^2) and R^{(n)}_{t+1,u,v} = t R^{(n+1)}_{t-1,u,v} + X_PC R^{(n+1)}_{t,u,v}.
// The pair data already hold P, p, 1/2p, the exponent of the a primitive and
// kappa = sqrt(2 pi^(5/2)) K_AB c_a c_b / p (normalised coefficients).
#pragma once

namespace gb {

constexpr int kOneLmax = 3;                  // per shell
constexpr int kOneL = 2 * kOneLmax;          // la + lb
constexpr int kOneTet = (kOneL + 1) * (kOneL + 2) * (kOneL + 3) / 6;  // (t,u,v) with t+u+v <= kOneL

struct OneElArgs {
    PairsView pairs;
    const int2* lab;     // per pair: la, lb
    const double* boys;  // Boys table (FP64)
    const double* xyz;   // [natom * 3] nuclei
    const double* Z;     // [natom] charges
    int natom, nbf;
    double* S;           // [nbf * nbf] row-major, each written once per element of a kept pair
    double* T;
    double* V;
};

// Index of (t, u, v), t + u + v <= kOneL, in a flat tetrahedral array.
__device__ __forceinline__ int one_tet(int t, int u, int v) {
    const int m = kOneL + 1;
    const int r = m + 2 - t;  // slabs before t hold C(m+2,3) - C(m+2-t,3) entries
    return ((m + 2) * (m + 1) * m - r * (r - 1) * (r - 2)) / 6 + u * (m - t) - u * (u - 1) / 2 + v;
}

// E^{ij}_t for i <= la, j <= jmax on one axis (E^{00}_0 = 1).
__device__ __forceinline__ void one_e_axis(int la, int jmax, double PA, double PB, double oo2p,
                                           double E[kOneLmax + 1][kOneLmax + 3][kOneL + 3]) {
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j <= jmax; ++j)
            for (int t = 0; t <= i + j; ++t) E[i][j][t] = 0.0;
    E[0][0][0] = 1.0;
    for (int i = 0; i < la; ++i)
        for (int t = 0; t <= i + 1; ++t)
            E[i + 1][0][t] = (t > 0 ? oo2p * E[i][0][t - 1] : 0.0) + (t <= i ? PA * E[i][0][t] : 0.0) +
                             (t + 1 <= i ? (t + 1) * E[i][0][t + 1] : 0.0);
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j < jmax; ++j)
            for (int t = 0; t <= i + j + 1; ++t)
                E[i][j + 1][t] = (t > 0 ? oo2p * E[i][j][t - 1] : 0.0) + (t <= i + j ? PB * E[i][j][t] : 0.0) +
                                 (t + 1 <= i + j ? (t + 1) * E[i][j][t + 1] : 0.0);
}

__device__ __forceinline__ int one_ncart(int l) { return (l + 1) * (l + 2) / 2; }

// Component k of a shell of angular momentum l (lx descending, then ly descending).
__device__ __forceinline__ void one_comp(int l, int k, int& x, int& y, int& z) {
    int n = 0;
    for (int lx = l; lx >= 0; --lx)
        for (int lz = 0; lz <= l - lx; ++lz, ++n)
            if (n == k) { x = lx; y = l - lx - lz; z = lz; return; }
}

__global__ void __launch_bounds__(128) k_one_electron(OneElArgs a) {
    const double kPi = 3.14159265358979323846;
    const double kS2pi52 = 5.9149671727956128778;  // sqrt(2 pi^(5/2)), as in kappa
    constexpr int NC = (kOneLmax + 1) * (kOneLmax + 2) / 2;
    for (int pr = blockIdx.x * blockDim.x + threadIdx.x; pr < a.pairs.npair; pr += gridDim.x * blockDim.x) {
        const int2 l = a.lab[pr];
        const int4 inf = a.pairs.info[pr];
        const double4 A = a.pairs.A[pr], B = a.pairs.B[pr];
        const int na = one_ncart(l.x), nb = one_ncart(l.y);
        int ca[NC][3], cb[NC][3];
        for (int k = 0; k < na; ++k) one_comp(l.x, k, ca[k][0], ca[k][1], ca[k][2]);
        for (int k = 0; k < nb; ++k) one_comp(l.y, k, cb[k][0], cb[k][1], cb[k][2]);
        double accS[NC * NC], accT[NC * NC], accV[NC * NC];
        for (int k = 0; k < na * nb; ++k) accS[k] = accT[k] = accV[k] = 0.0;
        double E[3][kOneLmax + 1][kOneLmax + 3][kOneL + 3];
        double R0[kOneTet], R1[kOneTet];
        const int L = l.x + l.y;
        for (int k = inf.w; k < inf.w + inf.z; ++k) {
            const double4 P = a.pairs.pp[k];
            const double2 q = a.pairs.pp2[k];
            const double p = P.w, oo2p = q.y;
            const double kcc = q.x * p * (1.0 / kS2pi52);  // K_AB c_a c_b
            const double beta = p - a.pairs.alpha[k];
            one_e_axis(l.x, l.y + 2, P.x - A.x, P.x - B.x, oo2p, E[0]);
            one_e_axis(l.x, l.y + 2, P.y - A.y, P.y - B.y, oo2p, E[1]);
            one_e_axis(l.x, l.y + 2, P.z - A.z, P.z - B.z, oo2p, E[2]);
            const double sq = sqrt(kPi / p);
            for (int x = 0; x < na; ++x)
                for (int y = 0; y < nb; ++y) {
                    double s1[3], t1[3];
                    for (int d = 0; d < 3; ++d) {
                        const int i = ca[x][d], j = cb[y][d];
                        s1[d] = E[d][i][j][0] * sq;
                        const double sm = j >= 2 ? E[d][i][j - 2][0] * sq : 0.0;
                        t1[d] = -0.5 * (j * (j - 1) * sm - 2.0 * beta * (2 * j + 1) * s1[d] +
                                        4.0 * beta * beta * E[d][i][j + 2][0] * sq);
                    }
                    accS[x * nb + y] += kcc * s1[0] * s1[1] * s1[2];
                    accT[x * nb + y] += kcc * (t1[0] * s1[1] * s1[2] + s1[0] * t1[1] * s1[2] + s1[0] * s1[1] * t1[2]);
                }
            for (int c = 0; c < a.natom; ++c) {
                const double X = P.x - a.xyz[3 * c], Y = P.y - a.xyz[3 * c + 1], Zc = P.z - a.xyz[3 * c + 2];
                double F[kOneL + 1];
                boys_f64<kOneL>(p * (X * X + Y * Y + Zc * Zc), F, a.boys);
                // R^{(n)} for n = L down to 0; level n holds t + u + v <= L - n
                double* cur = R0;
                double* nxt = R1;
                double m2p = 1.0;
                for (int n = 0; n < L; ++n) m2p *= -2.0 * p;
                cur[0] = m2p * F[L];
                for (int n = L - 1; n >= 0; --n) {
                    m2p /= -2.0 * p;
                    for (int t = 0; t <= L - n; ++t)
                        for (int u = 0; u <= L - n - t; ++u)
                            for (int v = 0; v <= L - n - t - u; ++v) {
                                double r;
                                if (t > 0) r = (t > 1 ? (t - 1) * cur[one_tet(t - 2, u, v)] : 0.0) + X * cur[one_tet(t - 1, u, v)];
                                else if (u > 0) r = (u > 1 ? (u - 1) * cur[one_tet(t, u - 2, v)] : 0.0) + Y * cur[one_tet(t, u - 1, v)];
                                else if (v > 0) r = (v > 1 ? (v - 1) * cur[one_tet(t, u, v - 2)] : 0.0) + Zc * cur[one_tet(t, u, v - 1)];
                                else r = m2p * F[n];
                                nxt[one_tet(t, u, v)] = r;
                            }
                    double* sw = cur;
                    cur = nxt;
                    nxt = sw;
                }
                const double pref = -a.Z[c] * 2.0 * kPi / p * kcc;
                for (int x = 0; x < na; ++x)
                    for (int y = 0; y < nb; ++y) {
                        const int ix = ca[x][0], jx = cb[y][0], iy = ca[x][1], jy = cb[y][1], iz = ca[x][2], jz = cb[y][2];
                        double v = 0.0;
                        for (int t = 0; t <= ix + jx; ++t)
                            for (int u = 0; u <= iy + jy; ++u) {
                                const double eu = E[0][ix][jx][t] * E[1][iy][jy][u];
                                for (int w = 0; w <= iz + jz; ++w) v += eu * E[2][iz][jz][w] * cur[one_tet(t, u, w)];
                            }
                        accV[x * nb + y] += pref * v;
                    }
            }
        }
        const bool diag = inf.x == inf.y;
        for (int x = 0; x < na; ++x)
            for (int y = 0; y < nb; ++y) {
                const size_t i = (size_t)(inf.x + x) * a.nbf + inf.y + y;
                a.S[i] = accS[x * nb + y];
                a.T[i] = accT[x * nb + y];
                a.V[i] = accV[x * nb + y];
                if (!diag) {
                    const size_t j = (size_t)(inf.y + y) * a.nbf + inf.x + x;
                    a.S[j] = accS[x * nb + y];
                    a.T[j] = accT[x * nb + y];
                    a.V[j] = accV[x * nb + y];
                }
            }
    }
}

}  // namespace gb
