/*
 * gb300_eri.h -- C ABI of the GB300 (sm_103a) screened-ERI / J-K / gradient library.
 *
 * What the library computes (arXiv 2412.13203, Sec. 2.1-2.2): the four-centre
 * electron repulsion integrals over contracted Cartesian Gaussian shells
 *   (ab|cd) = sum_klmn D_ak D_bl D_cm D_dn [a_k b_l | c_m d_n]        (Eq. 2)
 * for every angular-momentum class up to l = 3 (f), Schwarz-screened and
 * contracted on the fly with a density matrix into the Coulomb and exchange
 * matrices of a Fock build,
 *   J_mn = sum_ls (mn|ls) D_ls,     K_mn = sum_ls (ml|ns) D_ls,
 * and the nuclear gradient of E = tr(DJ)/2 - tr(DK)/4 at fixed D.  Around
 * that path: density screening for incremental builds, the one-electron
 * integrals of the SCF (Sec. 2.1) and the transform to pure d/f shells.
 * The atomic J/K reduction is the one of Sec. 6 ("each thread employs atomic
 * operations"), the pair/quartet blocking that of Sec. 4 (Block Constructor,
 * stages 1-2).
 *
 * Conventions
 *   - Units: bohr, hartree.  Cartesian shells.  Components ordered lx
 *     descending, then ly descending (d: xx xy xz yy yz zz).  Basis
 *     functions are ordered shell by shell as the caller lists them.
 *   - Primitive normalisation: N(a,l) = (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2l-1)!!);
 *     the library then rescales each shell's coefficients so that its
 *     contracted axial component x^l has unit norm.  Callers pass raw
 *     coefficients.
 *   - Screening: a shell quartet is evaluated iff Q_ab * Q_cd >= thresh,
 *     Q_ab = sqrt(max_i |(ab|ab)_ii|) (plain Schwarz; thresh <= 0 keeps all);
 *     mixed builds can also screen by density (JK_OPT_DENSITY_SCREEN).
 *   - Matrices D, J, K are nbf x nbf, row-major, contiguous float64 in DEVICE
 *     memory owned by the caller.  D must be symmetric (not checked unless
 *     JK_OPT_CHECK_SYMMETRY is set).  J and K are overwritten.
 *   - Every call is asynchronous on the given CUDA stream (NULL = legacy
 *     default stream) unless stated otherwise.
 *
 * Errors: every function returns JK_OK (0) or a negative status; the message
 * of the last failure on the calling thread is returned by jk_last_error().
 * No exception crosses this boundary.
 *
 * Device state: the library keeps per-device tables (the Boys-function grid,
 * the device address of jk_energy_noalloc's scratch) for the life of the
 * process.  They, and every handle, do not survive cudaDeviceReset: after a
 * reset of a device, call no entry point of this library on it again in the
 * same process.
 */
#ifndef GB300_ERI_H
#define GB300_ERI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    JK_OK = 0,
    JK_ERR_INVALID = -1,       /* bad argument (null pointer, negative size, ...) */
    JK_ERR_NOMEM = -2,         /* device or host allocation failed */
    JK_ERR_CUDA = -3,          /* a CUDA runtime call failed */
    JK_ERR_TIMEOUT = -4,       /* a bounded device wait gave up */
    JK_ERR_UNSUPPORTED = -5,   /* angular momentum above the compiled maximum */
    JK_ERR_NOT_SYMMETRIC = -6  /* D failed the optional symmetry check */
};

typedef enum { JK_FP64 = 0, JK_MIXED = 1 } jk_precision;

/* Atoms: natom centres, xyz[natom*3] in bohr, HOST memory, read during the call. */
typedef struct {
    int natom;
    const double* xyz;
} jk_atoms;

/* Shells (HOST memory, read during the call):
 *   atom[s]        centre index in [0, natom)
 *   l[s]           angular momentum, 0..JK_LMAX
 *   nprim[s]       number of primitives, >= 1
 *   prim_offset[s] first primitive of shell s in exps/coefs
 *   exps, coefs    exponents (> 0) and raw contraction coefficients */
typedef struct {
    int nshell;
    const int* atom;
    const int* l;
    const int* nprim;
    const int* prim_offset;
    const double* exps;
    const double* coefs;
} jk_shells;

#define JK_LMAX 3

/* Opaque handle: shell pairs, Schwarz factors and the quartet work lists,
 * resident in device memory and owned by the library until shellpairs_free. */
typedef struct jk_pairs_s* jk_pairs;

/* Block Constructor stage 1 + 2 (Sec. 4): normalise the shells, form every
 * unique shell pair and its primitive Gaussian products (p, P, K_AB c_a c_b),
 * compute the Schwarz factors from a diagonal (ab|ab) pass, sort the pairs
 * by angular class, primitive count and Q, and enumerate the surviving
 * quartet rows per class.  Synchronous: returns after the device work is
 * complete.  *out receives a new handle.  cuda_stream: cudaStream_t or NULL.
 * The arguments and the basis (l in 0..JK_LMAX and compiled, nprim >= 1,
 * atom index in range, exponents > 0, finite coefficients, coordinates and
 * threshold) are checked on the host before any CUDA call: a malformed input
 * returns JK_ERR_INVALID (JK_ERR_UNSUPPORTED for an l that is not compiled)
 * with *out = NULL and no device work. */
int shellpairs_build(const jk_atoms* atoms, const jk_shells* shells, double thresh,
                     jk_pairs* out, void* cuda_stream);

/* Sizes of a handle (any pointer may be NULL).
 *   nbf            number of Cartesian basis functions
 *   npairs         unique shell pairs kept (after the Q_ab * Q_max cut)
 *   nquartets      unique shell quartets surviving Schwarz (ab >= cd)
 *   nprimquartets  primitive quartets inside them */
int shellpairs_info(jk_pairs pairs, int* nbf, int64_t* npairs, int64_t* nquartets,
                    int64_t* nprimquartets);

/* J and K for one density (device pointers, nbf x nbf float64).
 * JK_FP64: every primitive quartet in FP64.  JK_MIXED: shell quartets whose
 * bound Q_ab Q_cd max|D| is below the mixed-precision cutoff tau
 * (jk_set_option) run in FP32 -- primitive arithmetic, contracted block and
 * the digestion dot products, from centre differences formed in FP64 --
 * and each digested sum is added to J and K in FP64 (split accumulation);
 * of the other quartets, the primitive quartets whose primitive Schwarz bound
 * q_p q_q max|D| reaches JK_OPT_PRIM_TAU run in FP64 and the rest in FP32
 * (JK_OPT_PRIM_TAU = 0: those quartets wholly FP64); the Schwarz factors and
 * the final J/K symmetrisation stay FP64, and the Boys function of FP32 quartets can be evaluated in FP64
 * below T = tsmall (JK_OPT_MIXED_TSMALL; default 0: the FP32 evaluation,
 * table and downward recursion, is as accurate there).  JK_FP64 accumulates J' and K'
 * with compensation (each update split into a multiple of 2^-32, summed
 * exactly while partial sums stay below 2^21, and a remainder summed
 * separately; handle-owned nbf x nbf scratch), so the result does not depend
 * on the order of the atomic updates beyond ~1e-20 per element.  The bound is density-weighted:
 * Q_ab Q_cd times the largest |D| element of the six shell blocks of D the
 * quartet's J and K updates read.  A JK_MIXED build synchronises the stream
 * once, after its split pass, to size its quartet lists; JK_FP64 builds are
 * fully asynchronous. */
int jk_build(jk_pairs pairs, const double* D, double* J, double* K, jk_precision prec,
             void* cuda_stream);

/* Nuclear gradient of E = tr(DJ)/2 - tr(DK)/4 at fixed D (device pointers):
 * dEdR[natom*3] (float64, device) is overwritten.  Derivative integrals by the
 * shift rule d phi_a/dA_i = 2 alpha phi_{a+1_i} - a_i phi_{a-1_i} on centres
 * A, B and C; the D centre by translational invariance.  Compiled for every
 * class up to (ff|ff) (a library built for a lower angular momentum returns
 * JK_ERR_UNSUPPORTED for classes above it).  JK_FP64: every derivative
 * integral in FP64.  JK_MIXED: the quartets whose density-weighted bound (as
 * in jk_build) is below JK_OPT_GRAD_TAU take FP32 derivative kernels (centre
 * differences formed in FP64, per-quartet sums added to dEdR in FP64), the
 * others FP64; this synchronises the stream once (list sizes) and leaves its
 * split in jk_last_split / jk_split_stats. */
int jk_grad(jk_pairs pairs, const double* D, double* dEdR, jk_precision prec, void* cuda_stream);

/* Multi-GPU split of one molecule (Sec. 4, stage 2: quartet blocks are
 * independent; Sec. 7 runs them over several GPUs).  The quartet rows of
 * every angular class are cut into nparts contiguous ranges of equal
 * algorithmic cost (the generator's operation count of each row's primitive
 * quartets and bra primitive pairs), so every part holds the same share of
 * every class, within the cost of one row.  jk_build_part computes J and K
 * (device, nbf x nbf, overwritten, symmetrised) from the quartets of part
 * `part` only; the sum of the nparts results is the full J and K (an
 * all-reduce across GPUs).  jk_grad_part likewise for dE/dR.  Precision and
 * stream as jk_build / jk_grad; the first call with a new nparts computes the
 * partition (one synchronisation) and caches it on the handle.
 * part outside [0, nparts) or nparts < 1: JK_ERR_INVALID. */
int jk_build_part(jk_pairs pairs, int part, int nparts, const double* D, double* J, double* K,
                  jk_precision prec, void* cuda_stream);
int jk_grad_part(jk_pairs pairs, int part, int nparts, const double* D, double* dEdR,
                 jk_precision prec, void* cuda_stream);

/* The partition rule used above, on the host (no device work): n consecutive
 * units of cost[n] (HOST, >= 0, finite) into nparts contiguous ranges;
 * bounds[nparts + 1] (HOST) receives 0 = b_0 <= b_1 <= ... <= b_nparts = n,
 * b_p the first unit at which the running cost reaches p/nparts of the total
 * (equal counts if the total is 0).  Every range then costs total/nparts
 * within the largest single cost.  JK_ERR_INVALID for a negative or
 * non-finite cost or nparts < 1. */
int jk_partition(int64_t n, const double* cost, int nparts, int64_t* bounds);

/* The row partition of a handle for nparts parts (host, synchronous on first
 * use): up to max_rows rows of 8 int64 -- bra class, ket class, part, first
 * row, end row, work items, algorithmic cost of the part, largest single-row
 * cost of the class -- for every class with work and every part.  *nrows
 * receives the number of rows. */
int jk_part_rows(jk_pairs pairs, int nparts, int max_rows, int64_t* rows, int* nrows);

/* Many independent molecules in one launch sequence (one persistent launch per
 * angular class over all molecules' work), optionally captured into a CUDA
 * graph (JK_OPT_GRAPH) that is replayed while the molecules, matrix pointers
 * and options stay the same.  The launch plan is cached across calls by the
 * identity of the handles (a handle built later never matches one freed
 * before, even at the same address) and shellpairs_free of any of its handles
 * releases it.  D[i], J[i], K[i] are device pointers of molecule i.
 * JK_MIXED: a split pass outside the graph selects the FP64 quartets as
 * jk_build does and synchronises once to size the lists. */
int jk_build_batched(int nmol, const jk_pairs* pairs, const double* const* D, double* const* J,
                     double* const* K, jk_precision prec, void* cuda_stream);

/* E = tr(DJ)/2 - tr(DK)/4 with a compensated device reduction; *E (host) is
 * written after the stream synchronises (synchronous). */
int jk_energy(int nbf, const double* D, const double* J, const double* K, double* E,
              void* cuda_stream);

/* jk_energy without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- hosts
 * that own all device memory through their own fixed-budget pool and forbid
 * libraries from allocating, or latency-critical loops where an allocation's
 * implicit device synchronisation is not acceptable.  The reduction's partial
 * sums live in a fixed file-scope device array of 16383 + 1 double2
 * (256 KiB), held by every GPU that loads the library until the process
 * exits.  nbf > 16383 is rejected with JK_ERR_INVALID (use jk_energy).
 * The first call on a device looks up that array's device address (a
 * one-time set-up per device); make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents;
 * calls that overlap on the GPU (different streams, no ordering) race on it
 * and must be serialised by the caller.  Arguments and result as jk_energy
 * (synchronous; *E is host memory). */
int jk_energy_noalloc(int nbf, const double* D, const double* J, const double* K, double* E,
                      void* cuda_stream);

/* Diagnostic: the device Boys evaluator used by the FP64 kernels (tabulated
 * Taylor grid + downward recursion, Sec. 2.2 "[00|00] analytically").
 * For each of n arguments T[i] (device, float64, T >= 0) writes
 * F[i*(L+1) + m] = F_m(T[i]), m = 0..L (device, float64).  L <= 13.
 * prec JK_MIXED evaluates the FP32 path used by mixed kernels (T >= tsmall). */
int jk_boys(int L, int n, const double* T, double* F, jk_precision prec, void* cuda_stream);

/* Tunables (process-wide). */
typedef enum {
    JK_OPT_MIXED_TAU = 0,        /* mixed path: FP32 iff Q_ab Q_cd max|D| < tau (default 5e-3) */
    JK_OPT_MIXED_TSMALL = 1,     /* mixed path: Boys of FP32 quartets in FP64 for T < tsmall (default 0:
                                  * measured to change no J/K/E error on the benchmark workloads, while
                                  * the FP64 branch kept the FP32 kernels' FP64 pipe busy) */
    JK_OPT_CHECK_SYMMETRY = 2,   /* nonzero: jk_build checks D == D^T first (synchronous):
                                  * JK_ERR_NOT_SYMMETRIC if not, JK_ERR_INVALID if D holds a NaN or
                                  * an infinity */
    JK_OPT_GRAPH = 3,            /* nonzero: jk_build_batched captures and replays a CUDA graph */
    JK_OPT_PROFILE = 4,          /* nonzero: jk_build records CUDA events around every class launch */
    JK_OPT_DENSITY_SCREEN = 5,   /* mixed builds (single and batched): skip a shell quartet whose bound
                                  * Q_ab Q_cd max|D| is below this value, with max|D| over the whole
                                  * matrix, and, for the quartets whose global bound reaches tau, over
                                  * the six D blocks the quartet reads (default 0: nothing is skipped).
                                  * For incremental builds, J(D) = J(D_prev) + J(D - D_prev): the
                                  * difference density makes the bounds small, so many quartets are
                                  * skipped.  Skipped quartets are counted in neither part of
                                  * jk_last_split. */
    JK_OPT_RPATH = 6,            /* nonzero: the FP32 kernels of (dd|dd), (dd|dp) and (dp|dp) evaluate
                                  * the Hermite R recursion in the order found by the greedy path
                                  * search of Algorithm 1 (Sec. 5, Graph Compiler; per kernel the
                                  * lambda of fewest operations) instead of the fixed t-u-v order
                                  * (default 1; 0: the fixed order).  Same integrals up to rounding. */
    JK_OPT_FAIL_ALLOC_AFTER = 7, /* fault injection for callers' error handling: n >= 0 lets n more
                                  * device allocations of the library succeed, then the next one
                                  * fails with JK_ERR_NOMEM (as if the device were full) and the
                                  * count stays at 0 (every later one fails) until the option is
                                  * set to a negative value (default -1: off).  No device memory
                                  * is touched by an injected failure. */
    JK_OPT_GRAD_TAU = 8,         /* mixed gradient (jk_grad with JK_MIXED): derivative integrals in FP32
                                  * for the quartets whose density-weighted bound (as for JK_OPT_MIXED_TAU)
                                  * is below this value, FP64 otherwise; every per-quartet gradient sum
                                  * is added to dE/dR in FP64 (default 3e-4) */
    JK_OPT_DF_TIER = 9,          /* mixed builds (single and batched): nonzero runs the quartets the
                                  * density-weighted bound keeps out of FP32 (l <= 2 classes) in
                                  * double-float arithmetic -- every value an unevaluated sum of two
                                  * floats, ~44 significant bits, all on the FP32 pipe -- instead of
                                  * FP64 (default 0); the FP64 build is unaffected */
    JK_OPT_PRIM_TAU = 10,        /* mixed builds (single and batched): primitive split of the quartets kept
                                  * out of FP32.  Each pair's primitive pairs carry their own Schwarz factor
                                  * q_p (shellpairs_build); of such a quartet only the primitive quartets
                                  * with q_p q_q max|D| >= this value (max|D| over the quartet's six D
                                  * blocks, as for JK_OPT_MIXED_TAU) run in FP64 / double-float, the others
                                  * in FP32, added into the same J and K.  0 turns the split off (every
                                  * primitive quartet of such a quartet in FP64 / double-float); default
                                  * 1e-4 */
    JK_OPT_GRAD_PRIM_TAU = 11    /* mixed gradient: the same primitive split of the quartets whose bound
                                  * reaches JK_OPT_GRAD_TAU -- their derivative integrals of primitive
                                  * quartets with q_p q_q max|D| below this value by the FP32 derivative
                                  * kernels, the others in FP64; 0 turns it off; default 1e-6 */
} jk_option;
int jk_set_option(jk_option opt, double value);
int jk_get_option(jk_option opt, double* value);

/* Diagnostic counters of the last jk_build on this handle (host, synchronous):
 * number of shell quartets run in FP32 and in FP64. */
int jk_last_split(jk_pairs pairs, int64_t* n_fp32, int64_t* n_fp64);

/* Workload Allocator (Sec. 6, Algorithm 2): per angular class, start at one
 * shell quartet per thread and keep doubling the quartets per thread
 * ("Combine") while the class's kernel gets faster, reverting otherwise,
 * until no class improves.  Timed with CUDA events on a prefix of each
 * class's work; J and K (device, nbf x nbf) are used as scratch and hold
 * meaningless values afterwards.  The chosen configuration is stored in the
 * handle and used by later jk_build calls of that precision.  Synchronous. */
int jk_autotune(jk_pairs pairs, const double* D, double* J, double* K, jk_precision prec, void* cuda_stream);

/* Read / restore the per-class launch configuration (e.g. a tuner cache kept
 * across runs): up to max_rows rows of 6 ints: bra class, ket class, FP64
 * block size, FP64 quartets per thread, FP32 block size, FP32 quartets per
 * thread.  Block sizes must be 32..128 in steps of 32. */
int jk_tuning(jk_pairs pairs, int max_rows, int* rows, int* nrows);
int jk_set_tuning(jk_pairs pairs, int nrows, const int* rows);

/* Number of kernels the last jk_build / jk_grad on this handle launched. */
int jk_last_launches(jk_pairs pairs, int64_t* nlaunch);

/* Per (bra class, ket class) work of a handle (host, synchronous).  Writes up
 * to max_rows rows of 6 int64: bra class, ket class (pair classes ordered
 * ss ps pp ds dp dd fs fp fd ff), shell quartets, primitive quartets,
 * (shell quartet x bra primitive pair) count, and the algorithmic FP64
 * operation count of the generated McMurchie-Davidson code for the whole
 * class.  *nrows receives the number of classes with work. */
int jk_class_stats(jk_pairs pairs, int max_rows, int64_t* rows, int* nrows);

/* Work of each precision in the last JK_MIXED jk_build on this handle (host,
 * synchronous; JK_ERR_INVALID if that build was not mixed).  Writes up to
 * max_rows rows of 8 int64: bra class, ket class, then for the FP32 quartets
 * and for the FP64 quartets each: shell quartets, primitive quartets and the
 * algorithmic operation count of the generated code (as jk_class_stats).
 * With the primitive split (JK_OPT_PRIM_TAU) the FP64 quartets' primitive
 * quartets and operations are the FP64 / double-float tier's share, and the
 * FP32 columns add the FP32 complement (the shell-quartet counts are those of
 * the quartet-level split).  *nrows receives the number of classes with work. */
int jk_split_stats(jk_pairs pairs, int max_rows, int64_t* rows, int* nrows);

/* Launch timings of the last jk_build with JK_OPT_PROFILE set (host,
 * synchronous): up to max_rows rows of 5 doubles: bra class, ket class,
 * precision (0 FP64, 1 FP32, 3 double-float, 4 the FP32 complement of a
 * primitively split FP64 list), shell quartets, milliseconds
 * (CUDA events on the build's stream).  *nrows receives the number of launches. */
int jk_profile(jk_pairs pairs, int max_rows, double* rows, int* nrows);

/* Diagnostic microbenchmark: sustained FMA throughput of this GPU's SIMT
 * pipes (prec JK_FP64: DFMA, JK_MIXED: FFMA), in FLOP/s (2 per FMA), timed
 * with CUDA events over `iters` dependent-chain iterations per thread. */
int jk_fma_peak(jk_precision prec, int iters, double* flops_per_s, void* cuda_stream);

/* One-electron integrals for the SCF around the J/K build (Sec. 2.1: the Fock
 * matrix is the one-electron part plus J - K/2): overlap S, kinetic energy T
 * and nuclear attraction V = -sum_C Z_C <a| 1/|r - R_C| |b>, with the nuclei
 * at the atoms given to shellpairs_build and charges[natom] (HOST, read during
 * the call).  S, T, V: DEVICE nbf x nbf row-major float64, caller-owned,
 * overwritten; the elements of shell pairs dropped by the Schwarz threshold
 * are 0 (build the handle with thresh 0 for the complete matrices).
 * Asynchronous on cuda_stream. */
int jk_one_electron(jk_pairs pairs, const double* charges, double* S, double* T, double* V, void* cuda_stream);

/* Limits compiled into this library (host, no device work): the highest
 * shell angular momentum shellpairs_build accepts and the highest one
 * jk_grad differentiates (both JK_LMAX = 3 in the default build). */
int jk_limits(int* lmax, int* grad_lmax);

/* Pure (real solid-harmonic) d and f shells.  The integrals of Sec. 2.2
 * (Eq. 1) are over Cartesian components; a basis with pure d/f shells is
 * served by transforming matrices between the two bases:
 *     D_cart = T D_pure T^T,  J_pure = T^T J_cart T,  K_pure = T^T K_cart T,
 * with T block-diagonal over the shells: identity for s and p (p stays x, y,
 * z), and for l = 2, 3 the 2l+1 real solid harmonics S_lm, m = -l..l (no
 * Condon-Shortley phase), each with the norm of the normalised axial
 * Cartesian component.  jk_build and jk_grad on D_cart then give the pure-
 * basis J/K and the gradient at fixed D_pure (T does not depend on the
 * geometry).  The pure basis orders shells as the Cartesian one does. */
typedef enum { JK_SPH_TO_CART = 0, JK_CART_TO_SPH = 1 } jk_sph_dir;

/* Number of pure basis functions of a handle (host, no device work). */
int jk_sph_nbf(jk_pairs pairs, int* nsph);

/* out = T in T^T (JK_SPH_TO_CART: in nsph x nsph, out nbf x nbf) or
 * out = T^T in T (JK_CART_TO_SPH: in nbf x nbf, out nsph x nsph); DEVICE
 * pointers, row-major float64, caller-owned; `in` and `out` must not overlap
 * (JK_ERR_INVALID).  Asynchronous on cuda_stream; the first call on a handle
 * also uploads the shell layout and the coefficient tables. */
int jk_sph_transform(jk_pairs pairs, jk_sph_dir dir, const double* in, double* out, void* cuda_stream);

void shellpairs_free(jk_pairs pairs);

/* Message of the last failure on the calling thread ("" if none). */
const char* jk_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GB300_ERI_H */
