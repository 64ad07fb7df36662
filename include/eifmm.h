/*
 * eifmm.h -- C ABI of the GB300 (sm_103a) library for the evaluation phase of
 * the Empirical Interpolation Fast Multipole Method (EIFMM) of F. Casenave,
 * "A Fast Summation Method for translation invariant kernels"
 * (arXiv:1408.0210).
 *
 * The library computes, for N targets x_i and sources y_j in a cube Omega,
 *     f(x_i) = sum_j sigma_j K(x_i, y_j),   K(x, y) = k(x - y)        (Eq. 1)
 * for many potential vectors sigma, with the multilevel EIFMM (Algorithm 3,
 * steps 1-7) for the far field and a direct sum over neighbouring leaves for
 * the near field f_N (Section 3.2).
 *
 * Calls:
 *   eifmm_training_sets / eifmm_eim_build   Algorithm 1 (offline, on the GPU)
 *   eifmm_ops_load / eifmm_ops_build        operator assembly (Section 4.1)
 *   eifmm_tree_build                        octree bin/sort (Section 3.3)
 *   eifmm_evaluate / _host / _batched       Algorithm 3 + near field
 *
 * General rules for every entry point:
 *   - no exceptions cross the ABI; every call returns an eifmm_status and, on
 *     failure, leaves a message for eifmm_last_error() (thread local);
 *   - opaque handles are owned by the library and freed by *_destroy;
 *   - "device" pointers are CUDA global-memory pointers of the current
 *     device; "host" pointers are ordinary process memory;
 *   - `stream` is a cudaStream_t (0 = legacy default stream); device work is
 *     enqueued on it and the call returns without waiting unless stated.
 *   - kernels are even functions (k(-z) = k(z)); the paper's second EIM
 *     (J_0, I_0) is then the transpose of the first (Section 3.3).
 */
#ifndef EIFMM_H
#define EIFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* eifmm_stream; /* same type as cudaStream_t */

typedef enum {
  EIFMM_OK = 0,
  EIFMM_EINVAL = 1,       /* invalid argument (null pointer, size, domain)   */
  EIFMM_ENOMEM = 2,       /* device or host allocation failed               */
  EIFMM_ECUDA = 3,        /* a CUDA call failed; see eifmm_last_error()      */
  EIFMM_ETIMEOUT = 4,     /* a bounded device-side wait gave up              */
  EIFMM_EUNSUPPORTED = 5  /* valid request this build does not implement    */
} eifmm_status;

/* Kernel k(z), z = x - y (Section 5 kernels plus test kernels). */
typedef enum {
  EIFMM_KERNEL_INV_R = 0,     /* 1/|z|  (Laplace, Section 5.3)                */
  EIFMM_KERNEL_CONFIG3 = 1,   /* exp(-|z|)/|z| + 1/sqrt(z0^2+0.01 z1^2+z2^2+1e-3) */
  EIFMM_KERNEL_QUAD = 2,      /* |z|^2: separable, rank 5 (exactness checks)  */
  EIFMM_KERNEL_ONE = 3,       /* 1: rank 1                                    */
  EIFMM_KERNEL_EXP_R2 = 4,    /* exp(-|z|^2)       (Section 5.4)              */
  EIFMM_KERNEL_COS20R_R = 5,  /* cos(20|z|)/|z|    (Section 5.4)              */
  EIFMM_KERNEL_SQRT_R2P1 = 6  /* sqrt(|z|^2 + 1)   (Section 5.4)              */
} eifmm_kernel;

/* Arithmetic of eifmm_evaluate.
 *   FP64:  every step in FP64 (the plain GPU EIFMM).
 *   MIXED: the arithmetic tier of the operators (eifmm_ops_plan,
 *          eifmm_ops_calibrate):
 *            tier 0: M2L on tcgen05 tensor cores with BF16 hi+lo operands (3
 *                    products, FP32 accumulation in several chains), P2M,
 *                    M2M, L2L, L2P, the Delta solves and the near field in
 *                    FP32 on coordinates local to each leaf;
 *            tier 1: M2L on tcgen05 with FP16 hi+lo operands (a power-of-
 *                    two scale per level for W and per coefficient for the
 *                    operator), each offset's FP32 accumulator drained from
 *                    tensor memory into round-to-nearest FP32 sums; FP32
 *                    elsewhere with one Newton step on every 1/r;
 *            tier 2: M2L on the FP32 SIMT pipes, each offset's sum in FP32
 *                    and the offsets added with compensated FP32 sums;
 *                    FP32 elsewhere with one Newton step on every 1/r;
 *            tier 3: far field in FP64 (its M2L in FP32 pairs, hi + lo,
 *                    with exact product splits: about 46 bits), near
 *                    field in FP32 (Kahan sums);
 *            tier 4: FP64 everywhere (near field too) but the M2L, which
 *                    runs in FP32 pairs as in tier 3.
 *          In every tier the M2L applies K^delta Delta (built once with
 *          FP64 solves) to W, so step 3 needs no solve.
 */
typedef enum { EIFMM_PREC_FP64 = 0, EIFMM_PREC_MIXED = 1 } eifmm_precision;

const char* eifmm_last_error(void);
const char* eifmm_version(void);

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Section 2): the EIM greedy, FP64 on the GPU.                */
/* ------------------------------------------------------------------------ */

/* Default training sets of level `level` >= 2 for a cube of side L (the paper
 * leaves them unspecified; Section 2 "training sets"):
 *   D_y: nJ^3 tensor grid on [-l_k, l_k]^3 including the faces (nJ >= 2);
 *   D_x: tensor product of the 1D nodes {0, +-1, ..., +-7} * l_k (while
 *        <= L - l_k) continued by a geometric progression of ratio 1.35 up
 *        to L - l_k, restricted to max-norm >= 3 l_k (the domain I_0^k).
 * l_k = L 2^-(level+1).  Row-major (n x 3) host arrays; pass X == NULL / Y ==
 * NULL to query the counts *nx / *ny only.  Errors: EINVAL for level < 2,
 * level > 10, nJ < 2, L <= 0 or null count pointers. */
eifmm_status eifmm_training_sets(int level, double L, int nJ, double* X,
                                 int64_t* nx, double* Y, int64_t* ny);

/* Algorithm 1 with the L-infinity norm on the grids X (nx x 3, D_x) and Y
 * (ny x 3, D_y), host FP64.  At each step the pivot is the first maximiser of
 * |delta_k K| in row-major (x, y) order; the loop stops before pivot k+1 when
 * |delta_k K(x_{k+1}, y_{k+1})| <= eps |Gamma_11| or when d_max pivots are
 * taken.  Host outputs (caller-owned):
 *   *d                      number of interpolation points d
 *   ia[d_max], ib[d_max]    training indices of x_k and y_k
 *   Gamma[d_max*d_max]      row-major, lower triangular (leading d x d)
 *   B[d_max*d_max]          row-major, unit lower triangular (leading d x d)
 *   piv[d_max+1]            |Gamma_kk| for k < d, then the first rejected pivot
 *   *eps_est                built-in error estimate piv[d]/piv[0] (Section 2)
 * For INV_R, QUAD and ONE the arithmetic is IEEE-exact (no fused multiply-add,
 * correctly rounded sqrt and divide), so the result is reproducible bit for
 * bit by any implementation that evaluates the same operations.  Device
 * scratch of nx*ny doubles is allocated and freed inside; the call
 * synchronises `stream`.  Errors: EINVAL (null pointers, nx/ny < 1, eps <= 0,
 * d_max < 1 or > 1024), ENOMEM, ECUDA. */
eifmm_status eifmm_eim_build(eifmm_kernel kern, const double* X, int64_t nx,
                             const double* Y, int64_t ny, double eps,
                             int d_max, int* d, int64_t* ia, int64_t* ib,
                             double* Gamma, double* B, double* piv,
                             double* eps_est, eifmm_stream stream);

/* ------------------------------------------------------------------------ */
/* Operators (Section 4.1 precomputations; M2L matrices of Section 4.2).    */
/* ------------------------------------------------------------------------ */
typedef struct eifmm_ops eifmm_ops;

/* EIM data of one level, host FP64, packed row-major: X = x_m^{I_0^k}
 * (d x 3), Y = y_l^{J_0^k} (d x 3), Gamma and B (d x d) from eifmm_eim_build. */
typedef struct {
  int d;
  const double* X;
  const double* Y;
  const double* Gamma;
  const double* B;
  double eps_est;
} eifmm_level_data;

/* Upload the EIM data of levels 2..depth (levels[k], entries 0 and 1 unused)
 * and assemble on the GPU, in FP64, the 2^D M2M operators
 * K_M2M^i = K^{I^k, J^{k+1}} Delta^{k+1} and the L2L operators
 * K_L2L^i = K' (Delta^{k-1})^t by triangular solves (Section 4.1), the 316
 * M2L matrices K^delta of every level (Section 4.2) and their reduced-
 * precision copies.  Ownership of the host arrays stays with the caller.
 * Errors: EINVAL (depth outside [2, 10], d outside [1, 512], null arrays,
 * L <= 0), ENOMEM, ECUDA. */
eifmm_status eifmm_ops_load(eifmm_kernel kern, double L, int depth,
                            const eifmm_level_data* levels, eifmm_ops** out);

/* Convenience: default training sets + eifmm_eim_build(eps, d_max) for every
 * level 2..depth + eifmm_ops_load + eifmm_ops_calibrate(eps).  Synchronises
 * `stream`. */
eifmm_status eifmm_ops_build(eifmm_kernel kern, double L, int depth,
                             double eps, int d_max, eifmm_stream stream,
                             eifmm_ops** out);

/* Built-in error estimate eps_k and rank d_k of level k (Section 2). */
eifmm_status eifmm_ops_error_estimate(const eifmm_ops* ops, int level,
                                      double* eps_k, int* d_k);

/* Arithmetic tier that EIFMM_PREC_MIXED uses with these operators:
 * 0 = BF16 hi+lo M2L and an FP32 far field, 1 = FP16 hi+lo M2L with per-offset
 * drains, 2 = FP32 SIMT M2L with compensated sums over the offsets,
 * 3 = FP64 far field (M2L in FP32 pairs), 4 = FP64 everywhere, the near
 * field too (M2L in FP32 pairs).  eifmm_ops_load sets it
 * from the built-in error estimate; `tier_override` >= 0 (at most 4) forces
 * a tier.  Errors: EINVAL (null ops, tier above 4). */
eifmm_status eifmm_ops_plan(eifmm_ops* ops, int tier_override, int* tier);

/* Measured choice of the tier (no counterpart in the paper, which computes in
 * FP64): a uniform problem of 32 points per leaf at depth min(depth, 4) is
 * evaluated in FP64 and in tiers 0, 1, 2, 3; the cheapest tier whose relative
 * L2 difference to FP64 is at most eps/4 is kept, else tier 4.  Allocates and
 * frees its own device memory; synchronises `stream`.  Errors: EINVAL,
 * ENOMEM, ECUDA. */
eifmm_status eifmm_ops_calibrate(eifmm_ops* ops, double eps, eifmm_stream stream,
                                 int* tier);

/* What the last eifmm_ops_calibrate measured: err4[t] is the relative L2
 * difference of tier t (t = 0..3) to FP64 on the calibration problem, or
 * -1 for a tier that was not evaluated (a cheaper one passed first, or its
 * operands could not be built); *tier the tier kept (-1 before any
 * calibration).  Either pointer may be NULL.  Errors: EINVAL (null ops). */
eifmm_status eifmm_ops_calibration(const eifmm_ops* ops, double* err4, int* tier);

/* M2L compression, first stage of Section 4.2, for the FP64 far field (the
 * FP64 path and the mixed tiers 3 and 4; the folded FP32 and tensor-core
 * tiers keep the full operators).  Per level, K_fat = [K^delta_1 ...
 * K^delta_316] (the unfolded M2L matrices of the far offsets); its leading
 * left singular vectors U (d x r) come from the eigen-decomposition of
 * K_fat K_fat^t in FP64, and r keeps what both filters of Section 4.2 keep:
 * the singular values with s_j / s_0 > eps, and the shortest leading run
 * whose sum reaches (1 - eps) of the total.  C^delta = U^t K^delta U (r x r)
 * replaces K^delta: step 4 becomes w~ = U^t What (What = Delta W by the FP64
 * solves), g~ = sum_J C^delta w~, g = U g~.  eps = 0 removes the
 * compression.  ranks (may be NULL): int[11], entry k = r of level k (0
 * outside 2..depth).  Synchronises `stream`.  Errors: EINVAL (null, eps
 * outside [0, 1), all-zero operators), ENOMEM, ECUDA. */
eifmm_status eifmm_ops_compress(eifmm_ops* ops, double eps, eifmm_stream stream,
                                int* ranks);

/* The compression basis of `level` (no counterpart in the paper; for
 * checks): U (HOST, d x r row-major, may be NULL), *d, *r (0 when the level
 * is not compressed), info (may be NULL): double[4] = {count of filter (i),
 * count of filter (ii), s_{r-1} / s_0, s_r / s_0}.  Synchronous.  Errors:
 * EINVAL (null handle, level outside [2, depth]), ECUDA. */
eifmm_status eifmm_ops_basis(const eifmm_ops* ops, int level, double* U, int* d,
                             int* r, double* info);

void eifmm_ops_destroy(eifmm_ops* ops);

/* ------------------------------------------------------------------------ */
/* Tree (Section 3.3): uniform octree, Morton order, stable bin/sort.       */
/* ------------------------------------------------------------------------ */
typedef struct eifmm_tree eifmm_tree;

/* Bin sources and targets into the 8^depth leaves of the cube
 * [lo, lo + L]^3: leaf coordinate floor((x - lo) * (2^depth / L)) clamped to
 * [0, 2^depth - 1], Morton key with the x bit lowest, stable sort by key (ties
 * keep the input order).  src_xyz / tgt_xyz are DEVICE arrays, row-major
 * n x 3 FP64; tgt_xyz may equal src_xyz.  exclude_self != 0 drops the pair
 * (i, i) and requires tgt_xyz == src_xyz.  lo is a host array of 3 doubles.
 * The tree keeps sorted copies; the inputs may be freed afterwards.  Errors:
 * EINVAL (null pointers, n < 0, depth outside [2, 10], L <= 0, a point
 * outside the cube, exclude_self with distinct sets), ENOMEM, ECUDA.
 * Synchronises `stream`. */
eifmm_status eifmm_tree_build(const double* src_xyz, int64_t n_src,
                              const double* tgt_xyz, int64_t n_tgt,
                              const double lo[3], double L, int depth,
                              int exclude_self, eifmm_stream stream,
                              eifmm_tree** out);

/* Copy the sorted Morton keys (n), the permutation perm[p] = input index of
 * sorted position p (n) and the leaf offsets (8^depth + 1) of the sources
 * (which = 0) or targets (which = 1) to HOST arrays; any output may be NULL.
 * Synchronous. */
eifmm_status eifmm_tree_export(const eifmm_tree* tree, int which,
                               uint32_t* keys, int32_t* perm,
                               int64_t* leaf_off);

/* Frees the tree and its workspace.  Evaluations of this tree that were
 * enqueued on the caller's streams must have finished (synchronise those
 * streams first); the library waits for its own streams of the tree. */
void eifmm_tree_destroy(eifmm_tree* tree);

/* Per-tree choices among equivalent kernels (no counterpart in the paper;
 * for comparisons and tests: every default is the fastest measured).
 *   M2L_128ROW: 1 runs the 128-row tensor-core M2L (M = target rows) where
 *     the transposed one (M = coefficients, N = 256 target rows) would run;
 *   P2P_PAIR_SYMMETRIC: 1 makes the tier-0 near field of one right-hand
 *     side with targets = sources visit each unordered leaf pair once;
 *   SINGLE_STREAM: 1 runs the whole evaluate on the caller's stream instead
 *     of the near field, far field and coarse M2L levels on streams of their
 *     own (the result is bitwise the same);
 *   M2L_FP64: 1 runs the FP64 M2L instead of the FP32-pair one in tiers 3
 *     and 4;
 *   M2L_STREAM_K: 1 runs the leaf-level transposed M2L as one CTA per SM
 *     over equal shares of the (tile, offset) work, split tiles added by a
 *     fix-up kernel, instead of one CTA per tile (at 2^20 points the launch
 *     is 2% shorter, but the evaluate slower: it holds every SM, so the
 *     near field cannot run beside it);
 *   NEAR_FIELD_LATE: 1 starts the mixed path's near field when the M2L
 *     starts (after the plane split of step 3) instead of with the far
 *     field, so that steps 1-3 run alone (at 2^20 points steps 1-3 take
 *     0.15 instead of 0.23 ms, but the near field then ends after the far
 *     field: 1.087 against 1.043 ms per evaluate).
 * The option holds for later evaluations of this tree.  Errors: EINVAL
 * (null tree, unknown option, value other than 0 or 1). */
typedef enum {
  EIFMM_OPT_M2L_128ROW = 0,
  EIFMM_OPT_P2P_PAIR_SYMMETRIC = 1,
  EIFMM_OPT_SINGLE_STREAM = 2,
  EIFMM_OPT_M2L_FP64 = 3,
  EIFMM_OPT_M2L_STREAM_K = 4,
  EIFMM_OPT_NEAR_FIELD_LATE = 5
} eifmm_option;
eifmm_status eifmm_tree_set_option(eifmm_tree* tree, eifmm_option opt, int value);

/* Morton bin/sort of one point set that allocates no memory at all.
 *
 * The paper has no counterpart.  This entry point serves callers that cannot
 * call cudaMalloc: programs whose device memory belongs to another allocator
 * (a framework's caching pool, which a raw cudaMalloc would bypass and could
 * starve of memory), programs that run inside a device-memory budget fixed
 * when they start, and loops that cannot pay for the implicit device-wide
 * synchronisation of cudaMalloc and cudaFree.
 *
 * It computes what eifmm_tree_build computes for the sources (same keys,
 * same stable permutation, same leaf offsets) into caller-owned DEVICE
 * arrays: keys_out[n] (sorted Morton keys), perm_out[n] (input index of
 * each sorted position) and leaf_off_out[8^depth + 1].  xyz is a DEVICE
 * row-major n x 3 FP64 array, lo a host array of 3 doubles.
 *
 * Scratch: the radix passes use a static device array of the library
 * (EIFMM_STATIC_SORT_SCRATCH_BYTES, about 8.5 MB), which every GPU that
 * loads the library holds until the process exits; n may not exceed
 * EIFMM_STATIC_SORT_MAX_POINTS (EINVAL otherwise, before any device work).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps
 * the last call's contents (the call clears the part that must start at
 * zero): calls that overlap on the GPU (concurrent streams, several host
 * threads) race on it and must be serialised by the caller.  The call
 * waits for `stream`: it copies the count of points outside the cube to
 * the host, synchronises the stream and returns EINVAL if the count is not
 * zero. */
#define EIFMM_STATIC_SORT_MAX_POINTS 1048576
#define EIFMM_STATIC_SORT_SCRATCH_BYTES 8913296
eifmm_status eifmm_tree_sort_static(const double* xyz, int64_t n,
                                    const double lo[3], double L, int depth,
                                    uint32_t* keys_out, int32_t* perm_out,
                                    int32_t* leaf_off_out,
                                    eifmm_stream stream);

/* ------------------------------------------------------------------------ */
/* Evaluation: Algorithm 3 (steps 1-7) + near field f_N (Section 3.2).      */
/* ------------------------------------------------------------------------ */

/* f = sum_j sigma_j K(x_i, y_j) for n_rhs potential vectors.  sigma and f are
 * DEVICE arrays, column-major: sigma[j + r*ld_sigma] (n_src x n_rhs), f[i +
 * r*ld_f] (n_tgt x n_rhs), both FP64 and in the caller's original point
 * order.  The ops must cover the tree's levels (ops depth >= tree depth;
 * levels deeper than the tree are not used) and have the tree's L.  The
 * tree owns the workspace; the first call for a given (ops, n_rhs) allocates
 * it and later calls allocate nothing.  Calls that share a tree must not
 * overlap.  sigma must be finite: the mixed path's library GEMMs (M2M,
 * L2L) do not carry infinities or NaNs through, so a non-finite sigma gives
 * an unspecified f.  Errors: EINVAL (null, n_rhs < 1 or > 256, ld < n, ops
 * depth below the tree's, L mismatch), ENOMEM, ECUDA. */
eifmm_status eifmm_evaluate(eifmm_tree* tree, const eifmm_ops* ops,
                            const double* sigma, int64_t ld_sigma, int n_rhs,
                            double* f, int64_t ld_f, eifmm_precision prec,
                            eifmm_stream stream);

/* Autotuner of the tensor-core M2L (step 4; the paper has no counterpart).
 * For the mixed path of tiers 0 and 1 it evaluates once with sigma = 0 (which
 * also sets up the workspace for n_rhs), then times at every level each
 * applicable M2L variant -- 1 transposed (M = coefficients, N = 256 target
 * rows), 2 128-row TMA, 3 transposed in stream-K form (leaf level) --
 * with the offset-group count halved, kept or doubled, against the built-in
 * rule (variant 0), using CUDA events on `stream`.  The fastest (by at least
 * 2% over the rule) is kept in the tree for later evaluations with the same
 * ops, n_rhs and precision.  For tier 0 with one right-hand side on a tree
 * whose targets are its sources it also times the near field (Section 3.2)
 * per target against its pair-symmetric form and keeps the faster (the
 * latter must win by 2%).  choice (may be null): int[2 * 11], entries 2k
 * and 2k+1 = variant and group shift of level k >= 2; entry 0 = 1 when the
 * pair-symmetric near field was kept.  Other paths and tiers:
 * nothing to tune, returns OK with zeros.  Synchronises `stream`.
 * Errors: as eifmm_evaluate. */
eifmm_status eifmm_autotune(eifmm_tree* tree, const eifmm_ops* ops, int n_rhs,
                            eifmm_precision prec, eifmm_stream stream, int* choice);

/* Same computation with HOST sigma and f (pinned memory recommended): the
 * call copies sigma to the device, evaluates, copies f back and synchronises
 * `stream` before returning. */
eifmm_status eifmm_evaluate_host(eifmm_tree* tree, const eifmm_ops* ops,
                                 const double* sigma_host, int64_t ld_sigma,
                                 int n_rhs, double* f_host, int64_t ld_f,
                                 eifmm_precision prec, eifmm_stream stream);

/* Many independent problems sharing one operator set (the paper's
 * many-query setting, Section 1; same kernel and L; each tree's depth at
 * most the operators'): problem p evaluates trees[p] with DEVICE sigma[p]
 * and f[p] (one RHS each, ld = n).  The problems run on 8 parallel branches
 * that fork from and join into `stream`, so the launches of small, uneven
 * problems overlap; largest estimated cost first, each problem goes to the
 * branch with the least estimated cost so far (cost: the leaf level's M2L,
 * boxes x d^2, plus the near field, targets x 27 x sources per leaf).
 * The first call evaluates them directly and records them into a CUDA
 * graph; a later call with the same trees, arrays, operators, precision,
 * tier and stream replays that graph with one launch.  The
 * library keeps one such graph per process (a call with other arguments
 * records a new one; destroying one of its trees or its operators drops
 * it).  The legacy default stream (NULL) is never captured: every call on it
 * evaluates directly.  Calls from several host threads are serialised.
 * Errors as eifmm_evaluate. */
eifmm_status eifmm_evaluate_batched(eifmm_tree* const* trees,
                                    const double* const* sigma,
                                    double* const* f, int n_problems,
                                    const eifmm_ops* ops,
                                    eifmm_precision prec,
                                    eifmm_stream stream);

/* Intermediates of the last eifmm_evaluate on this tree, copied to a HOST
 * array in the layout [box][rhs][m] (box in Morton order at `level`), FP64:
 *   what = 0 W (step 1-2), 1 What (step 3), 2 g (step 4), 3 l (step 5),
 *          4 lhat (step 6, level = depth), 5 f_far, 6 f_near (n_tgt x n_rhs
 *          column-major, original target order).
 * `n` is the capacity of `out` in doubles.  Synchronous.  Errors: EINVAL
 * when nothing was evaluated, the level is out of range, n is too small, or
 * (what 0-4) the operator set of that evaluation has been destroyed since. */
eifmm_status eifmm_debug_export(const eifmm_tree* tree, int what, int level,
                                double* out, int64_t n);

/* Exact sum of Eq. (1) on the GPU in FP64 (no approximation), for checking
 * accuracy: f[e + r*n_eval] = sum_j sigma[j + r*ld_sigma] K(x_{t_e}, y_j) with
 * t_e = tgt_idx[e] (DEVICE int64 array) or t_e = e when tgt_idx is NULL; the
 * pair t_e == j is skipped when exclude_self != 0.  tgt_xyz / src_xyz are
 * DEVICE row-major n x 3 arrays, sigma and f DEVICE column-major.  Errors:
 * EINVAL (null pointers, sizes), ECUDA. */
eifmm_status eifmm_direct_sum(eifmm_kernel kern, const double* tgt_xyz,
                              int64_t n_tgt, const double* src_xyz,
                              int64_t n_src, const double* sigma,
                              int64_t ld_sigma, int n_rhs, int exclude_self,
                              const int64_t* tgt_idx, int64_t n_eval,
                              double* f, eifmm_stream stream);

/* Measured arithmetic rates of the current GPU (no counterpart in the
 * paper): rates[0] FP32 FMA/s, rates[1] approximate reciprocal square roots/s
 * (rsqrt.approx.ftz.f32), rates[2] FP64 FMA/s, from register loops with 8
 * independent chains per thread over every SM, best of 3 timed runs.  They
 * are the roofline denominators of the point kernels and of the FP64 path.
 * Synchronises `stream`.  Errors: EINVAL (null), ENOMEM, ECUDA. */
eifmm_status eifmm_measure_rates(eifmm_stream stream, double* rates);

/* Self-test of failure detection (no counterpart in the paper).  Every wait
 * of the library's tensor-core kernels on an mbarrier is bounded (about 2 s
 * of clock cycles); when one runs out the kernel records a code in a device
 * error word, gives up its work, and the next evaluate returns ETIMEOUT.
 * This call runs that same bounded wait, with `limit_cycles`, on an mbarrier
 * that nothing completes, in a kernel that holds no copy, MMA or tensor
 * memory: it returns ETIMEOUT with *code (may be NULL) = 7, the code the
 * waiting kernel recorded, and leaves the context usable.  Synchronous.
 * Errors: EINVAL (negative limit), ENOMEM, ECUDA. */
eifmm_status eifmm_wait_selftest(int64_t limit_cycles, int* code);

/* Number of kernels this library has launched since it was loaded (all
 * devices, all threads). */
uint64_t eifmm_kernel_launches(void);

/* Device times (ms) of the last evaluate on this tree, recorded with CUDA
 * events on the launching stream when timing is on (eifmm_set_timing(1);
 * the evaluate then waits for its last event).  ms[20]: [0] sigma gather +
 * P2M (step 1), [1] M2M (2), [2] step 3 (Delta is folded into the M2L
 * operator: nothing in the FP64 path, the hi/lo operand planes of W in the
 * tensor-core tiers), [3] M2L (4), [4] L2L (5), [5] Delta^t solve (6);
 * mixed path: [6] L2P of the far field + wait for the near field, [7] sum +
 * un-permute; FP64 path: [6] wait for the near field, [7] L2P + sum +
 * un-permute (7); [8] the near-field launch alone (on the library's side
 * stream); [9 + k] the M2L launch of level k alone. */
void eifmm_set_timing(int on);
eifmm_status eifmm_last_step_times(const eifmm_tree* tree, float* ms20);

#ifdef __cplusplus
}
#endif
#endif /* EIFMM_H */
