/*
 * eifmm_oracle.h -- plain FP64 CPU oracle for the evaluation phase of the
 * Empirical Interpolation FMM (F. Casenave, "A Fast Summation Method for
 * translation invariant kernels", arXiv:1408.0210).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously-correct
 * reference that the GPU library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * GPU library never links, includes or calls anything here, and the two share
 * no code, headers, tables or constants.
 *
 * Conventions (all FP64, all host memory):
 *   - points are row-major n x 3 arrays (x0 y0 z0 x1 y1 z1 ...);
 *   - sigma / f are column-major n x nrhs with a leading dimension;
 *   - the kernel is K(x, y) = k(x - y) with an even k (k(-z) = k(z)), so the
 *     second EIM of Section 3.1 is the transpose of the first (Section 3.3,
 *     "one EIM by level" for symmetric kernels).
 *
 * Functions whose result is pinned only by invariants rather than by an
 * independent value say so in their comment; see the test suite for the pins.
 */
#ifndef EIFMM_ORACLE_H
#define EIFMM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_K_INV_R = 0,      /* 1/|z|                                            */
  ORC_K_CONFIG3 = 1,    /* exp(-|z|)/|z| + 1/sqrt(z0^2 + 0.01 z1^2 + z2^2 + 1e-3) */
  ORC_K_QUAD = 2,       /* |z|^2 (separable rank 5)                         */
  ORC_K_ONE = 3,        /* 1 (rank 1)                                       */
  ORC_K_EXP_R2 = 4,     /* exp(-|z|^2)                                      */
  ORC_K_COS20R_R = 5,   /* cos(20|z|)/|z|                                   */
  ORC_K_SQRT_R2P1 = 6   /* sqrt(|z|^2 + 1)                                  */
};

#define ORC_MAX_LEVEL 10

/* k(z) for kernel id `kern`. */
double orc_kernel(int kern, double z0, double z1, double z2);

/* O1, Eq. (1): f_i = sum_j sigma_j K(xbar_i, ybar_j), pair i == j skipped
 * when exclude_self != 0.  If tgt_idx != NULL only the n_eval targets listed
 * there are evaluated (f is n_eval x nrhs, ld n_eval); otherwise n_eval must
 * equal nt.  Sequential summation in source order, OpenMP over targets. */
void orc_direct_sum(int kern, const double* tgt, int64_t nt, const double* src,
                    int64_t ns, const double* sigma, int64_t ld_sigma, int nrhs,
                    int exclude_self, const int64_t* tgt_idx, int64_t n_eval,
                    double* f);
/* Same sum accumulated in long double (used to pin the FP64 summation). */
void orc_direct_sum_ld(int kern, const double* tgt, int64_t nt,
                       const double* src, int64_t ns, const double* sigma,
                       int64_t ld_sigma, int nrhs, int exclude_self,
                       const int64_t* tgt_idx, int64_t n_eval, double* f);

/* Uniform 2^D-tree of Section 3.3: leaf coordinate
 * floor((x - lo) * (2^depth / L)) clamped to [0, 2^depth - 1], Morton key with
 * the x bit lowest.  Returns the number of points outside [lo, lo + L]^3. */
int64_t orc_morton_keys(const double* xyz, int64_t n, const double lo[3],
                        double L, int depth, uint32_t* keys);
/* Stable sort of the points by key (ties by original index):
 * perm[p] = original index of sorted position p; leaf_off has 8^depth + 1
 * entries. */
void orc_sort_leaves(const uint32_t* keys, int64_t n, int depth, int32_t* perm,
                     int64_t* leaf_off);

/* Training sets of the EIM at level k (reading of Section 2, "training
 * sets"): D_y is the nJ^3 tensor grid on [-l_k, l_k]^3 including the faces;
 * D_x is the tensor product of a 1D node set (unit steps of l_k up to 7 l_k,
 * then a geometric progression of ratio 1.35 up to L - l_k) restricted to
 * max-norm >= 3 l_k.  Return the number of points; write them if ptr != NULL. */
int64_t orc_train_x(int level, double L, double* X);
int64_t orc_train_y(int level, double L, int nJ, double* Y);

/* Algorithm 1 (EIM greedy) with the L-infinity norm: at each step the pivot
 * (x_{k+1}, y_{k+1}) is the first maximiser of |delta_k K| over the training
 * grid (row-major order), B_{k+1,m} = q_m(y_{k+1}) and the row k+1 of Gamma is
 * the pivot on the diagonal and alpha (the recursion of Section 2) below it.
 * Stops before pivot k+1 when |delta_k K(x_{k+1}, y_{k+1})| <= eps |Gamma_11|
 * or when d_max points are taken.  Gamma and B are d_max x d_max row-major
 * (only the leading d x d block is written).  ia/ib receive the training
 * indices of x_k and y_k; piv[k] = |Gamma_kk| for k < d and piv[d] = the
 * first rejected pivot magnitude (0 if the grid is exhausted); *eps_est =
 * piv[d] / piv[0].  Returns d. */
int orc_eim(int kern, const double* X, int64_t nx, const double* Y, int64_t ny,
            double eps, int d_max, int64_t* ia, int64_t* ib, double* Gamma,
            double* B, double* piv, double* eps_est);

/* Delta v = B^-t Gamma^-1 v and Delta^t v = Gamma^-t B^-1 v by the two
 * triangular solves of Section 4.1 (in place, Gamma/B packed d x d). */
void orc_apply_delta(int d, const double* Gamma, const double* B, double* v);
void orc_apply_delta_t(int d, const double* Gamma, const double* B, double* v);

/* EIM data of one level (the symmetric-kernel single EIM (I_0^k, J_0^k)). */
typedef struct {
  int d;
  const double* X;      /* d x 3: x_m^{I_0^k} (= y_m^{I_0^k})          */
  const double* Y;      /* d x 3: y_l^{J_0^k} (= x_l^{J_0^k})          */
  const double* Gamma;  /* d x d row-major, lower triangular          */
  const double* B;      /* d x d row-major, unit lower triangular     */
  /* Optional M2L compression (Section 4.2, first stage): r > 0 columns of
   * U (d x r row-major, orthonormal), the kept left singular vectors of
   * K_fat = [K^delta_1 ... K^delta_316].  Step 4 then applies
   * C^delta = U^t K^delta U of size r x r between the projections
   * w~ = U^t What and g = U g~.  r = 0: the full d x d M2L. */
  int r;
  const double* U;
} orc_level;

/* The M2L operators of level k (Eq. M2Lstep): Kd[t][m'][l] =
 * K(x_{m'}^{J_0^k}, y_l^{J_0^k} + delta_t) for the 343 offsets
 * t = (dx+3) + 7 (dy+3) + 49 (dz+3), delta_t = 2 l_k (dx, dy, dz); zero for
 * the 27 offsets of the neighbourhood.  Y (d x 3) holds the interpolation
 * points.  Returns the count of shifted points outside I_0. */
int64_t orc_m2l_operators(int kern, double L, int k, int d, const double* Y, double* Kd);

/* Optional intermediate results, canonical layout [box][rhs][m] with the
 * box index in Morton order at its level; any pointer may be NULL. */
typedef struct {
  double* W[ORC_MAX_LEVEL + 1];
  double* What[ORC_MAX_LEVEL + 1];
  double* g[ORC_MAX_LEVEL + 1];
  double* l[ORC_MAX_LEVEL + 1];
  double* lhat;     /* leaf level */
  double* f_far;    /* n_tgt x nrhs column-major, original target order */
  double* f_near;
  int64_t domain_violations; /* shifted evaluation points outside I_0/J_0 */
  int64_t m2l_pairs;         /* (I, J) pairs visited by step 4            */
  int64_t p2p_pairs;         /* (i, j) pairs visited by the near field    */
} orc_dump;

/* O2: Algorithm 3 (steps 1-7) plus the near field f_N, FP64, plain loops.
 * lv[k] is used for k = 2..depth.  f is n_tgt x nrhs (ld_f).  Returns 0, or
 * a negative value for invalid arguments. */
int orc_eifmm(int kern, double L, const double lo[3], int depth,
              const orc_level* lv, const double* tgt, int64_t nt,
              const double* src, int64_t ns, const double* sigma,
              int64_t ld_sigma, int nrhs, int exclude_self, double* f,
              int64_t ld_f, orc_dump* dump);

/* Interaction list I(I) of box `box` (Morton index) at level k (Section
 * 3.3.2): fills up to 189 Morton indices, returns the count. */
int orc_interaction_list(int level, int64_t box, int64_t* out);
/* Neighbourhood N(I) (boxes at max-norm coordinate distance <= 1). */
int orc_neighbours(int level, int64_t box, int64_t* out);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
