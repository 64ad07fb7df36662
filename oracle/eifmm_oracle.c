/*
 * eifmm_oracle.c -- plain FP64 CPU oracle for the EIFMM evaluation path of
 * arXiv:1408.0210 (F. Casenave).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the GPU library.  Everything is
 * written as plain loops that follow the paper's formulas in the paper's
 * order; OpenMP only splits independent outer loops (targets, boxes) and
 * never changes the order of any floating-point sum.  Built with
 * -ffp-contract=off so that no multiply-add is fused.
 */
#include "eifmm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Kernels: K(x, y) = k(x - y), Section 3.1 (translation invariance).       */
/* ------------------------------------------------------------------------ */
double orc_kernel(int kern, double z0, double z1, double z2) {
  double r2 = z0 * z0 + z1 * z1 + z2 * z2;
  switch (kern) {
    case ORC_K_INV_R:
      return 1.0 / sqrt(r2);
    case ORC_K_CONFIG3: {
      double r = sqrt(r2);
      double a = z0 * z0 + 0.01 * (z1 * z1) + z2 * z2 + 1e-3;
      return exp(-r) / r + 1.0 / sqrt(a);
    }
    case ORC_K_QUAD:
      return r2;
    case ORC_K_ONE:
      return 1.0;
    case ORC_K_EXP_R2:
      return exp(-r2);
    case ORC_K_COS20R_R: {
      double r = sqrt(r2);
      return cos(20.0 * r) / r;
    }
    case ORC_K_SQRT_R2P1:
      return sqrt(r2 + 1.0);
    default:
      return NAN;
  }
}

static double kxy(int kern, const double* x, const double* y) {
  return orc_kernel(kern, x[0] - y[0], x[1] - y[1], x[2] - y[2]);
}

/* ------------------------------------------------------------------------ */
/* O1: the exact sum of Eq. (1).                                            */
/* ------------------------------------------------------------------------ */
void orc_direct_sum(int kern, const double* tgt, int64_t nt, const double* src,
                    int64_t ns, const double* sigma, int64_t ld_sigma, int nrhs,
                    int exclude_self, const int64_t* tgt_idx, int64_t n_eval,
                    double* f) {
  (void)nt;
  int64_t e;
#pragma omp parallel for schedule(dynamic, 16)
  for (e = 0; e < n_eval; ++e) {
    int64_t i = tgt_idx ? tgt_idx[e] : e;
    for (int r = 0; r < nrhs; ++r) {
      double s = 0.0;
      for (int64_t j = 0; j < ns; ++j) {
        if (exclude_self && j == i) continue;
        s += sigma[j + r * ld_sigma] * kxy(kern, tgt + 3 * i, src + 3 * j);
      }
      f[e + r * n_eval] = s;
    }
  }
}

void orc_direct_sum_ld(int kern, const double* tgt, int64_t nt,
                       const double* src, int64_t ns, const double* sigma,
                       int64_t ld_sigma, int nrhs, int exclude_self,
                       const int64_t* tgt_idx, int64_t n_eval, double* f) {
  (void)nt;
  int64_t e;
#pragma omp parallel for schedule(dynamic, 16)
  for (e = 0; e < n_eval; ++e) {
    int64_t i = tgt_idx ? tgt_idx[e] : e;
    for (int r = 0; r < nrhs; ++r) {
      long double s = 0.0L;
      for (int64_t j = 0; j < ns; ++j) {
        if (exclude_self && j == i) continue;
        s += (long double)sigma[j + r * ld_sigma] *
             (long double)kxy(kern, tgt + 3 * i, src + 3 * j);
      }
      f[e + r * n_eval] = (double)s;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Tree (Section 3.3: kappa + 1 levels, level k has 2^k boxes per axis).    */
/* ------------------------------------------------------------------------ */
static uint32_t morton3(uint32_t ix, uint32_t iy, uint32_t iz, int depth) {
  uint32_t key = 0;
  for (int b = 0; b < depth; ++b) {
    key |= ((ix >> b) & 1u) << (3 * b);
    key |= ((iy >> b) & 1u) << (3 * b + 1);
    key |= ((iz >> b) & 1u) << (3 * b + 2);
  }
  return key;
}

static void demorton3(int64_t key, int depth, int64_t c[3]) {
  c[0] = c[1] = c[2] = 0;
  for (int b = 0; b < depth; ++b) {
    c[0] |= ((key >> (3 * b)) & 1) << b;
    c[1] |= ((key >> (3 * b + 1)) & 1) << b;
    c[2] |= ((key >> (3 * b + 2)) & 1) << b;
  }
}

static int64_t morton_of(const int64_t c[3], int depth) {
  return (int64_t)morton3((uint32_t)c[0], (uint32_t)c[1], (uint32_t)c[2], depth);
}

int64_t orc_morton_keys(const double* xyz, int64_t n, const double lo[3],
                        double L, int depth, uint32_t* keys) {
  const double scale = ldexp(1.0, depth) / L;
  const int64_t nmax = ((int64_t)1 << depth) - 1;
  int64_t outside = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t c[3];
    for (int a = 0; a < 3; ++a) {
      double x = xyz[3 * i + a];
      if (!(x >= lo[a] && x <= lo[a] + L)) ++outside;
      double t = floor((x - lo[a]) * scale);
      int64_t v = (int64_t)t;
      if (!(t >= 0.0)) v = 0;
      if (v > nmax) v = nmax;
      c[a] = v;
    }
    keys[i] = (uint32_t)morton_of(c, depth);
  }
  return outside;
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

void orc_sort_leaves(const uint32_t* keys, int64_t n, int depth, int32_t* perm,
                     int64_t* leaf_off) {
  uint64_t* kv = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) kv[i] = ((uint64_t)keys[i] << 32) | (uint64_t)i;
  qsort(kv, (size_t)n, sizeof(uint64_t), cmp_u64);
  const int64_t nleaf = (int64_t)1 << (3 * depth);
  for (int64_t b = 0; b <= nleaf; ++b) leaf_off[b] = 0;
  for (int64_t p = 0; p < n; ++p) {
    perm[p] = (int32_t)(kv[p] & 0xffffffffu);
    leaf_off[(kv[p] >> 32) + 1] += 1;
  }
  for (int64_t b = 0; b < nleaf; ++b) leaf_off[b + 1] += leaf_off[b];
  free(kv);
}

/* ------------------------------------------------------------------------ */
/* Training sets (reading of Section 2: the paper leaves them unspecified). */
/* ------------------------------------------------------------------------ */
#define ORC_TRAIN_RATIO 1.35
#define ORC_TRAIN_UNIFORM 7.0

/* 1D node values in units of l_k, symmetric, ascending. */
static int nodes_1d(int level, double* out) {
  const double M = ldexp(1.0, level + 1) - 1.0; /* (L - l_k) / l_k */
  double pos[256];
  int np = 0;
  pos[np++] = 0.0;
  double t = 1.0;
  while (t <= ORC_TRAIN_UNIFORM && t <= M) {
    pos[np++] = t;
    t += 1.0;
  }
  t = pos[np - 1];
  while (t < M) {
    t = t * ORC_TRAIN_RATIO;
    if (t > M) t = M;
    pos[np++] = t;
  }
  int n = 0;
  for (int i = np - 1; i >= 1; --i) {
    if (out) out[n] = -pos[i];
    ++n;
  }
  for (int i = 0; i < np; ++i) {
    if (out) out[n] = pos[i];
    ++n;
  }
  return n;
}

int64_t orc_train_x(int level, double L, double* X) {
  double u[512];
  int n = nodes_1d(level, u);
  const double l = L * ldexp(1.0, -(level + 1));
  int64_t cnt = 0;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c) {
        double m = fabs(u[a]);
        if (fabs(u[b]) > m) m = fabs(u[b]);
        if (fabs(u[c]) > m) m = fabs(u[c]);
        if (m < 3.0) continue; /* I_0^k: max-norm >= 3 l_k */
        if (X) {
          X[3 * cnt + 0] = u[a] * l;
          X[3 * cnt + 1] = u[b] * l;
          X[3 * cnt + 2] = u[c] * l;
        }
        ++cnt;
      }
  return cnt;
}

int64_t orc_train_y(int level, double L, int nJ, double* Y) {
  const double l = L * ldexp(1.0, -(level + 1));
  int64_t cnt = 0;
  for (int a = 0; a < nJ; ++a)
    for (int b = 0; b < nJ; ++b)
      for (int c = 0; c < nJ; ++c) {
        if (Y) {
          Y[3 * cnt + 0] = ((double)(2 * a - (nJ - 1)) / (double)(nJ - 1)) * l;
          Y[3 * cnt + 1] = ((double)(2 * b - (nJ - 1)) / (double)(nJ - 1)) * l;
          Y[3 * cnt + 2] = ((double)(2 * c - (nJ - 1)) / (double)(nJ - 1)) * l;
        }
        ++cnt;
      }
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, the EIM greedy, with Gamma by the recursion of Section 2.   */
/* ------------------------------------------------------------------------ */
int orc_eim(int kern, const double* X, int64_t nx, const double* Y, int64_t ny,
            double eps, int d_max, int64_t* ia, int64_t* ib, double* Gamma,
            double* B, double* piv, double* eps_est) {
  const int64_t nn = nx * ny;
  /* R holds delta_k K on the training grid: R[i][j] = (delta_k K)(x_i, y_j). */
  double* R = (double*)malloc(sizeof(double) * (size_t)(nn > 0 ? nn : 1));
  /* q[m][j] = q_m(y_j), the basis functions of Algorithm 1. */
  double* q = (double*)malloc(sizeof(double) * (size_t)((d_max > 0 ? d_max : 1) * ny));
  double* col = (double*)malloc(sizeof(double) * (size_t)(nx > 0 ? nx : 1));
  int64_t i;
#pragma omp parallel for
  for (i = 0; i < nx; ++i)
    for (int64_t j = 0; j < ny; ++j) R[i * ny + j] = kxy(kern, X + 3 * i, Y + 3 * j);

  double g11 = 0.0;
  int d = 0;
  *eps_est = 0.0;
  for (;;) {
    /* argmax over the grid of |delta_d K|, first maximiser in row-major
     * order: the x-argmax of the L-infinity norm, then the y-argmax. */
    int64_t best = 0;
    double bv = -1.0;
#pragma omp parallel
    {
      int64_t lb = 0;
      double lv = -1.0;
#pragma omp for schedule(static)
      for (int64_t t = 0; t < nn; ++t) {
        double v = fabs(R[t]);
        if (v > lv) { lv = v; lb = t; }
      }
#pragma omp critical
      {
        if (lv > bv || (lv == bv && lb < best)) { bv = lv; best = lb; }
      }
    }
    if (nn == 0) bv = 0.0;
    const int64_t a = nn ? best / ny : 0, b = nn ? best % ny : 0;
    const double p = nn ? R[best] : 0.0;
    if (d == 0) g11 = fabs(p);
    piv[d] = fabs(p);
    if (d == d_max || p == 0.0 || fabs(p) <= eps * g11) {
      *eps_est = g11 > 0.0 ? fabs(p) / g11 : 0.0;
      break;
    }
    ia[d] = a;
    ib[d] = b;
    /* q_{d+1} = (delta_d K)(x_{d+1}, .) / (delta_d K)(x_{d+1}, y_{d+1}) */
    for (int64_t j = 0; j < ny; ++j) q[(int64_t)d * ny + j] = R[a * ny + j] / p;
    /* B_{d+1, m} = q_m(y_{d+1}), unit diagonal. */
    for (int m = 0; m < d; ++m) B[(int64_t)d * d_max + m] = q[(int64_t)m * ny + b];
    B[(int64_t)d * d_max + d] = 1.0;
    /* Gamma_{d+1, d+1} = pivot, Gamma_{d+1, m} = alpha_m with
     * sum_{m'} B_{l m'} alpha_{m'} = K(x_{d+1}, y_l), l = 1..d. */
    for (int m = 0; m < d; ++m) {
      double s = kxy(kern, X + 3 * a, Y + 3 * ib[m]);
      for (int mm = 0; mm < m; ++mm)
        s -= B[(int64_t)m * d_max + mm] * Gamma[(int64_t)d * d_max + mm];
      Gamma[(int64_t)d * d_max + m] = s;
    }
    Gamma[(int64_t)d * d_max + d] = p;
    /* delta_{d+1} K = delta_d K - (delta_d K)(., y_{d+1}) q_{d+1}(.) */
    for (int64_t t = 0; t < nx; ++t) col[t] = R[t * ny + b];
#pragma omp parallel for
    for (i = 0; i < nx; ++i) {
      const double ci = col[i];
      for (int64_t j = 0; j < ny; ++j) R[i * ny + j] = R[i * ny + j] - ci * q[(int64_t)d * ny + j];
    }
    /* the new residual vanishes exactly on x_{d+1} and on y_{d+1} */
    for (int64_t j = 0; j < ny; ++j) R[a * ny + j] = 0.0;
    for (int64_t t = 0; t < nx; ++t) R[t * ny + b] = 0.0;
    ++d;
  }
  free(R);
  free(q);
  free(col);
  return d;
}

/* ------------------------------------------------------------------------ */
/* Section 4.1: Delta = B^-t Gamma^-1 applied by two triangular solves.     */
/* ------------------------------------------------------------------------ */
void orc_apply_delta(int d, const double* G, const double* B, double* v) {
  for (int i = 0; i < d; ++i) { /* Gamma z = v */
    double s = v[i];
    for (int m = 0; m < i; ++m) s -= G[i * d + m] * v[m];
    v[i] = s / G[i * d + i];
  }
  for (int i = d - 1; i >= 0; --i) { /* B^t w = z */
    double s = v[i];
    for (int m = i + 1; m < d; ++m) s -= B[m * d + i] * v[m];
    v[i] = s;
  }
}

void orc_apply_delta_t(int d, const double* G, const double* B, double* v) {
  for (int i = 0; i < d; ++i) { /* B z = v */
    double s = v[i];
    for (int m = 0; m < i; ++m) s -= B[i * d + m] * v[m];
    v[i] = s;
  }
  for (int i = d - 1; i >= 0; --i) { /* Gamma^t w = z */
    double s = v[i];
    for (int m = i + 1; m < d; ++m) s -= G[m * d + i] * v[m];
    v[i] = s / G[i * d + i];
  }
}

/* ------------------------------------------------------------------------ */
/* Box lists (Section 3.2 neighbourhood, Section 3.3.2 interaction list).  */
/* ------------------------------------------------------------------------ */
int orc_interaction_list(int level, int64_t box, int64_t* out) {
  int64_t c[3], lo_[3], hi_[3];
  const int64_t n = (int64_t)1 << level;
  demorton3(box, level, c);
  for (int a = 0; a < 3; ++a) {
    int64_t p = c[a] >> 1;
    lo_[a] = 2 * (p - 1);
    hi_[a] = 2 * (p + 1) + 1;
    if (lo_[a] < 0) lo_[a] = 0;
    if (hi_[a] > n - 1) hi_[a] = n - 1;
  }
  int cnt = 0;
  int64_t j[3];
  for (j[2] = lo_[2]; j[2] <= hi_[2]; ++j[2])
    for (j[1] = lo_[1]; j[1] <= hi_[1]; ++j[1])
      for (j[0] = lo_[0]; j[0] <= hi_[0]; ++j[0]) {
        if (llabs(j[0] - c[0]) <= 1 && llabs(j[1] - c[1]) <= 1 && llabs(j[2] - c[2]) <= 1)
          continue; /* not well separated */
        out[cnt++] = morton_of(j, level);
      }
  return cnt;
}

int orc_neighbours(int level, int64_t box, int64_t* out) {
  int64_t c[3];
  const int64_t n = (int64_t)1 << level;
  demorton3(box, level, c);
  int cnt = 0;
  int64_t j[3];
  for (j[2] = c[2] - 1; j[2] <= c[2] + 1; ++j[2])
    for (j[1] = c[1] - 1; j[1] <= c[1] + 1; ++j[1])
      for (j[0] = c[0] - 1; j[0] <= c[0] + 1; ++j[0]) {
        if (j[0] < 0 || j[1] < 0 || j[2] < 0 || j[0] >= n || j[1] >= n || j[2] >= n) continue;
        out[cnt++] = morton_of(j, level);
      }
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* O2: Algorithm 3 plus the near field.                                     */
/* ------------------------------------------------------------------------ */
static double half_width(double L, int k) { return L * ldexp(1.0, -(k + 1)); } /* l_k */

static void box_center(const double lo[3], double L, int k, int64_t box, double c[3]) {
  int64_t ic[3];
  demorton3(box, k, ic);
  const double l = half_width(L, k);
  for (int a = 0; a < 3; ++a) c[a] = lo[a] + (double)(2 * ic[a] + 1) * l;
}

static double maxnorm(const double z[3]) {
  double m = fabs(z[0]);
  if (fabs(z[1]) > m) m = fabs(z[1]);
  if (fabs(z[2]) > m) m = fabs(z[2]);
  return m;
}

static int in_J0(const double z[3], double l) { return maxnorm(z) <= l * (1.0 + 1e-12); }
static int in_I0(const double z[3], double l, double L) {
  double m = maxnorm(z);
  return m >= 3.0 * l * (1.0 - 1e-12) && m <= (L - l) * (1.0 + 1e-12);
}

int64_t orc_m2l_operators(int kern, double L, int k, int d, const double* Y, double* Kd) {
  const double lk = half_width(L, k);
  int64_t viol = 0;
  memset(Kd, 0, sizeof(double) * (size_t)(343 * d * d));
  for (int t = 0; t < 343; ++t) {
    const int dx = t % 7 - 3, dy = (t / 7) % 7 - 3, dz = t / 49 - 3;
    if (abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1) continue;
    const double dl[3] = {2.0 * dx * lk, 2.0 * dy * lk, 2.0 * dz * lk};
    for (int mp = 0; mp < d; ++mp) {
      const double* x = Y + 3 * mp;
      const double xm[3] = {x[0] - dl[0], x[1] - dl[1], x[2] - dl[2]};
      if (!in_I0(xm, lk, L)) ++viol;
      for (int l = 0; l < d; ++l) {
        const double* y = Y + 3 * l;
        const double ys[3] = {y[0] + dl[0], y[1] + dl[1], y[2] + dl[2]};
        Kd[((int64_t)t * d + mp) * d + l] = kxy(kern, x, ys);
      }
    }
  }
  return viol;
}

int orc_eifmm(int kern, double L, const double lo[3], int depth,
              const orc_level* lv, const double* tgt, int64_t nt,
              const double* src, int64_t ns, const double* sigma,
              int64_t ld_sigma, int nrhs, int exclude_self, double* f,
              int64_t ld_f, orc_dump* dump) {
  if (depth < 2 || depth > ORC_MAX_LEVEL || nrhs < 1 || L <= 0.0) return -1;
  if (exclude_self && nt != ns) return -2;
  const int kap = depth;
  const int R = nrhs;
  int64_t viol = 0, m2l_pairs = 0, p2p_pairs = 0;

  /* tree of targets and of sources */
  const int64_t nleaf = (int64_t)1 << (3 * kap);
  uint32_t* kt = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(nt + 1));
  uint32_t* ks = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(ns + 1));
  int32_t* pt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nt + 1));
  int32_t* ps = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ns + 1));
  int64_t* ot = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nleaf + 1));
  int64_t* os = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nleaf + 1));
  orc_morton_keys(tgt, nt, lo, L, kap, kt);
  orc_morton_keys(src, ns, lo, L, kap, ks);
  orc_sort_leaves(kt, nt, kap, pt, ot);
  orc_sort_leaves(ks, ns, kap, ps, os);

  int64_t nb[ORC_MAX_LEVEL + 1];
  for (int k = 0; k <= kap; ++k) nb[k] = (int64_t)1 << (3 * k);
  double* W[ORC_MAX_LEVEL + 1] = {0};
  double* Wh[ORC_MAX_LEVEL + 1] = {0};
  double* g[ORC_MAX_LEVEL + 1] = {0};
  double* lc[ORC_MAX_LEVEL + 1] = {0};
  for (int k = 2; k <= kap; ++k) {
    size_t sz = sizeof(double) * (size_t)(nb[k] * R * lv[k].d);
    W[k] = (double*)calloc(1, sz ? sz : 8);
    Wh[k] = (double*)calloc(1, sz ? sz : 8);
    g[k] = (double*)calloc(1, sz ? sz : 8);
    lc[k] = (double*)calloc(1, sz ? sz : 8);
  }

  /* Step 1 (P2M): W_m^I = sum_{y_j in I} sigma_j K(x_m^{I_0}, y_j - c_I). */
  {
    const int d = lv[kap].d;
    const double lk = half_width(L, kap);
    int64_t b;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : viol)
    for (b = 0; b < nleaf; ++b) {
      double c[3];
      box_center(lo, L, kap, b, c);
      for (int64_t p = os[b]; p < os[b + 1]; ++p) {
        const int64_t j = ps[p];
        double z[3] = {src[3 * j] - c[0], src[3 * j + 1] - c[1], src[3 * j + 2] - c[2]};
        if (!in_J0(z, lk)) ++viol;
        for (int m = 0; m < d; ++m) {
          const double kv = kxy(kern, lv[kap].X + 3 * m, z);
          for (int r = 0; r < R; ++r)
            W[kap][(b * R + r) * d + m] += sigma[j + r * ld_sigma] * kv;
        }
      }
    }
  }

  /* Step 2 (M2M), with the 2^D precomputed operators of Section 4.1:
   * K_M2M^i = K^{I^k, J^{k+1}} Delta^{k+1}, K_{m,p} = K(x_m^{I_0^k} + c_P - c_C, y_p^{J_0^{k+1}}). */
  for (int k = kap - 1; k >= 2; --k) {
    const int dk = lv[k].d, dc = lv[k + 1].d;
    const double lc1 = half_width(L, k + 1);
    double* M = (double*)malloc(sizeof(double) * (size_t)(8 * dk * dc) + 8);
    for (int i = 0; i < 8; ++i) {
      const double sh[3] = {-((i & 1) ? 1.0 : -1.0) * lc1, -((i & 2) ? 1.0 : -1.0) * lc1,
                            -((i & 4) ? 1.0 : -1.0) * lc1}; /* c_P - c_C */
      for (int m = 0; m < dk; ++m) {
        double* row = M + ((int64_t)i * dk + m) * dc;
        const double xs[3] = {lv[k].X[3 * m] + sh[0], lv[k].X[3 * m + 1] + sh[1],
                              lv[k].X[3 * m + 2] + sh[2]};
        if (!in_I0(xs, lc1, L)) ++viol;
        for (int p = 0; p < dc; ++p) row[p] = kxy(kern, xs, lv[k + 1].Y + 3 * p);
        /* row <- (Delta^t row^t)^t, i.e. row * Delta */
        orc_apply_delta_t(dc, lv[k + 1].Gamma, lv[k + 1].B, row);
      }
    }
    int64_t P;
#pragma omp parallel for schedule(static)
    for (P = 0; P < nb[k]; ++P)
      for (int i = 0; i < 8; ++i) {
        const int64_t C = 8 * P + i;
        for (int r = 0; r < R; ++r)
          for (int m = 0; m < dk; ++m) {
            double s = 0.0;
            const double* row = M + ((int64_t)i * dk + m) * dc;
            for (int q2 = 0; q2 < dc; ++q2) s += row[q2] * W[k + 1][(C * R + r) * dc + q2];
            W[k][(P * R + r) * dk + m] += s;
          }
      }
    free(M);
  }

  /* Step 3: What^{I^k} = Delta^{I_0^k, J_0^k} W^{I^k}. */
  for (int k = 2; k <= kap; ++k) {
    const int d = lv[k].d;
    int64_t t;
#pragma omp parallel for schedule(static)
    for (t = 0; t < nb[k] * R; ++t) {
      memcpy(Wh[k] + t * d, W[k] + t * d, sizeof(double) * (size_t)d);
      orc_apply_delta(d, lv[k].Gamma, lv[k].B, Wh[k] + t * d);
    }
  }

  /* Step 4 (M2L): g^I = sum_{J in I(I)} K^delta What^J,
   * K^delta_{m'l} = K(x_{m'}^{J_0^k}, y_l^{J_0^k} + delta), delta = c_J - c_I. */
  for (int k = 2; k <= kap; ++k) {
    const int d = lv[k].d;
    const double lk = half_width(L, k);
    double* Kd = (double*)malloc(sizeof(double) * (size_t)(343 * d * d) + 8);
    viol += orc_m2l_operators(kern, L, k, d, lv[k].Y, Kd);
    const int r = lv[k].r;
    if (r > 0) {
      /* Section 4.2: K^delta ~ U C^delta U^t with C^delta = U^t K^delta U, so
       * g^I = U sum_J C^delta (U^t What^J). */
      const double* U = lv[k].U;
      double* Cd = (double*)malloc(sizeof(double) * (size_t)(343 * r * r) + 8);
      double* KU = (double*)malloc(sizeof(double) * (size_t)(d * r) + 8);
      for (int t = 0; t < 343; ++t) {
        const int dx = t % 7 - 3, dy = (t / 7) % 7 - 3, dz = t / 49 - 3;
        if (abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1) continue;
        const double* K = Kd + (int64_t)t * d * d;
        for (int mp = 0; mp < d; ++mp) /* K^delta U */
          for (int q = 0; q < r; ++q) {
            double s = 0.0;
            for (int l = 0; l < d; ++l) s += K[(int64_t)mp * d + l] * U[(int64_t)l * r + q];
            KU[(int64_t)mp * r + q] = s;
          }
        for (int qp = 0; qp < r; ++qp) /* U^t (K^delta U) */
          for (int q = 0; q < r; ++q) {
            double s = 0.0;
            for (int mp = 0; mp < d; ++mp) s += U[(int64_t)mp * r + qp] * KU[(int64_t)mp * r + q];
            Cd[((int64_t)t * r + qp) * r + q] = s;
          }
      }
      double* wt = (double*)malloc(sizeof(double) * (size_t)(nb[k] * R * r) + 8);
      int64_t J;
#pragma omp parallel for schedule(static)
      for (J = 0; J < nb[k] * R; ++J) /* w~ = U^t What */
        for (int q = 0; q < r; ++q) {
          double s = 0.0;
          for (int l = 0; l < d; ++l) s += U[(int64_t)l * r + q] * Wh[k][J * d + l];
          wt[J * r + q] = s;
        }
      int64_t I;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : m2l_pairs)
      for (I = 0; I < nb[k]; ++I) {
        int64_t lst[189], ci[3], cj[3];
        const int n = orc_interaction_list(k, I, lst);
        demorton3(I, k, ci);
        m2l_pairs += n;
        double gt[r];
        for (int rr = 0; rr < R; ++rr) {
          for (int qp = 0; qp < r; ++qp) gt[qp] = 0.0;
          for (int e = 0; e < n; ++e) {
            const int64_t Jb = lst[e];
            demorton3(Jb, k, cj);
            const int t = (int)((cj[0] - ci[0] + 3) + 7 * (cj[1] - ci[1] + 3) + 49 * (cj[2] - ci[2] + 3));
            for (int qp = 0; qp < r; ++qp) {
              double s = 0.0;
              const double* row = Cd + ((int64_t)t * r + qp) * r;
              for (int q = 0; q < r; ++q) s += row[q] * wt[(Jb * R + rr) * r + q];
              gt[qp] += s;
            }
          }
          for (int mp = 0; mp < d; ++mp) { /* g = U g~ */
            double s = 0.0;
            for (int qp = 0; qp < r; ++qp) s += U[(int64_t)mp * r + qp] * gt[qp];
            g[k][(I * R + rr) * d + mp] += s;
          }
        }
      }
      free(wt);
      free(KU);
      free(Cd);
      free(Kd);
      continue;
    }
    int64_t I;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : m2l_pairs)
    for (I = 0; I < nb[k]; ++I) {
      int64_t lst[189], ci[3], cj[3];
      const int n = orc_interaction_list(k, I, lst);
      demorton3(I, k, ci);
      m2l_pairs += n;
      for (int e = 0; e < n; ++e) {
        const int64_t J = lst[e];
        demorton3(J, k, cj);
        const int t = (int)((cj[0] - ci[0] + 3) + 7 * (cj[1] - ci[1] + 3) + 49 * (cj[2] - ci[2] + 3));
        for (int r = 0; r < R; ++r)
          for (int mp = 0; mp < d; ++mp) {
            double s = 0.0;
            const double* row = Kd + ((int64_t)t * d + mp) * d;
            for (int l = 0; l < d; ++l) s += row[l] * Wh[k][(J * R + r) * d + l];
            g[k][(I * R + r) * d + mp] += s;
          }
      }
    }
    free(Kd);
  }

  /* Step 5 (L2L): l^{I^2} = g^{I^2};
   * l^{I^k} = g^{I^k} + K_L2L^i l^{P(I^k)}, K_L2L = K' (Delta^{k-1})^t,
   * K'_{m'p'} = K(x_{m'}^{J_0^k} + c_I - c_P, y_{p'}^{I_0^{k-1}}). */
  memcpy(lc[2], g[2], sizeof(double) * (size_t)(nb[2] * R * lv[2].d));
  for (int k = 3; k <= kap; ++k) {
    const int dk = lv[k].d, dp = lv[k - 1].d;
    const double lk = half_width(L, k), lpar = half_width(L, k - 1);
    double* M = (double*)malloc(sizeof(double) * (size_t)(8 * dk * dp) + 8);
    for (int i = 0; i < 8; ++i) {
      const double sh[3] = {((i & 1) ? 1.0 : -1.0) * lk, ((i & 2) ? 1.0 : -1.0) * lk,
                            ((i & 4) ? 1.0 : -1.0) * lk}; /* c_I - c_P */
      for (int mp = 0; mp < dk; ++mp) {
        double* row = M + ((int64_t)i * dk + mp) * dp;
        const double xs[3] = {lv[k].Y[3 * mp] + sh[0], lv[k].Y[3 * mp + 1] + sh[1],
                              lv[k].Y[3 * mp + 2] + sh[2]};
        if (!in_J0(xs, lpar)) ++viol;
        for (int pp = 0; pp < dp; ++pp) row[pp] = kxy(kern, xs, lv[k - 1].X + 3 * pp);
        /* row <- (Delta row^t)^t, i.e. row * Delta^t */
        orc_apply_delta(dp, lv[k - 1].Gamma, lv[k - 1].B, row);
      }
    }
    int64_t I;
#pragma omp parallel for schedule(static)
    for (I = 0; I < nb[k]; ++I) {
      const int i = (int)(I & 7);
      const int64_t P = I >> 3;
      for (int r = 0; r < R; ++r)
        for (int mp = 0; mp < dk; ++mp) {
          double s = 0.0;
          const double* row = M + ((int64_t)i * dk + mp) * dp;
          for (int q2 = 0; q2 < dp; ++q2) s += row[q2] * lc[k - 1][(P * R + r) * dp + q2];
          lc[k][(I * R + r) * dk + mp] = g[k][(I * R + r) * dk + mp] + s;
        }
    }
    free(M);
  }

  /* Step 6: lhat^{I^kappa} = Delta^{J_0, I_0} l = (Delta^{I_0, J_0})^t l. */
  const int dl_ = lv[kap].d;
  double* lh = (double*)malloc(sizeof(double) * (size_t)(nleaf * R * dl_) + 8);
  {
    int64_t t;
#pragma omp parallel for schedule(static)
    for (t = 0; t < nleaf * R; ++t) {
      memcpy(lh + t * dl_, lc[kap] + t * dl_, sizeof(double) * (size_t)dl_);
      orc_apply_delta_t(dl_, lv[kap].Gamma, lv[kap].B, lh + t * dl_);
    }
  }

  /* Step 7 (L2P): f_F(x_i) = sum_{l'} K(x_i - c_I, y_{l'}^{I_0}) lhat_{l'}, and
   * the near field f_N(x_i) = sum_{y_j in N(I)} sigma_j K(x_i, y_j). */
  double* ffar = (double*)calloc((size_t)(nt * R + 1), sizeof(double));
  double* fnear = (double*)calloc((size_t)(nt * R + 1), sizeof(double));
  {
    const double lk = half_width(L, kap);
    int64_t b;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : viol, p2p_pairs)
    for (b = 0; b < nleaf; ++b) {
      if (ot[b] == ot[b + 1]) continue;
      double c[3];
      int64_t nbr[27];
      box_center(lo, L, kap, b, c);
      const int nn = orc_neighbours(kap, b, nbr);
      for (int64_t p = ot[b]; p < ot[b + 1]; ++p) {
        const int64_t i = pt[p];
        const double z[3] = {tgt[3 * i] - c[0], tgt[3 * i + 1] - c[1], tgt[3 * i + 2] - c[2]};
        if (!in_J0(z, lk)) ++viol;
        for (int r = 0; r < R; ++r) {
          double s = 0.0;
          for (int lp = 0; lp < dl_; ++lp)
            s += kxy(kern, z, lv[kap].X + 3 * lp) * lh[(b * R + r) * dl_ + lp];
          ffar[i + r * nt] = s;
        }
        for (int e = 0; e < nn; ++e) {
          const int64_t J = nbr[e];
          for (int64_t q2 = os[J]; q2 < os[J + 1]; ++q2) {
            const int64_t j = ps[q2];
            if (exclude_self && j == i) continue;
            ++p2p_pairs;
            const double kv = kxy(kern, tgt + 3 * i, src + 3 * j);
            for (int r = 0; r < R; ++r) fnear[i + r * nt] += sigma[j + r * ld_sigma] * kv;
          }
        }
      }
    }
  }
  for (int64_t i = 0; i < nt; ++i)
    for (int r = 0; r < R; ++r) f[i + r * ld_f] = ffar[i + r * nt] + fnear[i + r * nt];

  if (dump) {
    for (int k = 2; k <= kap; ++k) {
      const size_t sz = sizeof(double) * (size_t)(nb[k] * R * lv[k].d);
      if (dump->W[k]) memcpy(dump->W[k], W[k], sz);
      if (dump->What[k]) memcpy(dump->What[k], Wh[k], sz);
      if (dump->g[k]) memcpy(dump->g[k], g[k], sz);
      if (dump->l[k]) memcpy(dump->l[k], lc[k], sz);
    }
    if (dump->lhat) memcpy(dump->lhat, lh, sizeof(double) * (size_t)(nleaf * R * dl_));
    if (dump->f_far) memcpy(dump->f_far, ffar, sizeof(double) * (size_t)(nt * R));
    if (dump->f_near) memcpy(dump->f_near, fnear, sizeof(double) * (size_t)(nt * R));
    dump->domain_violations = viol;
    dump->m2l_pairs = m2l_pairs;
    dump->p2p_pairs = p2p_pairs;
  }

  for (int k = 2; k <= kap; ++k) {
    free(W[k]);
    free(Wh[k]);
    free(g[k]);
    free(lc[k]);
  }
  free(lh);
  free(ffar);
  free(fnear);
  free(kt);
  free(ks);
  free(pt);
  free(ps);
  free(ot);
  free(os);
  return 0;
}
