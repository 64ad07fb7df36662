// ops.cu -- operator assembly on the GPU in FP64 (Section 4.1 and 4.2).
//
//  K_M2M^i (level k, child octant i) = K^{I^k, J^{k+1}} Delta^{k+1} with
//    K^{I^k,J^{k+1}}_{m,p} = K(x_m^{I_0^k} + c_P - c_C, y_p^{J_0^{k+1}});
//    each row r is replaced by r Delta = (Delta^t r^t)^t through the two
//    triangular solves B z = r^t, Gamma^t w = z (never an explicit inverse).
//  K_L2L^i (level k) = K' (Delta^{k-1})^t with
//    K'_{m',p'} = K(x_{m'}^{J_0^k} + c_I - c_P, y_{p'}^{I_0^{k-1}});
//    each row by Gamma z = r^t, B^t w = z.
//  K^delta_{m'l} = K(x_{m'}^{J_0^k}, y_l^{J_0^k} + delta) for the 316 offsets
//    delta = (c_J - c_I) of an interaction list.
// For an even kernel the (J_0, I_0) EIM is the transpose of the (I_0, J_0)
// one: x^{J_0} = y^{J_0} (= Y), y^{I_0} = x^{I_0} (= X), Delta^{J_0 I_0} =
// (Delta^{I_0 J_0})^t.
#include <vector>

#include "internal.h"

namespace eifmm {
namespace {

// v <- Delta^t v = Gamma^-t B^-1 v (row-major packed d x d).
__device__ void dev_delta_t(int d, const double* G, const double* B, double* v) {
  for (int i = 0; i < d; ++i) {
    double s = v[i];
    for (int m = 0; m < i; ++m) s -= B[i * d + m] * v[m];
    v[i] = s;
  }
  for (int i = d - 1; i >= 0; --i) {
    double s = v[i];
    for (int m = i + 1; m < d; ++m) s -= G[m * d + i] * v[m];
    v[i] = s / G[i * d + i];
  }
}

// v <- Delta v = B^-t Gamma^-1 v.
__device__ void dev_delta(int d, const double* G, const double* B, double* v) {
  for (int i = 0; i < d; ++i) {
    double s = v[i];
    for (int m = 0; m < i; ++m) s -= G[i * d + m] * v[m];
    v[i] = s / G[i * d + i];
  }
  for (int i = d - 1; i >= 0; --i) {
    double s = v[i];
    for (int m = i + 1; m < d; ++m) s -= B[m * d + i] * v[m];
    v[i] = s;
  }
}

// One thread per (octant i, row m); the row lives in `scratch`.
__global__ void k_build_m2m(int kern, int dk, int dc, double lc1,
                            const double* __restrict__ Xk,
                            const double* __restrict__ Yc,
                            const double* __restrict__ Gc,
                            const double* __restrict__ Bc,
                            double* __restrict__ scratch,
                            double* __restrict__ m2mT, double* __restrict__ m2m_rm) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 8 * dk) return;
  const int i = t / dk, m = t - i * dk;
  double* row = scratch + (int64_t)t * dc;
  // c_P - c_C = -(s_i) l_{k+1}
  const double sh0 = (i & 1) ? -lc1 : lc1, sh1 = (i & 2) ? -lc1 : lc1, sh2 = (i & 4) ? -lc1 : lc1;
  const double x0 = Xk[3 * m] + sh0, x1 = Xk[3 * m + 1] + sh1, x2 = Xk[3 * m + 2] + sh2;
  for (int p = 0; p < dc; ++p)
    row[p] = kern_f64_ieee(kern, x0 - Yc[3 * p], x1 - Yc[3 * p + 1], x2 - Yc[3 * p + 2]);
  dev_delta_t(dc, Gc, Bc, row);
  for (int q = 0; q < dc; ++q) m2mT[((int64_t)i * dc + q) * dk + m] = row[q];
  for (int q = 0; q < dc; ++q) m2m_rm[((int64_t)i * dk + m) * dc + q] = row[q];
}

__global__ void k_build_l2l(int kern, int dk, int dp, double lk,
                            const double* __restrict__ Yk,
                            const double* __restrict__ Xp,
                            const double* __restrict__ Gp,
                            const double* __restrict__ Bp,
                            double* __restrict__ scratch,
                            double* __restrict__ l2lT, double* __restrict__ l2l_rm) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 8 * dk) return;
  const int i = t / dk, m = t - i * dk;
  double* row = scratch + (int64_t)t * dp;
  // c_I - c_P = s_i l_k
  const double sh0 = (i & 1) ? lk : -lk, sh1 = (i & 2) ? lk : -lk, sh2 = (i & 4) ? lk : -lk;
  const double x0 = Yk[3 * m] + sh0, x1 = Yk[3 * m + 1] + sh1, x2 = Yk[3 * m + 2] + sh2;
  for (int p = 0; p < dp; ++p)
    row[p] = kern_f64_ieee(kern, x0 - Xp[3 * p], x1 - Xp[3 * p + 1], x2 - Xp[3 * p + 2]);
  dev_delta(dp, Gp, Bp, row);
  for (int q = 0; q < dp; ++q) l2lT[((int64_t)i * dp + q) * dk + m] = row[q];
  for (int q = 0; q < dp; ++q) l2l_rm[((int64_t)i * dk + m) * dp + q] = row[q];
}

// kdT[slot][l][m'] = K(Y_{m'}, Y_l + delta_slot)
__global__ void k_build_kd(int kern, int d, double lk, const double* __restrict__ Y,
                           double* __restrict__ kdT) {
  const int slot = blockIdx.y;
  const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
  const bool near = abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1;
  const double d0 = 2.0 * dx * lk, d1 = 2.0 * dy * lk, d2 = 2.0 * dz * lk;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d * d; t += gridDim.x * blockDim.x) {
    const int l = t / d, mp = t - l * d;
    double v = 0.0;
    if (!near)
      v = kern_f64_ieee(kern, Y[3 * mp] - (Y[3 * l] + d0), Y[3 * mp + 1] - (Y[3 * l + 1] + d1),
                        Y[3 * mp + 2] - (Y[3 * l + 2] + d2));
    kdT[((int64_t)slot * d + l) * d + mp] = v;
  }
}

// packed triangles: colp[k*d - k(k-1)/2 + (j-k)] = M[j][k] (j >= k),
// rowp[k(k+1)/2 + j] = M[k][j] (j <= k).
__global__ void k_pack_tri(const double* __restrict__ M, int d, double* __restrict__ colp,
                           double* __restrict__ rowp) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d * d) return;
  const int i = t / d, j = t - i * d;  // M[i][j]
  if (j <= i) {
    colp[(int64_t)j * d - (int64_t)j * (j - 1) / 2 + (i - j)] = M[t];
    rowp[(int64_t)i * (i + 1) / 2 + j] = M[t];
  }
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__global__ void k_transpose(const double* __restrict__ a, double* __restrict__ b, int d) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d * d) return;
  const int i = t / d, j = t - i * d;
  b[j * d + i] = a[t];
}

eifmm_status to_f32(const double* a, float** b, int64_t n, cudaStream_t s) {
  EIFMM_TRY(dalloc(b, n > 0 ? n : 1));
  if (n > 0) {
    k_to_f32<<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(a, *b, n);
    EIFMM_CHECK_LAUNCH();
  }
  return EIFMM_OK;
}

}  // namespace

eifmm_status assemble_ops(Ops* ops, cudaStream_t s) {
  const int depth = ops->depth;
  const int kern = (int)ops->kern;
  // column-major copies of Gamma and B
  for (int k = 2; k <= depth; ++k) {
    LevelOps& v = ops->lv[k];
    const int d = v.d;
    EIFMM_TRY(dalloc(&v.G_cm, (size_t)d * d));
    EIFMM_TRY(dalloc(&v.B_cm, (size_t)d * d));
    k_transpose<<<(d * d + 255) / 256, 256, 0, s>>>(v.G_rm, v.G_cm, d);
    EIFMM_CHECK_LAUNCH();
    k_transpose<<<(d * d + 255) / 256, 256, 0, s>>>(v.B_rm, v.B_cm, d);
    EIFMM_CHECK_LAUNCH();
  }
  double* scratch = nullptr;
  EIFMM_TRY(dalloc(&scratch, (size_t)8 * kMaxD * kMaxD));
  for (int k = 2; k <= depth; ++k) {
    LevelOps& v = ops->lv[k];
    const double lk = ops->L * ldexp(1.0, -(k + 1));
    if (k < depth) {
      const LevelOps& c = ops->lv[k + 1];
      EIFMM_TRY(dalloc(&v.m2mT, (size_t)8 * v.d * c.d));
      EIFMM_TRY(dalloc(&v.m2m, (size_t)8 * v.d * c.d));
      k_build_m2m<<<(8 * v.d + 63) / 64, 64, 0, s>>>(kern, v.d, c.d, ops->L * ldexp(1.0, -(k + 2)),
                                                     v.X, c.Y, c.G_rm, c.B_rm, scratch, v.m2mT, v.m2m);
      EIFMM_CHECK_LAUNCH();
      EIFMM_TRY(to_f32(v.m2mT, &v.m2mT32, (int64_t)8 * v.d * c.d, s));
      EIFMM_TRY(to_f32(v.m2m, &v.m2m32, (int64_t)8 * v.d * c.d, s));
    }
    if (k > 2) {
      const LevelOps& p = ops->lv[k - 1];
      EIFMM_TRY(dalloc(&v.l2lT, (size_t)8 * v.d * p.d));
      EIFMM_TRY(dalloc(&v.l2l, (size_t)8 * v.d * p.d));
      k_build_l2l<<<(8 * v.d + 63) / 64, 64, 0, s>>>(kern, v.d, p.d, lk, v.Y, p.X, p.G_rm, p.B_rm,
                                                     scratch, v.l2lT, v.l2l);
      EIFMM_CHECK_LAUNCH();
      EIFMM_TRY(to_f32(v.l2lT, &v.l2lT32, (int64_t)8 * v.d * p.d, s));
      EIFMM_TRY(to_f32(v.l2l, &v.l2l32, (int64_t)8 * v.d * p.d, s));
    }
    EIFMM_TRY(dalloc(&v.kdT, (size_t)kNumSlots * v.d * v.d));
    k_build_kd<<<dim3((v.d * v.d + 255) / 256 < 64 ? (v.d * v.d + 255) / 256 : 64, kNumSlots), 256, 0, s>>>(
        kern, v.d, lk, v.Y, v.kdT);
    EIFMM_CHECK_LAUNCH();
    EIFMM_TRY(to_f32(v.G_cm, &v.G32_cm, (int64_t)v.d * v.d, s));
    EIFMM_TRY(to_f32(v.G_rm, &v.G32_rm, (int64_t)v.d * v.d, s));
    EIFMM_TRY(to_f32(v.B_cm, &v.B32_cm, (int64_t)v.d * v.d, s));
    EIFMM_TRY(to_f32(v.B_rm, &v.B32_rm, (int64_t)v.d * v.d, s));
    EIFMM_TRY(to_f32(v.X, &v.X32, (int64_t)3 * v.d, s));
    const int64_t np = (int64_t)v.d * (v.d + 1) / 2;
    EIFMM_TRY(dalloc(&v.G_colp, np));
    EIFMM_TRY(dalloc(&v.G_rowp, np));
    EIFMM_TRY(dalloc(&v.B_colp, np));
    EIFMM_TRY(dalloc(&v.B_rowp, np));
    k_pack_tri<<<(v.d * v.d + 255) / 256, 256, 0, s>>>(v.G_rm, v.d, v.G_colp, v.G_rowp);
    EIFMM_CHECK_LAUNCH();
    k_pack_tri<<<(v.d * v.d + 255) / 256, 256, 0, s>>>(v.B_rm, v.d, v.B_colp, v.B_rowp);
    EIFMM_CHECK_LAUNCH();
    EIFMM_TRY(to_f32(v.G_colp, &v.G32_colp, np, s));
    EIFMM_TRY(to_f32(v.G_rowp, &v.G32_rowp, np, s));
    EIFMM_TRY(to_f32(v.B_colp, &v.B32_colp, np, s));
    EIFMM_TRY(to_f32(v.B_rowp, &v.B32_rowp, np, s));
  }
  // slot lists of the 8 parity classes: offsets o in {-2..3} for an even
  // coordinate and {-3..2} for an odd one, minus the 27 neighbours.
  std::vector<int> lists(8 * kListLen);
  for (int c = 0; c < 8; ++c) {
    int n = 0;
    const int b0 = c & 1, b1 = (c >> 1) & 1, b2 = (c >> 2) & 1;
    for (int dz = -2 - b2; dz <= 3 - b2; ++dz)
      for (int dy = -2 - b1; dy <= 3 - b1; ++dy)
        for (int dx = -2 - b0; dx <= 3 - b0; ++dx) {
          if (abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1) continue;
          lists[c * kListLen + n++] = (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3);
        }
  }
  EIFMM_TRY(dalloc(&ops->d_slot_lists, lists.size()));
  EIFMM_CUDA(cudaMemcpyAsync(ops->d_slot_lists, lists.data(), lists.size() * sizeof(int),
                             cudaMemcpyHostToDevice, s));
  EIFMM_CUDA(cudaStreamSynchronize(s));
  dfree(scratch);
  return EIFMM_OK;
}

void free_ops(Ops* ops) {
  for (int k = 0; k <= kMaxLevel; ++k) {
    LevelOps& v = ops->lv[k];
    dfree(v.X); dfree(v.Y); dfree(v.G_rm); dfree(v.G_cm); dfree(v.B_rm); dfree(v.B_cm);
    dfree(v.m2mT); dfree(v.l2lT); dfree(v.kdT); dfree(v.m2mT32); dfree(v.l2lT32);
    dfree(v.m2m); dfree(v.l2l); dfree(v.m2m32); dfree(v.l2l32);
    dfree(v.G_colp); dfree(v.G_rowp); dfree(v.B_colp); dfree(v.B_rowp);
    dfree(v.G32_colp); dfree(v.G32_rowp); dfree(v.B32_colp); dfree(v.B32_rowp);
    dfree(v.G32_cm); dfree(v.G32_rm); dfree(v.B32_cm); dfree(v.B32_rm); dfree(v.X32);
    dfree(v.kd_img);
    v = LevelOps();
  }
  dfree(ops->d_slot_lists);
  ops->d_slot_lists = nullptr;
}

}  // namespace eifmm
