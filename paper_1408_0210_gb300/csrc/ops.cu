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
#include "solve.cuh"

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

// Per-slot transpose of a [slot][d][d] stack: out[s][j][i] = in[s][i][j].
__global__ void k_transpose_slots(const double* __restrict__ in, int d, double* __restrict__ out) {
  const int64_t slot = blockIdx.y;
  const double* a = in + slot * d * d;
  double* b = out + slot * d * d;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d * d; t += gridDim.x * blockDim.x) {
    const int i = t / d, j = t - i * d;
    b[(int64_t)j * d + i] = a[t];
  }
}

// Tiles of one lower-triangular solve operator L' (layout in solve.cuh):
// L'[a][b] = M[p][q] with (p, q) = (a, b), or (dpad-1-a, dpad-1-b) when
// `rev`; `transpose` reads M[q][p].  Entries beyond d are those of the
// identity.  Entries on and above the diagonal are stored as zeros: the
// diagonal is held by the pivots (or is one), and the zeros let the solve
// update every row of a diagonal tile with one vector load per four rows.
__global__ void k_build_delta_tiles(const double* __restrict__ M, int d, int nb, int transpose, int rev,
                                    double* __restrict__ t64, float* __restrict__ t32,
                                    double* __restrict__ piv64, float* __restrict__ piv32) {
  const int dpad = nb * 32;
  const int64_t n = (int64_t)nb * (nb + 1) / 2 * 1024;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int tile = (int)(e >> 10), J = 0;
    while (tile > J) { tile -= J + 1; ++J; }
    const int K = tile, k = (int)((e >> 5) & 31), i = (int)(e & 31);
    const int a = J * 32 + i, b = K * 32 + k;
    double v = 0.0;
    if (b < a) {
      const int p = rev ? dpad - 1 - a : a, q = rev ? dpad - 1 - b : b;
      if (p < d && q < d) v = transpose ? M[(int64_t)q * d + p] : M[(int64_t)p * d + q];
      else v = p == q ? 1.0 : 0.0;
    }
    t64[e] = v;
    t32[e] = (float)v;
  }
  if (piv64 != nullptr)
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < dpad; a += gridDim.x * blockDim.x) {
      const int p = rev ? dpad - 1 - a : a;
      const double g = p < d ? M[(int64_t)p * d + p] : 1.0;
      piv64[a] = g;
      piv32[a] = (float)(1.0 / g);
    }
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
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
    EIFMM_TRY(to_f32(v.X, &v.X32, (int64_t)3 * v.d, s));
    // Delta: Gamma then B^t; Delta^t: B then Gamma^t (reversed order)
    const int nb = (v.d + 31) / 32;
    const int64_t nt = delta_tiles_elems(v.d);
    const double* src[4] = {v.G_rm, v.B_rm, v.B_rm, v.G_rm};
    const int trans[4] = {0, 1, 0, 1}, rev[4] = {0, 1, 0, 1}, piv[4] = {0, -1, -1, 1};
    for (int o = 0; o < 4; ++o) {
      EIFMM_TRY(dalloc(&v.dt64[o], nt));
      EIFMM_TRY(dalloc(&v.dt32[o], nt));
      if (piv[o] >= 0) {
        EIFMM_TRY(dalloc(&v.piv64[piv[o]], nb * 32));
        EIFMM_TRY(dalloc(&v.piv32[piv[o]], nb * 32));
      }
      k_build_delta_tiles<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(
          src[o], v.d, nb, trans[o], rev[o], v.dt64[o], v.dt32[o], piv[o] >= 0 ? v.piv64[piv[o]] : nullptr,
          piv[o] >= 0 ? v.piv32[piv[o]] : nullptr);
      EIFMM_CHECK_LAUNCH();
    }
    // The M2L operator applied to W: K^delta Delta (Steps 3 and 4 together,
    // g = sum_J K^delta (Delta W^J)).  Row m' of K^delta Delta is Delta^t
    // applied to row m' of K^delta, so the product comes from the FP64
    // triangular solves, never from an explicit inverse.  kdT is
    // overwritten with it, same layout.
    {
      double* rows = nullptr;
      EIFMM_TRY(dalloc(&rows, (size_t)kNumSlots * v.d * v.d));
      const dim3 tg((v.d * v.d + 255) / 256 < 64 ? (v.d * v.d + 255) / 256 : 64, kNumSlots);
      k_transpose_slots<<<tg, 256, 0, s>>>(v.kdT, v.d, rows);  // rows[slot][m'][l] = K^delta_{m'l}
      EIFMM_CHECK_LAUNCH();
      DeltaBatch b;
      b.nlev = 1;
      b.lv[0] = delta_level(v.d, delta_ops64(v), true, rows, v.d, rows, v.d, nullptr,
                            (int64_t)kNumSlots * v.d);
      eifmm_status rc = launch_delta_batch<double, double, double, 0>(b, true, s);
      if (rc == EIFMM_OK) {
        k_transpose_slots<<<tg, 256, 0, s>>>(rows, v.d, v.kdT);
        if (cudaGetLastError() != cudaSuccess) rc = EIFMM_ECUDA;
      }
      EIFMM_CUDA(cudaStreamSynchronize(s));
      dfree(rows);
      if (rc != EIFMM_OK) return rc;
    }
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
  EIFMM_TRY(build_xfer_blas(ops, s));
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
    dfree(v.X); dfree(v.Y); dfree(v.G_rm); dfree(v.B_rm);
    dfree(v.m2mT); dfree(v.l2lT); dfree(v.kdT); dfree(v.m2mT32); dfree(v.l2lT32);
    dfree(v.m2m); dfree(v.l2l); dfree(v.m2m32); dfree(v.l2l32); dfree(v.m2m_cb); dfree(v.l2l_cb);
    for (int o = 0; o < 4; ++o) { dfree(v.dt64[o]); dfree(v.dt32[o]); }
    for (int o = 0; o < 2; ++o) { dfree(v.piv64[o]); dfree(v.piv32[o]); }
    dfree(v.X32);
    dfree(v.kd_img);
    dfree(v.kscale);
    dfree(v.U);
    dfree(v.Ct);
    dfree(v.kd32);
    v = LevelOps();
  }
  dfree(ops->d_slot_lists);
  ops->d_slot_lists = nullptr;
}

}  // namespace eifmm
