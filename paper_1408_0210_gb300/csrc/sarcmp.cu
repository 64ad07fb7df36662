// sarcmp.cu -- the first stage of the M2L compression of Section 4.2 for
// the FP64 far field (the FP64 path and tiers 3 and 4 of the mixed path).
//
// K_fat = [K^delta_1 ... K^delta_316] (d x 316 d, the far offsets of a
// level).  Its leading left singular vectors U (d x r) come from the
// eigenvectors of the Gram matrix K_fat K_fat^t = sum_delta K^delta
// K^delta^t (FP64 on the GPU; cyclic Jacobi on the host), its singular values
// from the square roots of the eigenvalues, and r from the two filters of
// Section 4.2: the values s_j / s_0 above eps, and the shortest leading run
// whose sum reaches (1 - eps) of the total; r keeps both.  The kernels here
// are even, so K^{-delta} = (K^delta)^t and U also spans the row space.
// Then
//   C^delta = U^t K^delta U                       (r x r per offset)
// and step 4 runs as
//   w~ = U^t What,  g~ = sum_J C^delta w~^J,  g = U g~,
// with What = Delta W by the FP64 triangular solves (the unfolded K^delta:
// folding Delta into the operator, as the uncompressed path does, makes it
// incompressible).  A rotation of the basis among directions of nearly
// equal singular values -- what the squared singular values of the Gram
// matrix cannot resolve below about 1e-8 s_0 -- changes C^delta and w~ but
// not their product beyond the size of those values, which the truncation
// drops anyway.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "internal.h"
#include "solve.cuh"

namespace eifmm {
namespace {

// K^delta of level k unfolded: kd[slot][l][m'] = K(Y_m', Y_l + delta), zero
// for the 27 near offsets (as k_build_kd in ops.cu, recomputed here).
__global__ void k_kd_plain(int kern, int d, double lk, const double* __restrict__ Y, double* __restrict__ kd) {
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
    kd[((int64_t)slot * d + l) * d + mp] = v;
  }
}

// G[a][b] = sum over slots and l of K^delta_{a l} K^delta_{b l}; one block
// per row a, threads over b.
__global__ void k_gram(const double* __restrict__ kd, int d, double* __restrict__ G) {
  const int a = blockIdx.x;
  for (int b = threadIdx.x; b < d; b += blockDim.x) {
    double s = 0.0;
    for (int slot = 0; slot < kNumSlots; ++slot) {
      const double* K = kd + (int64_t)slot * d * d;
      for (int l = 0; l < d; ++l) s += K[(int64_t)l * d + a] * K[(int64_t)l * d + b];
    }
    G[(int64_t)a * d + b] = s;
  }
}

// T[slot][a][j] = sum_l K^delta_{a l} U[l][j]   (U row-major d x r)
__global__ void k_kd_u(const double* __restrict__ kd, const double* __restrict__ U, int d, int r,
                       double* __restrict__ T) {
  const int slot = blockIdx.y;
  const double* K = kd + (int64_t)slot * d * d;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d * r; t += gridDim.x * blockDim.x) {
    const int a = t / r, j = t - a * r;
    double s = 0.0;
    for (int l = 0; l < d; ++l) s += K[(int64_t)l * d + a] * U[(int64_t)l * r + j];
    T[((int64_t)slot * d + a) * r + j] = s;
  }
}

// Ct[slot][j][i] = C^delta_{ij} = sum_a U[a][i] T[slot][a][j]: the layout of
// the M2L kernels ([slot][l][m'] = operator_{m' l}) with d -> r.
__global__ void k_ut_t(const double* __restrict__ T, const double* __restrict__ U, int d, int r,
                       double* __restrict__ Ct) {
  const int slot = blockIdx.y;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < r * r; t += gridDim.x * blockDim.x) {
    const int j = t / r, i = t - j * r;
    double s = 0.0;
    for (int a = 0; a < d; ++a) s += U[(int64_t)a * r + i] * T[((int64_t)slot * d + a) * r + j];
    Ct[((int64_t)slot * r + j) * r + i] = s;
  }
}

// C[M x N] = A[M x K] B, B row-major K x N (TB = false) or B^t with B
// row-major N x K (TB = true); FP64, 64 x 64 tiles, 4 x 4 per thread.
template <bool TB>
__global__ void __launch_bounds__(256)
k_gemm64(int64_t M, int N, int K, const double* __restrict__ A, int lda, const double* __restrict__ B, int ldb,
         double* __restrict__ C, int ldc) {
  __shared__ double sA[16][64 + 1];
  __shared__ double sB[16][64 + 1];
  const int tid = threadIdx.x;
  const int ntn = (N + 63) / 64;
  const int64_t tm = blockIdx.x / ntn;
  const int tn = (int)(blockIdx.x % ntn);
  const int64_t m0 = tm * 64;
  const int n0 = tn * 64;
  const int ti = (tid >> 4) * 4, tj = (tid & 15) * 4;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = tid; e < 16 * 64; e += 256) {
      const int kk = e & 15, mm = e >> 4;  // A: 64 rows x 16 terms
      const int64_t gm = m0 + mm;
      sA[kk][mm] = (gm < M && k0 + kk < K) ? A[gm * lda + k0 + kk] : 0.0;
      if (TB) {  // B^t: rows n of B, terms k
        const int gn = n0 + mm;
        sB[kk][mm] = (gn < N && k0 + kk < K) ? B[(int64_t)gn * ldb + k0 + kk] : 0.0;
      } else {
        const int kb = e >> 6, nb = e & 63;
        sB[kb][nb] = (n0 + nb < N && k0 + kb < K) ? B[(int64_t)(k0 + kb) * ldb + n0 + nb] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[kk][ti + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[kk][tj + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ti + i;
    if (gm >= M) break;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (n0 + tj + j < N) C[gm * ldc + n0 + tj + j] = acc[i][j];
  }
}

eifmm_status gemm64(bool tb, int64_t M, int N, int K, const double* A, int lda, const double* B, int ldb,
                    double* C, int ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return EIFMM_OK;
  const int64_t blocks = ((M + 63) / 64) * ((N + 63) / 64);
  if (blocks > 2147483647LL) {
    set_error("compressed M2L: projection too large for one launch");
    return EIFMM_EUNSUPPORTED;
  }
  if (tb) k_gemm64<true><<<(unsigned)blocks, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
  else k_gemm64<false><<<(unsigned)blocks, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
  EIFMM_CHECK_LAUNCH();
  return EIFMM_OK;
}

// Eigen-decomposition of the symmetric d x d matrix a (row-major, destroyed)
// by cyclic Jacobi rotations (each rotation zeroes one off-diagonal entry;
// sweeps until the off-diagonal part is below 1e-15 of the whole).  Returns
// the eigenvalues in w and the eigenvectors as the columns of v (row-major).
void jacobi_eig(std::vector<double>& a, int d, std::vector<double>& w, std::vector<double>& v) {
  v.assign((size_t)d * d, 0.0);
  for (int i = 0; i < d; ++i) v[(size_t)i * d + i] = 1.0;
  auto A = [&](int i, int j) -> double& { return a[(size_t)i * d + j]; };
  double total = 0.0;
  for (double x : a) total += x * x;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < d; ++p)
      for (int q = p + 1; q < d; ++q) off += 2.0 * A(p, q) * A(p, q);
    if (off <= 1e-30 * total) break;
    for (int p = 0; p < d; ++p)
      for (int q = p + 1; q < d; ++q) {
        const double apq = A(p, q);
        if (apq == 0.0) continue;
        const double theta = (A(q, q) - A(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < d; ++k) {  // columns p, q
          const double akp = A(k, p), akq = A(k, q);
          A(k, p) = c * akp - s * akq;
          A(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < d; ++k) {  // rows p, q
          const double apk = A(p, k), aqk = A(q, k);
          A(p, k) = c * apk - s * aqk;
          A(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < d; ++k) {
          const double vkp = v[(size_t)k * d + p], vkq = v[(size_t)k * d + q];
          v[(size_t)k * d + p] = c * vkp - s * vkq;
          v[(size_t)k * d + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(d);
  for (int i = 0; i < d; ++i) w[i] = A(i, i);
}

}  // namespace

// The two filters of Section 4.2 on singular values s (descending): the
// count of s_j / s_0 > eps, and the shortest leading run whose sum reaches
// (1 - eps) of the total; r keeps both.
int sarcmp_rank(const std::vector<double>& s, double eps, int* r_i, int* r_ii) {
  const int n = (int)s.size();
  int a = 0;
  for (int j = 0; j < n; ++j)
    if (s[j] / s[0] > eps) ++a;
  double total = 0.0;
  for (double x : s) total += x;
  double c = 0.0;
  int b = n;
  for (int j = 0; j < n; ++j) {
    c += s[j];
    if (c >= (1.0 - eps) * total) {
      b = j + 1;
      break;
    }
  }
  if (r_i) *r_i = a;
  if (r_ii) *r_ii = b;
  return std::max(std::max(a, b), 1);
}

void free_compression(LevelOps& v) {
  dfree(v.U);
  dfree(v.Ct);
  v.U = nullptr;
  v.Ct = nullptr;
  v.r = 0;
}

eifmm_status compress_ops(Ops* ops, double eps, cudaStream_t s) {
  for (int k = 2; k <= ops->depth; ++k) free_compression(ops->lv[k]);
  ops->compressed = false;
  if (!(eps > 0.0)) return EIFMM_OK;
  for (int k = 2; k <= ops->depth; ++k) {
    LevelOps& v = ops->lv[k];
    const int d = v.d;
    const double lk = ops->L * std::ldexp(1.0, -(k + 1));
    double *kd = nullptr, *G = nullptr, *T = nullptr;
    eifmm_status rc = EIFMM_OK;
    do {
      if ((rc = dalloc(&kd, (size_t)kNumSlots * d * d)) != EIFMM_OK) break;
      if ((rc = dalloc(&G, (size_t)d * d)) != EIFMM_OK) break;
      k_kd_plain<<<dim3((d * d + 255) / 256 < 64 ? (d * d + 255) / 256 : 64, kNumSlots), 256, 0, s>>>(
          (int)ops->kern, d, lk, v.Y, kd);
      count_launch();
      k_gram<<<d, 128, 0, s>>>(kd, d, G);
      count_launch();
      std::vector<double> g((size_t)d * d), w, vec;
      if (cudaMemcpyAsync(g.data(), G, g.size() * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("eifmm_ops_compress: Gram matrix failed");
        rc = EIFMM_ECUDA;
        break;
      }
      jacobi_eig(g, d, w, vec);
      std::vector<int> order(d);
      std::iota(order.begin(), order.end(), 0);
      std::sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
      std::vector<double> sv(d);
      for (int j = 0; j < d; ++j) sv[j] = std::sqrt(std::max(w[order[j]], 0.0));
      if (!(sv[0] > 0.0)) {
        set_error("eifmm_ops_compress: zero M2L operators at level " + std::to_string(k));
        rc = EIFMM_EINVAL;
        break;
      }
      const int r = sarcmp_rank(sv, eps, &v.r_i, &v.r_ii);
      std::vector<double> u((size_t)d * r);
      for (int a = 0; a < d; ++a)
        for (int j = 0; j < r; ++j) u[(size_t)a * r + j] = vec[(size_t)a * d + order[j]];
      if ((rc = dalloc(&v.U, (size_t)d * r)) != EIFMM_OK) break;
      if (cudaMemcpyAsync(v.U, u.data(), u.size() * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        rc = EIFMM_ECUDA;
        set_error("eifmm_ops_compress: upload failed");
        break;
      }
      if ((rc = dalloc(&T, (size_t)kNumSlots * d * r)) != EIFMM_OK) break;
      if ((rc = dalloc(&v.Ct, (size_t)kNumSlots * r * r)) != EIFMM_OK) break;
      k_kd_u<<<dim3((d * r + 255) / 256 < 64 ? (d * r + 255) / 256 : 64, kNumSlots), 256, 0, s>>>(kd, v.U, d, r, T);
      count_launch();
      k_ut_t<<<dim3((r * r + 255) / 256 < 64 ? (r * r + 255) / 256 : 64, kNumSlots), 256, 0, s>>>(T, v.U, d, r, v.Ct);
      count_launch();
      if (cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("eifmm_ops_compress: operator build failed");
        rc = EIFMM_ECUDA;
        break;
      }
      v.r = r;
      v.s_kept = sv[r - 1] / sv[0];
      v.s_next = r < d ? sv[r] / sv[0] : 0.0;
    } while (false);
    dfree(kd);
    dfree(G);
    dfree(T);
    if (rc != EIFMM_OK) {
      for (int q = 2; q <= ops->depth; ++q) free_compression(ops->lv[q]);
      return rc;
    }
  }
  ops->compressed = true;
  ops->compress_eps = eps;
  return EIFMM_OK;
}

// Step 4 at level k with the compressed operators, on the FP64 arrays of
// the FP64 far field: What = Delta W into Wh[k], w~ = What U into tmp,
// g~ = sum C^delta w~ into Wh[k] (FP32-pair arithmetic or FP64, as the
// uncompressed M2L of the same path), g = g~ U^t.

eifmm_status m2l_compressed(Workspace& ws, const Ops* ops, int k, int R, bool pair, cudaStream_t s) {
  const LevelOps& v = ops->lv[k];
  const int d = v.d, r = v.r;
  const int64_t rows = ((int64_t)1 << (3 * k)) * R;
  DeltaBatch b;
  b.nlev = 1;
  b.lv[0] = delta_level(d, delta_ops64(v), false, ws.W[k], d, ws.Wh[k], d, nullptr, rows);
  EIFMM_TRY((launch_delta_batch<double, double, double, 0>(b, false, s)));
  double* wt = (double*)ws.tmp;  // rows x r
  EIFMM_TRY(gemm64(false, rows, r, d, ws.Wh[k], d, v.U, r, wt, r, s));
  if (pair)
    EIFMM_TRY(launch_m2l_df(k, r, R, v.Ct, ops->d_slot_lists, wt, ws.Wh[k], ws.part64, ws.part64_cap, ws.nsm, s));
  else
    EIFMM_TRY(launch_m2l64(k, r, R, v.Ct, ops->d_slot_lists, wt, ws.Wh[k], ws.part64, ws.part64_cap, ws.nsm, s));
  EIFMM_TRY(gemm64(true, rows, d, r, ws.Wh[k], r, v.U, r, ws.g[k], d, s));
  return EIFMM_OK;
}

}  // namespace eifmm
