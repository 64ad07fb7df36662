// transfer.cuh -- steps 2 (M2M) and 5 (L2L) of Algorithm 3 with the 2^D
// precomputed operators of Section 4.1, one warp per group of output rows:
// lanes split the reduction index, so even the coarse levels (64 boxes at
// level 2) expose thousands of independent warps.
#pragma once
#include "internal.h"

namespace eifmm {

constexpr int kXferRows = 4;  // output rows per warp

// W^P_m = sum_{i=0..7} sum_q (K_M2M^i)_{m q} W^{C_i}_q, C_i = 8P + i.
// M: [8][dk][dc] row-major; W rows have leading dimensions ldk / ldc; the
// rows m in [dk, ldk) are written as zeros.
template <typename T>
__global__ void __launch_bounds__(128)
k_m2m_warp(int dk, int dc, int ldk, int ldc, int R, const T* __restrict__ M,
           const T* __restrict__ Wc, T* __restrict__ Wp, int64_t nparent) {
  const int lane = threadIdx.x & 31;
  const int ngroups = (ldk + kXferRows - 1) / kXferRows;
  const int64_t gw = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  if (gw >= nparent * R * ngroups) return;
  const int64_t P = gw / ((int64_t)R * ngroups);
  const int rem = (int)(gw - P * R * ngroups);
  const int r = rem / ngroups, m0 = (rem % ngroups) * kXferRows;
  T acc[kXferRows];
#pragma unroll
  for (int j = 0; j < kXferRows; ++j) acc[j] = (T)0;
  for (int i = 0; i < 8; ++i) {
    const T* w = Wc + ((8 * P + i) * R + r) * ldc;
    const T* mrow = M + ((int64_t)i * dk + m0) * dc;
    for (int q = lane; q < dc; q += 32) {
      const T wq = w[q];
#pragma unroll
      for (int j = 0; j < kXferRows; ++j)
        if (m0 + j < dk) acc[j] += mrow[(int64_t)j * dc + q] * wq;
    }
  }
#pragma unroll
  for (int j = 0; j < kXferRows; ++j)
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
  if (lane < kXferRows && m0 + lane < ldk) {
    T v = (T)0;
#pragma unroll
    for (int j = 0; j < kXferRows; ++j)
      if (j == lane) v = acc[j];
    Wp[(P * R + r) * ldk + m0 + lane] = (m0 + lane < dk) ? v : (T)0;
  }
}

// l^I_{m'} = g^I_{m'} + sum_{q'} (K_L2L^i)_{m' q'} l^{P(I)}_{q'}, i = I mod 8.
template <typename T>
__global__ void __launch_bounds__(128)
k_l2l_warp(int dk, int dp, int ldk, int ldp, int R, const T* __restrict__ Lm,
           const T* __restrict__ lpar, const T* __restrict__ g, T* __restrict__ lout,
           int64_t nbox) {
  const int lane = threadIdx.x & 31;
  const int ngroups = (ldk + kXferRows - 1) / kXferRows;
  const int64_t gw = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  if (gw >= nbox * R * ngroups) return;
  const int64_t I = gw / ((int64_t)R * ngroups);
  const int rem = (int)(gw - I * R * ngroups);
  const int r = rem / ngroups, m0 = (rem % ngroups) * kXferRows;
  const int i = (int)(I & 7);
  const T* lp = lpar + ((I >> 3) * R + r) * ldp;
  const T* mrow = Lm + ((int64_t)i * dk + m0) * dp;
  T acc[kXferRows];
#pragma unroll
  for (int j = 0; j < kXferRows; ++j) acc[j] = (T)0;
  for (int q = lane; q < dp; q += 32) {
    const T v = lp[q];
#pragma unroll
    for (int j = 0; j < kXferRows; ++j)
      if (m0 + j < dk) acc[j] += mrow[(int64_t)j * dp + q] * v;
  }
#pragma unroll
  for (int j = 0; j < kXferRows; ++j)
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
  if (lane < kXferRows && m0 + lane < ldk) {
    T v = (T)0;
#pragma unroll
    for (int j = 0; j < kXferRows; ++j)
      if (j == lane) v = acc[j];
    const int64_t o2 = (I * R + r) * ldk + m0 + lane;
    lout[o2] = (m0 + lane < dk) ? g[o2] + v : (T)0;
  }
}

inline unsigned xfer_blocks(int64_t nout, int R, int ldk) {
  const int64_t warps = nout * R * ((ldk + kXferRows - 1) / kXferRows);
  return (unsigned)((warps + 3) / 4);
}

}  // namespace eifmm

namespace eifmm {

// ---------------------------------------------------------------------------
// The same two steps as tiled GEMMs for the FP32 path: over all parents at
// once, C = A B with A the precomputed operator (rows m) and B the columns of
// child (M2M) or parent (L2L) coefficient vectors.  Block tile 64 x 64, K
// step 16, 256 threads with 4 x 4 outputs each.
//   M2M: C[m][c] = sum_{i, q} (K_M2M^i)_{m q} W^{child i of P}_q, c = P R + r,
//        the reduction index k = i * dc + q runs over the 8 children.
//   L2L: C[m][c] = g[m][c] + sum_q (K_L2L^i)_{m q} l^P_q for the child i of
//        blockIdx.z, c = P R + r.
// Rows m in [d, ld) of every output column are written as zeros.
// ---------------------------------------------------------------------------
struct XferGemm {
  int mode;          // 0 = M2M (child blockIdx.z, partial sums in P8), 1 = L2L
  int dk, ldk;       // output rank and leading dimension
  int dc, ldc;       // input rank and leading dimension (child for M2M, parent for L2L)
  int R;
  int64_t ncol;      // parents * R
  const float* A;    // [8][dk][dc] row-major
  const float* B;    // input coefficient rows
  const float* G;    // L2L: g of the output level (same layout as C)
  float* C;          // output coefficient rows
  float* P8;         // M2M: [8][ncol][ldk] partial sums, one per child
};

// 64 x 64 output tile per CTA, 4 x 4 per thread, K in steps of 16 through a
// double-buffered shared tile: the global loads of step k+1 are issued into
// registers before the FMAs of step k.
static __global__ void __launch_bounds__(256) k_xfer_gemm(XferGemm a) {
  __shared__ __align__(16) float As[2][16][64 + 4];
  __shared__ __align__(16) float Bs[2][16][64 + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * 64;
  const int64_t c0 = (int64_t)blockIdx.y * 64;
  const int i_l2l = blockIdx.z;  // the child octant (both modes)
  const int K = a.dc;
  // this thread's four (k, row) load slots: k = tid & 15, rows (tid >> 4) + 16 j
  const int kk_ld = tid & 15;
  const float* arow[4];
  const float* brow[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int rr = (tid >> 4) + 16 * j;
    const int m = m0 + rr;
    arow[j] = m < a.dk ? a.A + ((int64_t)i_l2l * a.dk + m) * a.dc : nullptr;
    const int64_t c = c0 + rr;
    brow[j] = nullptr;
    if (c < a.ncol) {
      const int64_t P = c / a.R;
      const int r = (int)(c - P * a.R);
      brow[j] = a.mode == 0 ? a.B + ((8 * P + i_l2l) * a.R + r) * a.ldc : a.B + (P * a.R + r) * a.ldc;
    }
  }
  float ra[4], rb[4];
  auto gload = [&](int k0) {
    const int k = k0 + kk_ld;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      ra[j] = (arow[j] != nullptr && k < K) ? __ldg(arow[j] + k) : 0.f;
      rb[j] = (brow[j] != nullptr && k < K) ? __ldg(brow[j] + k) : 0.f;
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      As[buf][kk_ld][(tid >> 4) + 16 * j] = ra[j];
      Bs[buf][kk_ld][(tid >> 4) + 16 * j] = rb[j];
    }
  };
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
  gload(0);
  sstore(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const bool more = k0 + 16 < K;
    if (more) gload(k0 + 16);
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      // rows m along tx, columns c along ty: a thread's 4 outputs of one
      // column are 4 consecutive floats of one coefficient row in memory
      const float4 a4 = *reinterpret_cast<const float4*>(&As[buf][kk][tx * 4]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[buf][kk][ty * 4]);
      const float ar[4] = {a4.x, a4.y, a4.z, a4.w};
      const float br[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(ar[u], br[v], acc[u][v]);
    }
    if (more) sstore(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  // float4 stores: 16 lanes write 64 consecutive coefficients of one row
  const int mb = m0 + tx * 4;
  if (mb < a.ldk) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t c = c0 + ty * 4 + v;
      if (c >= a.ncol) continue;
      const int64_t P = c / a.R;
      const int r = (int)(c - P * a.R);
      const int64_t row = a.mode == 0 ? (P * a.R + r) : ((8 * P + i_l2l) * a.R + r);
      const int64_t o = row * a.ldk + mb;
      float4 val = make_float4(mb + 0 < a.dk ? acc[0][v] : 0.f, mb + 1 < a.dk ? acc[1][v] : 0.f,
                               mb + 2 < a.dk ? acc[2][v] : 0.f, mb + 3 < a.dk ? acc[3][v] : 0.f);
      if (a.mode == 0) {
        *reinterpret_cast<float4*>(a.P8 + (int64_t)i_l2l * a.ncol * a.ldk + o) = val;
      } else {
        const float4 g = *reinterpret_cast<const float4*>(a.G + o);
        val.x = mb + 0 < a.dk ? g.x + val.x : 0.f;
        val.y = mb + 1 < a.dk ? g.y + val.y : 0.f;
        val.z = mb + 2 < a.dk ? g.z + val.z : 0.f;
        val.w = mb + 3 < a.dk ? g.w + val.w : 0.f;
        *reinterpret_cast<float4*>(a.C + o) = val;
      }
    }
  }
}

// W = sum over the 8 children of the partial sums, in a fixed order.
static __global__ void k_sum8(const float4* __restrict__ p8, int64_t n4, float4* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    float4 v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = p8[c * n4 + i];
#pragma unroll
    for (int w = 1; w < 8; w <<= 1)
#pragma unroll
      for (int c = 0; c < 8; c += 2 * w) {
        v[c].x += v[c + w].x;
        v[c].y += v[c + w].y;
        v[c].z += v[c + w].z;
        v[c].w += v[c + w].w;
      }
    out[i] = v[0];
  }
}

inline eifmm_status launch_xfer_gemm(const XferGemm& a, cudaStream_t s) {
  const dim3 grid((unsigned)((a.ldk + 63) / 64), (unsigned)((a.ncol + 63) / 64), 8);
  k_xfer_gemm<<<grid, 256, 0, s>>>(a);
  EIFMM_CHECK_LAUNCH();
  if (a.mode == 0) {
    const int64_t n4 = a.ncol * a.ldk / 4;
    k_sum8<<<(unsigned)((n4 + 255) / 256 < 8192 ? (n4 + 255) / 256 : 8192), 256, 0, s>>>(
        (const float4*)a.P8, n4, (float4*)a.C);
    EIFMM_CHECK_LAUNCH();
  }
  return EIFMM_OK;
}

}  // namespace eifmm
