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
