// fmm64.cu -- the plain FP64 GPU EIFMM: Algorithm 3 (steps 1-7) + f_N.
//
// Layout of every far-field array of level k: [box (Morton)][rhs][m], FP64.
// These kernels are the FP64 reference path on the GPU (and the baseline the
// mixed-precision path is measured against): one thread per output entry,
// operands staged in shared memory, operators read coalesced along m.
#include <cstdlib>

#include "internal.h"
#include "transfer.cuh"
#include "solve.cuh"

namespace eifmm {
namespace {

constexpr int TPB = 128;
constexpr int RC = 4;  // right-hand sides per pass in the point kernels

__device__ __forceinline__ void leaf_center(int64_t key, int depth, double lo0,
                                            double lo1, double lo2, double lk,
                                            double* c) {
  int ic[3];
  morton_decode(key, depth, ic);
  c[0] = lo0 + (2.0 * ic[0] + 1.0) * lk;
  c[1] = lo1 + (2.0 * ic[1] + 1.0) * lk;
  c[2] = lo2 + (2.0 * ic[2] + 1.0) * lk;
}

__global__ void k_gather_sigma(const double* __restrict__ sigma, int64_t ld,
                               const int32_t* __restrict__ perm, int64_t n, int R,
                               double* __restrict__ s64, float* __restrict__ s32) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int64_t i = perm[p];
  for (int r = 0; r < R; ++r) {
    const double v = sigma[i + r * ld];
    if (s64) s64[p + r * n] = v;
    if (s32) s32[p + r * n] = (float)v;
  }
}

// Step 1: W_m^I = sum_{y_j in I} sigma_j K(x_m^{I_0}, y_j - c_I).
template <int KERN>
__global__ void __launch_bounds__(TPB)
k_p2m64(int kern_rt, const int32_t* __restrict__ leaves, const int32_t* __restrict__ off,
        const double* __restrict__ px, const double* __restrict__ py,
        const double* __restrict__ pz, const double* __restrict__ sig, int64_t n,
        int R, int depth, double lo0, double lo1, double lo2, double lk,
        const double* __restrict__ X, int d, double* __restrict__ W) {
  const int kern = KERN >= 0 ? KERN : kern_rt;
  __shared__ double sz[3][TPB];
  __shared__ double ss[RC][TPB];
  const int b = leaves[blockIdx.x];
  double c[3];
  leaf_center(b, depth, lo0, lo1, lo2, lk, c);
  const int beg = off[b], end = off[b + 1];
  for (int r0 = 0; r0 < R; r0 += RC) {
    for (int m0 = 0; m0 < d; m0 += TPB) {
      const int m = m0 + threadIdx.x;
      double xm0 = 0, xm1 = 0, xm2 = 0;
      if (m < d) { xm0 = X[3 * m]; xm1 = X[3 * m + 1]; xm2 = X[3 * m + 2]; }
      double acc[RC] = {0, 0, 0, 0};
      for (int j0 = beg; j0 < end; j0 += TPB) {
        const int j = j0 + threadIdx.x;
        __syncthreads();
        if (j < end) {
          sz[0][threadIdx.x] = px[j] - c[0];
          sz[1][threadIdx.x] = py[j] - c[1];
          sz[2][threadIdx.x] = pz[j] - c[2];
#pragma unroll
          for (int rr = 0; rr < RC; ++rr) ss[rr][threadIdx.x] = (r0 + rr < R) ? sig[j + (r0 + rr) * n] : 0.0;
        }
        __syncthreads();
        const int cnt = min(TPB, end - j0);
        if (m < d)
          for (int t = 0; t < cnt; ++t) {
            const double kv = kern_f64(kern, xm0 - sz[0][t], xm1 - sz[1][t], xm2 - sz[2][t]);
#pragma unroll
            for (int rr = 0; rr < RC; ++rr) acc[rr] += ss[rr][t] * kv;
          }
      }
      if (m < d)
        for (int rr = 0; rr < RC && r0 + rr < R; ++rr) W[((int64_t)b * R + r0 + rr) * d + m] = acc[rr];
    }
  }
}



// Step 4: g^I = sum_{J in I(I)} K^delta What^J.  A block owns 8 target boxes
// of one parity class (same octant, 8 consecutive parents): they share the
// 189 candidate offsets; sources outside the cube contribute zero.
constexpr int M2L_NB = 8;
constexpr int M2L_MPT = 4;  // rows per thread: d <= 512
template <bool SPLIT>
__global__ void __launch_bounds__(TPB)
k_m2l64(int level, int d, int R, const double* __restrict__ kdT,
        const int* __restrict__ slot_lists, const double* __restrict__ Wh,
        double* __restrict__ g, int groups, int64_t part_stride) {
  extern __shared__ double sw[];  // [M2L_NB][d]
  const int r = blockIdx.y;
  // SPLIT: offset group blockIdx.z of `groups` takes its share of the
  // offset list and writes slice blockIdx.z of the partial buffer g
  const int s_beg = SPLIT ? (int)blockIdx.z * kListLen / groups : 0;
  const int s_end = SPLIT ? ((int)blockIdx.z + 1) * kListLen / groups : kListLen;
  if (SPLIT) g += (int64_t)blockIdx.z * part_stride;
  const int oct = blockIdx.x & 7;
  const int64_t pg = blockIdx.x >> 3;
  const int n = 1 << level;
  int ci[M2L_NB][3];
  int64_t I[M2L_NB];
  for (int b = 0; b < M2L_NB; ++b) {
    I[b] = 8 * (M2L_NB * pg + b) + oct;
    morton_decode(I[b], level, ci[b]);
  }
  double acc[M2L_MPT][M2L_NB];
#pragma unroll
  for (int t = 0; t < M2L_MPT; ++t)
#pragma unroll
    for (int b = 0; b < M2L_NB; ++b) acc[t][b] = 0.0;
  const int* lst = slot_lists + oct * kListLen;
  // the loop keeps its constant trip count and skips the other groups'
  // offsets: with the group's range as the loop bounds the same kernel ran
  // 4.5 times slower at the 2^20-point leaf level (737 against 163 ms)
  for (int s = 0; s < kListLen; ++s) {
    if (SPLIT && (s < s_beg || s >= s_end)) continue;  // block-uniform
    const int slot = lst[s];
    const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
    __syncthreads();
    bool any = false;
    for (int b = 0; b < M2L_NB; ++b) {
      const int jx = ci[b][0] + dx, jy = ci[b][1] + dy, jz = ci[b][2] + dz;
      const bool ok = jx >= 0 && jy >= 0 && jz >= 0 && jx < n && jy < n && jz < n;
      any |= ok;
      const int64_t J = ok ? morton_encode(jx, jy, jz, level) : 0;
      for (int l = threadIdx.x; l < d; l += TPB) sw[b * d + l] = ok ? Wh[(J * R + r) * d + l] : 0.0;
    }
    __syncthreads();
    if (!any) continue;
    const double* K = kdT + (int64_t)slot * d * d;
    for (int l = 0; l < d; ++l) {
      double wv[M2L_NB];
#pragma unroll
      for (int b = 0; b < M2L_NB; ++b) wv[b] = sw[b * d + l];
#pragma unroll
      for (int t = 0; t < M2L_MPT; ++t) {
        const int mp = threadIdx.x + t * TPB;
        if (mp < d) {
          const double kv = K[(int64_t)l * d + mp];
#pragma unroll
          for (int b = 0; b < M2L_NB; ++b) acc[t][b] += kv * wv[b];
        }
      }
    }
  }
#pragma unroll
  for (int t = 0; t < M2L_MPT; ++t) {
    const int mp = threadIdx.x + t * TPB;
    if (mp < d)
#pragma unroll
      for (int b = 0; b < M2L_NB; ++b) g[(I[b] * R + r) * d + mp] = acc[t][b];
  }
}


// Step 4 of the mixed path's tier 3 (FP64 far field) with the FP64 numbers
// carried as unevaluated sums of two FP32 numbers (hi + lo, about 46
// significant bits) on the FP32 pipes, which run 72 times faster than the
// FP64 ones on this GPU.  Each product hi_a hi_b is split exactly with an
// FMA (p + e), the cross terms hi_a lo_b + lo_a hi_b are added in FP32, and
// the running sum is an FP32 pair updated with an error-free two-sum.
// Inputs and output are the FP64 arrays of the FP64 path; the split into
// pairs happens while the tiles are staged.  Tile: 64 target boxes of one
// parity class x 64 rows m', 4 x 4 per thread, terms l in chunks of 16.
constexpr int DF_BOX = 64, DF_ROW = 64, DF_L = 16, DF_THREADS = 256;

__device__ __forceinline__ void df_split(double x, float& h, float& l) {
  h = (float)x;
  l = (float)(x - (double)h);
}

// Three CTAs per SM (80 registers; small spills outside the inner loop):
// the leaf level at 2^20 points, eps 1e-6, took 131 ms with two (128
// registers), 122 ms with three, 125 ms with four (64 registers, spills)
// and 182 ms with one.
__global__ void __launch_bounds__(DF_THREADS, 3)
k_m2l_df(int level, int d, int R, const double* __restrict__ kdT, const int* __restrict__ slot_lists,
         const double* __restrict__ W, double* __restrict__ g, int groups, int64_t part_stride) {
  __shared__ __align__(16) float sWh[DF_L][DF_BOX], sWl[DF_L][DF_BOX];  // [l][box]
  __shared__ __align__(16) float sTh[DF_L][DF_ROW], sTl[DF_L][DF_ROW];  // [l][m']
  __shared__ int64_t s_src[DF_BOX];
  __shared__ int s_c[DF_BOX][3];
  const int tid = threadIdx.x;
  const int r = (int)blockIdx.z % R, grp = (int)blockIdx.z / R;  // column, offset group
  const int s_beg = grp * kListLen / groups, s_end = (grp + 1) * kListLen / groups;
  g += (int64_t)grp * part_stride;
  const int oct = blockIdx.x & 7;
  const int64_t per_class = (int64_t)1 << (3 * (level - 1));
  const int nb = per_class < DF_BOX ? (int)per_class : DF_BOX;
  const int64_t p0 = (blockIdx.x >> 3) * (int64_t)DF_BOX;
  const int m0 = blockIdx.y * DF_ROW;
  const int n = 1 << level;
  if (tid < DF_BOX) {
    int c[3] = {0, 0, 0};
    if (tid < nb) morton_decode(8 * (p0 + tid) + oct, level, c);
    s_c[tid][0] = c[0];
    s_c[tid][1] = c[1];
    s_c[tid][2] = c[2];
  }
  // rows from the warp index: a warp whose 8 rows all lie at or beyond d
  // (the padding of the last row tile) skips the sums
  const int tm = (tid >> 4) * 4, tb = (tid & 15) * 4;
  const bool rows_live = m0 + (tid >> 5) * 8 < d;
  // running sums (hi, lo) of boxes tb.. x rows tm..; rows 2jp, 2jp + 1 side
  // by side in a float2, the pair arithmetic done two rows at a time by the
  // f32x2 builtins (the same IEEE operations as one row at a time: a - b is
  // fma(b, -1, a), and -p is formed as (-w) t)
  float2 ah[4][2], al[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) ah[i][j] = al[i][j] = make_float2(0.f, 0.f);
  const float2 m1 = make_float2(-1.f, -1.f);
  const int* lst = slot_lists + oct * kListLen;
  const int lb = tid >> 2, lq = (tid & 3) * 4;   // staging: box lb, terms lq..lq+3
  const int ll = tid >> 4, lm = (tid & 15) * 4;  // staging: term ll, rows lm..lm+3
  for (int s = 0; s < kListLen; ++s) {
    if (s < s_beg || s >= s_end) continue;  // block-uniform
    const int slot = lst[s];
    const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
    __syncthreads();
    if (tid < DF_BOX) {
      const int jx = s_c[tid][0] + dx, jy = s_c[tid][1] + dy, jz = s_c[tid][2] + dz;
      const bool ok = tid < nb && jx >= 0 && jy >= 0 && jz >= 0 && jx < n && jy < n && jz < n;
      s_src[tid] = ok ? (morton_encode(jx, jy, jz, level) * R + r) * d : -1;
    }
    __syncthreads();
    const double* K = kdT + (int64_t)slot * d * d;
    const int64_t so = s_src[lb];
    // the FP64 entries of the next chunk are loaded while the current one is
    // summed
    double wq[4], kq[4];
    auto load = [&](int l0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int l = l0 + lq + q;
        wq[q] = (so >= 0 && l < d) ? W[so + l] : 0.0;
        const int lk = l0 + ll, mp = m0 + lm + q;
        kq[q] = (lk < d && mp < d) ? __ldg(K + (int64_t)lk * d + mp) : 0.0;
      }
    };
    load(0);
    for (int l0 = 0; l0 < d; l0 += DF_L) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        df_split(wq[q], sWh[lq + q][lb], sWl[lq + q][lb]);
        df_split(kq[q], sTh[ll][lm + q], sTl[ll][lm + q]);
      }
      __syncthreads();
      if (l0 + DF_L < d) load(l0 + DF_L);
#pragma unroll 4
      for (int u = 0; u < DF_L && rows_live; ++u) {
        const float4 wh = *reinterpret_cast<const float4*>(&sWh[u][tb]);
        const float4 wl = *reinterpret_cast<const float4*>(&sWl[u][tb]);
        const float4 th = *reinterpret_cast<const float4*>(&sTh[u][tm]);
        const float4 tl = *reinterpret_cast<const float4*>(&sTl[u][tm]);
        const float whv[4] = {wh.x, wh.y, wh.z, wh.w}, wlv[4] = {wl.x, wl.y, wl.z, wl.w};
        const float2 T[2] = {make_float2(th.x, th.y), make_float2(th.z, th.w)};
        const float2 TL[2] = {make_float2(tl.x, tl.y), make_float2(tl.z, tl.w)};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 Wp = make_float2(whv[i], whv[i]), Wn = make_float2(-whv[i], -whv[i]);
          const float2 WL = make_float2(wlv[i], wlv[i]);
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            // explicit roundings: no contraction may merge the product into
            // the two-sum
            const float2 pn = __fmul2_rn(Wn, T[j]);                           // -p, p = wh th
            const float2 e = __ffma2_rn(Wp, T[j], pn);                        // wh th - p
            const float2 c = __ffma2_rn(Wp, TL[j], __fmul2_rn(WL, T[j]));      // wh tl + wl th
            const float2 sum = __ffma2_rn(pn, m1, ah[i][j]);                  // ah + p
            const float2 bb = __ffma2_rn(ah[i][j], m1, sum);                  // sum - ah
            const float2 t2 = __ffma2_rn(__ffma2_rn(bb, m1, sum), m1, ah[i][j]);  // ah - (sum - bb)
            const float2 err = __ffma2_rn(__fadd2_rn(pn, bb), m1, t2);        // t2 + (p - bb)
            al[i][j] = __fadd2_rn(al[i][j], __fadd2_rn(err, __fadd2_rn(e, c)));
            ah[i][j] = sum;
          }
        }
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (tb + i >= nb) break;
    const int64_t I = 8 * (p0 + tb + i) + oct;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int mp = m0 + tm + j;
      const float h2 = (j & 1) ? ah[i][j >> 1].y : ah[i][j >> 1].x;
      const float l2 = (j & 1) ? al[i][j >> 1].y : al[i][j >> 1].x;
      if (mp < d) g[(I * R + r) * d + mp] = (double)h2 + (double)l2;
    }
  }
}

// Step 7 + sum + un-permute: f(x_i) = sum_l' K(x_i - c_I, y_l'^{I_0}) lhat_l'
// + f_N(x_i), written to the caller's original order.
template <int KERN>
__global__ void __launch_bounds__(TPB)
k_l2p64(int kern_rt, const int32_t* __restrict__ leaves, const int32_t* __restrict__ off,
        const int32_t* __restrict__ perm, const double* __restrict__ px,
        const double* __restrict__ py, const double* __restrict__ pz, int64_t n,
        int R, int depth, double lo0, double lo1, double lo2, double lk,
        const double* __restrict__ X, int d, const double* __restrict__ lh,
        const double* __restrict__ fnear, double* __restrict__ ffar,
        double* __restrict__ f, int64_t ld_f) {
  const int kern = KERN >= 0 ? KERN : kern_rt;
  extern __shared__ double sm[];  // X (3d) then lhat (RC * d)
  double* sX = sm;
  double* sl = sm + 3 * d;
  const int b = leaves[blockIdx.x];
  double c[3];
  leaf_center(b, depth, lo0, lo1, lo2, lk, c);
  const int beg = off[b], end = off[b + 1];
  for (int t = threadIdx.x; t < 3 * d; t += TPB) sX[t] = X[t];
  for (int r0 = 0; r0 < R; r0 += RC) {
    __syncthreads();
    for (int t = threadIdx.x; t < RC * d; t += TPB) {
      const int rr = t / d, l = t - rr * d;
      sl[t] = (r0 + rr < R) ? lh[((int64_t)b * R + r0 + rr) * d + l] : 0.0;
    }
    __syncthreads();
    for (int p = beg + threadIdx.x; p < end; p += TPB) {
      const double z0 = px[p] - c[0], z1 = py[p] - c[1], z2 = pz[p] - c[2];
      double acc[RC] = {0, 0, 0, 0};
      for (int l = 0; l < d; ++l) {
        const double kv = kern_f64(kern, z0 - sX[3 * l], z1 - sX[3 * l + 1], z2 - sX[3 * l + 2]);
#pragma unroll
        for (int rr = 0; rr < RC; ++rr) acc[rr] += kv * sl[rr * d + l];
      }
      const int64_t i = perm[p];
      for (int rr = 0; rr < RC && r0 + rr < R; ++rr) {
        const int rg = r0 + rr;
        if (ffar) ffar[p + rg * n] = acc[rr];
        f[i + rg * ld_f] = acc[rr] + fnear[p + rg * n];
      }
    }
  }
}

// Near field f_N(x_i) = sum over the 27 neighbouring leaves, FP64.
template <int KERN>
__global__ void __launch_bounds__(TPB)
k_p2p64(int kern_rt, const int32_t* __restrict__ leaves, const int32_t* __restrict__ toff,
        const double* __restrict__ tx, const double* __restrict__ ty,
        const double* __restrict__ tz, int64_t nt, const int32_t* __restrict__ soff,
        const double* __restrict__ sx, const double* __restrict__ sy,
        const double* __restrict__ sz, const double* __restrict__ sig, int64_t ns,
        int R, int depth, int exclude_self, double* __restrict__ fnear) {
  const int kern = KERN >= 0 ? KERN : kern_rt;
  __shared__ double s[3][TPB];
  __shared__ double ssg[RC][TPB];
  const int b = leaves[blockIdx.x];
  int c[3];
  morton_decode(b, depth, c);
  const int n = 1 << depth;
  const int beg = toff[b], end = toff[b + 1];
  for (int r0 = 0; r0 < R; r0 += RC) {
    for (int p0 = beg; p0 < end; p0 += TPB) {
      const int p = p0 + threadIdx.x;
      const bool act = p < end;
      const double x0 = act ? tx[p] : 0.0, x1 = act ? ty[p] : 0.0, x2 = act ? tz[p] : 0.0;
      double acc[RC] = {0, 0, 0, 0};
      for (int nb = 0; nb < 27; ++nb) {
        const int jx = c[0] + nb % 3 - 1, jy = c[1] + (nb / 3) % 3 - 1, jz = c[2] + nb / 9 - 1;
        if (jx < 0 || jy < 0 || jz < 0 || jx >= n || jy >= n || jz >= n) continue;
        const int64_t J = morton_encode(jx, jy, jz, depth);
        const int sb = soff[J], se = soff[J + 1];
        for (int q0 = sb; q0 < se; q0 += TPB) {
          __syncthreads();
          const int q = q0 + threadIdx.x;
          if (q < se) {
            s[0][threadIdx.x] = sx[q];
            s[1][threadIdx.x] = sy[q];
            s[2][threadIdx.x] = sz[q];
#pragma unroll
            for (int rr = 0; rr < RC; ++rr) ssg[rr][threadIdx.x] = (r0 + rr < R) ? sig[q + (r0 + rr) * ns] : 0.0;
          }
          __syncthreads();
          const int cnt = min(TPB, se - q0);
          if (act)
            for (int t = 0; t < cnt; ++t) {
              if (exclude_self && q0 + t == p) continue;
              const double kv = kern_f64(kern, x0 - s[0][t], x1 - s[1][t], x2 - s[2][t]);
#pragma unroll
              for (int rr = 0; rr < RC; ++rr) acc[rr] += ssg[rr][t] * kv;
            }
        }
      }
      if (act)
        for (int rr = 0; rr < RC && r0 + rr < R; ++rr) fnear[p + (int64_t)(r0 + rr) * nt] = acc[rr];
    }
  }
}

// Exact FP64 sum for accuracy checks: one block per evaluated target.
__global__ void __launch_bounds__(256)
k_direct64(int kern, const double* __restrict__ tgt, const double* __restrict__ src,
           int64_t ns, const double* __restrict__ sig, int64_t ld, int R, int exclude_self,
           const int64_t* __restrict__ idx, int64_t n_eval, double* __restrict__ f) {
  __shared__ double red[8][8];
  const int64_t e = blockIdx.x;
  const int64_t i = idx ? idx[e] : e;
  const double x0 = tgt[3 * i], x1 = tgt[3 * i + 1], x2 = tgt[3 * i + 2];
  for (int r0 = 0; r0 < R; r0 += 8) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t j = threadIdx.x; j < ns; j += 256) {
      if (exclude_self && j == i) continue;
      const double kv = kern_f64_ieee(kern, x0 - src[3 * j], x1 - src[3 * j + 1], x2 - src[3 * j + 2]);
#pragma unroll
      for (int rr = 0; rr < 8; ++rr)
        if (r0 + rr < R) acc[rr] += sig[j + (r0 + rr) * ld] * kv;
    }
#pragma unroll
    for (int rr = 0; rr < 8; ++rr)
      for (int o = 16; o > 0; o >>= 1) acc[rr] += __shfl_down_sync(0xffffffffu, acc[rr], o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0)
      for (int rr = 0; rr < 8; ++rr) red[w][rr] = acc[rr];
    __syncthreads();
    if (threadIdx.x < 8 && r0 + (int)threadIdx.x < R) {
      double s = 0.0;
      for (int ww = 0; ww < 8; ++ww) s += red[ww][threadIdx.x];
      f[e + (r0 + threadIdx.x) * n_eval] = s;
    }
  }
}

}  // namespace

eifmm_status launch_direct_sum(int kern, const double* tgt, const double* src, int64_t n_src,
                               const double* sigma, int64_t ld, int R, int exclude_self,
                               const int64_t* idx, int64_t n_eval, double* f, cudaStream_t s) {
  k_direct64<<<(unsigned)n_eval, 256, 0, s>>>(kern, tgt, src, n_src, sigma, ld, R, exclude_self,
                                              idx, n_eval, f);
  EIFMM_CHECK_LAUNCH();
  return EIFMM_OK;
}

eifmm_status launch_gather_sigma(const double* sigma, int64_t ld, const PointSet& src, int R,
                                 double* s64, float* s32, cudaStream_t s) {
  if (src.n == 0) return EIFMM_OK;
  k_gather_sigma<<<(unsigned)((src.n + 255) / 256), 256, 0, s>>>(sigma, ld, src.perm, src.n, R, s64, s32);
  EIFMM_CHECK_LAUNCH();
  return EIFMM_OK;
}

eifmm_status launch_p2p64(const Tree* t, int kern, const double* sig, int R, double* fnear,
                          cudaStream_t s) {
  const PointSet& T = t->tgt;
  const PointSet& S = t->src;
  if (T.n_nonempty == 0) return EIFMM_OK;
  if (kern == EIFMM_KERNEL_INV_R)
    k_p2p64<EIFMM_KERNEL_INV_R><<<T.n_nonempty, TPB, 0, s>>>(
        kern, T.nonempty, T.leaf_off, T.x, T.y, T.z, T.n, S.leaf_off, S.x, S.y, S.z, sig, S.n, R,
        t->depth, t->exclude_self, fnear);
  else
    k_p2p64<-1><<<T.n_nonempty, TPB, 0, s>>>(kern, T.nonempty, T.leaf_off, T.x, T.y, T.z, T.n,
                                             S.leaf_off, S.x, S.y, S.z, sig, S.n, R, t->depth,
                                             t->exclude_self, fnear);
  EIFMM_CHECK_LAUNCH();
  return EIFMM_OK;
}


static void record(Workspace& ws, int i, cudaStream_t s) {
  if (timing_enabled()) cudaEventRecord(ws.ev_t[i], s);
}

// Step 4 of level k on FP64 arrays [box R + r][d]: the operator stack kdT
// ([343][l][m'], d x d) applied by FP32-pair arithmetic or in FP64.
// Offset groups of the FP64 and pair-arithmetic M2L: a coarse level has few
// blocks (8 to 64 at levels 2 and 3), each walking all 189 offsets, so the
// offset list is split until the blocks cover two waves of the SMs (at most
// 16 groups); the groups' partial sums are then added in group order.
int m2l64_groups(int64_t blocks, int nsm) {
  int g = 1;
  while (g < 16 && blocks * g < 2 * (int64_t)nsm) g *= 2;
  return g;
}

int64_t m2l_df_blocks(int level, int d, int R) {
  const int64_t nb = (int64_t)1 << (3 * level);
  return ((nb / 8 + DF_BOX - 1) / DF_BOX) * 8 * ((d + DF_ROW - 1) / DF_ROW) * R;
}
int64_t m2l64_blocks(int level, int R) { return ((int64_t)1 << (3 * level)) / 8 / M2L_NB * 8 * R; }

// g[i] = sum over the groups of part[grp * stride + i], in group order
__global__ void k_sum_groups64(const double* __restrict__ part, int groups, int64_t stride,
                               double* __restrict__ g) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < stride;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = part[i];
    for (int k = 1; k < groups; ++k) v += part[k * stride + i];
    g[i] = v;
  }
}

static eifmm_status sum_groups64(const double* part, int groups, int64_t n, double* g, cudaStream_t s) {
  const int64_t blocks = (n + 255) / 256;
  k_sum_groups64<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(part, groups, n, g);
  EIFMM_CHECK_LAUNCH();
  return EIFMM_OK;
}

eifmm_status launch_m2l_df(int level, int d, int R, const double* kdT, const int* slot_lists, const double* W,
                           double* g, double* part, size_t part_cap, int nsm, cudaStream_t s) {
  const int64_t nb = (int64_t)1 << (3 * level);
  const int64_t n = nb * R * d;
  int G = m2l64_groups(m2l_df_blocks(level, d, R), nsm);
  if ((size_t)G * n > part_cap) G = 1;
  k_m2l_df<<<dim3((unsigned)(((nb / 8 + DF_BOX - 1) / DF_BOX) * 8), (unsigned)((d + DF_ROW - 1) / DF_ROW),
                  (unsigned)(R * G)), DF_THREADS, 0, s>>>(level, d, R, kdT, slot_lists, W, G > 1 ? part : g, G, n);
  EIFMM_CHECK_LAUNCH();
  return G > 1 ? sum_groups64(part, G, n, g, s) : EIFMM_OK;
}

eifmm_status launch_m2l64(int level, int d, int R, const double* kdT, const int* slot_lists, const double* W,
                          double* g, double* part, size_t part_cap, int nsm, cudaStream_t s) {
  const int64_t nb = (int64_t)1 << (3 * level);
  const int64_t n = nb * R * d;
  int G = m2l64_groups(m2l64_blocks(level, R), nsm);
  if ((size_t)G * n > part_cap) G = 1;
  if (G > 1)
    k_m2l64<true><<<dim3((unsigned)(nb / 8 / M2L_NB * 8), R, G), TPB, M2L_NB * d * sizeof(double), s>>>(
        level, d, R, kdT, slot_lists, W, part, G, n);
  else
    k_m2l64<false><<<dim3((unsigned)(nb / 8 / M2L_NB * 8), R), TPB, M2L_NB * d * sizeof(double), s>>>(
        level, d, R, kdT, slot_lists, W, g, 1, n);
  EIFMM_CHECK_LAUNCH();
  return G > 1 ? sum_groups64(part, G, n, g, s) : EIFMM_OK;
}

eifmm_status eval_fp64(Tree* t, const Ops* ops, const double* sigma, int64_t ld_sigma, int R,
                       double* f, int64_t ld_f, cudaStream_t s, bool near32, bool pair_m2l) {
  Workspace& ws = t->ws;
  const int kap = t->depth;
  const int kern = (int)ops->kern;
  const PointSet& S = t->src;
  const PointSet& T = t->tgt;
  const double lk = t->L * ldexp(1.0, -(kap + 1));
  record(ws, 0, s);
  EIFMM_TRY(launch_gather_sigma(sigma, ld_sigma, S, R, ws.sig, near32 ? ws.sig32 : nullptr, s));
  // near field on the side stream, concurrent with the far field (on the
  // caller's stream, before it, with the single-stream option)
  EIFMM_CUDA(cudaEventRecord(ws.ev_fork, s));
  EIFMM_CUDA(cudaStreamWaitEvent(ws.side, ws.ev_fork, 0));
  const cudaStream_t nf_stream = t->opt[EIFMM_OPT_SINGLE_STREAM] ? s : ws.side;
  if (timing_enabled()) cudaEventRecord(ws.ev_nf[0], nf_stream);
  if (near32) EIFMM_TRY(launch_p2p32(t, kern, ws.sig32, R, ws.fnear, nf_stream, true));
  else EIFMM_TRY(launch_p2p64(t, kern, ws.sig, R, ws.fnear, nf_stream));
  if (timing_enabled()) cudaEventRecord(ws.ev_nf[1], nf_stream);
  EIFMM_CUDA(cudaEventRecord(ws.ev_join, ws.side));

  // step 1
  const LevelOps& vl = ops->lv[kap];
  EIFMM_CUDA(cudaMemsetAsync(ws.W[kap], 0, sizeof(double) * ((size_t)1 << (3 * kap)) * R * vl.d, s));
  if (S.n_nonempty > 0) {
    if (kern == EIFMM_KERNEL_INV_R)
      k_p2m64<EIFMM_KERNEL_INV_R><<<S.n_nonempty, TPB, 0, s>>>(
          kern, S.nonempty, S.leaf_off, S.x, S.y, S.z, ws.sig, S.n, R, kap, t->lo[0], t->lo[1],
          t->lo[2], lk, vl.X, vl.d, ws.W[kap]);
    else
      k_p2m64<-1><<<S.n_nonempty, TPB, 0, s>>>(kern, S.nonempty, S.leaf_off, S.x, S.y, S.z, ws.sig,
                                               S.n, R, kap, t->lo[0], t->lo[1], t->lo[2], lk, vl.X,
                                               vl.d, ws.W[kap]);
    EIFMM_CHECK_LAUNCH();
  }
  record(ws, 1, s);
  // step 2
  for (int k = kap - 1; k >= 2; --k) {
    const int dk = ops->lv[k].d, dc = ops->lv[k + 1].d;
    const int64_t np = (int64_t)1 << (3 * k);
    k_m2m_warp<double><<<xfer_blocks(np, R, dk), 128, 0, s>>>(dk, dc, dk, dc, R, ops->lv[k].m2m,
                                                             ws.W[k + 1], ws.W[k], np);
    EIFMM_CHECK_LAUNCH();
  }
  record(ws, 2, s);
  // step 3: What = Delta W is folded into the M2L operator (kdT holds
  // K^delta Delta), so step 4 reads W; What itself is formed only when it is
  // exported
  record(ws, 3, s);
  // step 4 (the compressed operators of Section 4.2 when they are built)
  for (int k = 2; k <= kap; ++k) {
    if (timing_enabled()) cudaEventRecord(ws.ev_m2l[k], s);
    const bool pair = pair_m2l && !t->opt[EIFMM_OPT_M2L_FP64];  // tiers 3 and 4: FP32 pairs
    if (ops->compressed && ops->lv[k].r > 0)
      EIFMM_TRY(m2l_compressed(ws, ops, k, R, pair, s));
    else if (pair)
      EIFMM_TRY(launch_m2l_df(k, ops->lv[k].d, R, ops->lv[k].kdT, ops->d_slot_lists, ws.W[k], ws.g[k],
                              ws.part64, ws.part64_cap, ws.nsm, s));
    else
      EIFMM_TRY(launch_m2l64(k, ops->lv[k].d, R, ops->lv[k].kdT, ops->d_slot_lists, ws.W[k], ws.g[k],
                             ws.part64, ws.part64_cap, ws.nsm, s));
    if (timing_enabled()) cudaEventRecord(ws.ev_m2le[k], s);
  }
  record(ws, 4, s);
  // step 5 (l^2 = g^2)
  for (int k = 3; k <= kap; ++k) {
    const int dk = ops->lv[k].d, dp = ops->lv[k - 1].d;
    const int64_t nb = (int64_t)1 << (3 * k);
    k_l2l_warp<double><<<xfer_blocks(nb, R, dk), 128, 0, s>>>(dk, dp, dk, dp, R, ops->lv[k].l2l,
                                                             ws.l[k - 1], ws.g[k], ws.l[k], nb);
    EIFMM_CHECK_LAUNCH();
  }
  record(ws, 5, s);
  // step 6
  {
    DeltaBatch b;
    b.nlev = 1;
    b.lv[0] = delta_level(vl.d, delta_ops64(vl), true, ws.l[kap], vl.d, ws.lh, vl.d, nullptr,
                          ((int64_t)1 << (3 * kap)) * R);
    EIFMM_TRY((launch_delta_batch<double, double, double, 0>(b, true, s)));
  }
  record(ws, 6, s);
  // step 7 + near field + un-permute
  EIFMM_CUDA(cudaStreamWaitEvent(s, ws.ev_join, 0));
  record(ws, 7, s);
  if (T.n_nonempty > 0) {
    const size_t sm = (size_t)(3 * vl.d + RC * vl.d) * sizeof(double);
    if (kern == EIFMM_KERNEL_INV_R)
      k_l2p64<EIFMM_KERNEL_INV_R><<<T.n_nonempty, TPB, sm, s>>>(
          kern, T.nonempty, T.leaf_off, T.perm, T.x, T.y, T.z, T.n, R, kap, t->lo[0], t->lo[1],
          t->lo[2], lk, vl.X, vl.d, ws.lh, ws.fnear, ws.ffar, f, ld_f);
    else
      k_l2p64<-1><<<T.n_nonempty, TPB, sm, s>>>(kern, T.nonempty, T.leaf_off, T.perm, T.x, T.y, T.z,
                                                T.n, R, kap, t->lo[0], t->lo[1], t->lo[2], lk, vl.X,
                                                vl.d, ws.lh, ws.fnear, ws.ffar, f, ld_f);
    EIFMM_CHECK_LAUNCH();
  }
  record(ws, 8, s);
  return EIFMM_OK;
}

}  // namespace eifmm
