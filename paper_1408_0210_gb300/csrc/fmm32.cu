// fmm32.cu -- the mixed-precision EIFMM (Algorithm 3 + near field).
//
// Tier 0: P2M, M2M, the Delta^t solve, L2L and L2P in FP32 on coordinates
// local to each leaf; M2L of the folded operator K^delta Delta on tcgen05
// with BF16 hi + lo operand planes (m2l_tc.cu).  Tier 1: a Newton step on
// every 1/r and M2L with scaled FP16 hi + lo planes, each offset's tensor-
// core accumulator drained into round-to-nearest FP32 sums (levels without
// an FP16 tile use the tier-2 SIMT M2L).
// Tier 2: the M2L on the FP32 SIMT pipes (compensated sums over the offsets),
// the Delta^t solve in FP32, a Newton step on every 1/r.  Tier 3: the FP64 far field of fmm64.cu.  Tiers 0-3 evaluate the
// near field here in FP32 (tiers >= 1 with Kahan compensated summation).
// The tier is chosen by a measured calibration (api.cu).
//
// Far-field arrays: [row = box * R + r][dp] FP32, dp = d rounded up to 64,
// padding columns zero.
#include <algorithm>

#include <cstring>
#include <cstdlib>

#include "internal.h"
#include "m2l_tc.h"
#include "transfer.cuh"
#include "solve.cuh"

namespace eifmm {

eifmm_status launch_gather_sigma(const double* sigma, int64_t ld, const PointSet& src, int R,
                                 double* s64, float* s32, cudaStream_t s);

namespace {

// forward neighbour offsets of the pair-symmetric near field
constexpr int kSymSlots = 13;

constexpr int TPB = 128;
constexpr int RC = 4;

__host__ __device__ inline int64_t nboxes(int k) { return (int64_t)1 << (3 * k); }

// ---------------------------------------------------------------- step 1 --
// W_m^I = sum_{y_j in I} sigma_j K(x_m^{I_0}, y_j - c_I), FP32, local coords.
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// K(z) in FP32 for the point kernels.  1/r: the approximate reciprocal square
// root (about 2 ulp), with one Newton step when ACC.  Other kernels:
// kern_f32 / kern_f32_fast.
template <int KERN, bool ACC>
__device__ __forceinline__ float kern_pt(int kern, float z0, float z1, float z2) {
  if (KERN == EIFMM_KERNEL_INV_R) {
    const float r2 = fmaf(z0, z0, fmaf(z1, z1, z2 * z2));
    const float y = rsqrt_approx(r2);
    return ACC ? y * fmaf(-0.5f * r2, y * y, 1.5f) : y;
  }
  return ACC ? kern_f32(kern, z0, z1, z2) : kern_f32_fast(kern, z0, z1, z2);
}

// Step 1: one CTA per leaf, threads = m (the d coefficients); the leaf's
// points are staged as (x, y, z, sigma_r0) in shared memory.  (Four leaves
// per CTA measured slower: 57 against 54 us at 1M points.)
template <int KERN, int RCT, bool ACC>
__global__ void __launch_bounds__(TPB)
k_p2m32(int kern_rt, const int32_t* __restrict__ off, const float* __restrict__ lx,
        const float* __restrict__ ly, const float* __restrict__ lz,
        const float* __restrict__ sig, int64_t n, int R, const float* __restrict__ X, int d,
        int dp, float* __restrict__ W) {
  const int kern = KERN >= 0 ? KERN : kern_rt;
  __shared__ float4 sp[TPB];
  __shared__ float ss[RCT > 1 ? RCT : 1][TPB];
  const int64_t b = blockIdx.x;
  const int beg = off[b], end = off[b + 1];
  for (int r0 = 0; r0 < R; r0 += RCT) {
    for (int m0 = 0; m0 < dp; m0 += TPB) {
      const int m = m0 + threadIdx.x;
      float x0 = 0.f, x1 = 0.f, x2 = 0.f;
      if (m < d) { x0 = X[3 * m]; x1 = X[3 * m + 1]; x2 = X[3 * m + 2]; }
      float acc[RCT];
#pragma unroll
      for (int rr = 0; rr < RCT; ++rr) acc[rr] = 0.f;
      for (int j0 = beg; j0 < end; j0 += TPB) {
        const int j = j0 + threadIdx.x;
        __syncthreads();
        if (j < end) {
          sp[threadIdx.x] = make_float4(lx[j], ly[j], lz[j], RCT == 1 ? sig[j + r0 * n] : 0.f);
          if (RCT > 1)
#pragma unroll
            for (int rr = 0; rr < RCT; ++rr) ss[rr][threadIdx.x] = (r0 + rr < R) ? sig[j + (r0 + rr) * n] : 0.f;
        }
        __syncthreads();
        const int cnt = min(TPB, end - j0);
        if (m < d)
#pragma unroll 4
          for (int t = 0; t < cnt; ++t) {
            const float4 y = sp[t];
            const float kv = kern_pt<KERN, ACC>(kern, x0 - y.x, x1 - y.y, x2 - y.z);
#pragma unroll
            for (int rr = 0; rr < RCT; ++rr) acc[rr] = fmaf(RCT == 1 ? y.w : ss[rr][t], kv, acc[rr]);
          }
      }
      if (m < dp)  // padding columns are zero
        for (int rr = 0; rr < RCT && r0 + rr < R; ++rr) W[(b * R + r0 + rr) * dp + m] = m < d ? acc[rr] : 0.f;
    }
  }
}
// Step 7: one CTA per non-empty target leaf, threads = (point, slice of l):
// P points of the leaf (up to TPB per pass) times S = TPB / P interleaved
// slices of the d terms.  It writes the far field (ffar, leaf order); with
// f non-null it also adds the near field (and the pair-symmetric partials,
// gsym) and writes f in the caller's order, otherwise k_combine does that.
template <int KERN, int RCT, bool ACC>
__global__ void __launch_bounds__(TPB)
k_l2p32(int kern_rt, const int32_t* __restrict__ leaves, const int32_t* __restrict__ off,
        const int32_t* __restrict__ perm, const float* __restrict__ lx,
        const float* __restrict__ ly, const float* __restrict__ lz, int64_t n, int R,
        const float* __restrict__ X, int d, int dp, const float* __restrict__ lh,
        double* __restrict__ fnear, double* __restrict__ ffar, double* __restrict__ f,
        int64_t ld_f, const float* __restrict__ gsym, int depth) {
  const int kern = KERN >= 0 ? KERN : kern_rt;
  // pair-symmetric near field (gsym): the backward neighbours A = B - o of
  // this leaf B that exist and hold points wrote partials gsym[s][p]
  __shared__ int s_gmask;
  // (x_l, lhat_l of the first right-hand side) [d], lhat of the pass [RCT d]
  // when RCT > 1, slice partials [RCT TPB]
  extern __shared__ float4 smf4[];
  float4* sX = smf4;
  float* sl = (float*)(smf4 + d);
  float* sp = sl + (RCT > 1 ? RCT * d : 0);
  const int tid = threadIdx.x;
  const int b = leaves[blockIdx.x];
  const int beg = off[b], end = off[b + 1];
  if (gsym && tid == 0) {
    int c[3], m = 0;
    morton_decode(b, depth, c);
    const int nside = 1 << depth;
    for (int s = 0; s < 13; ++s) {
      const int nb = 14 + s;
      const int ax = c[0] - (nb % 3 - 1), ay = c[1] - ((nb / 3) % 3 - 1), az = c[2] - (nb / 9 - 1);
      if (ax >= 0 && ay >= 0 && az >= 0 && ax < nside && ay < nside && az < nside) {
        const int64_t A = morton_encode(ax, ay, az, depth);
        if (off[A + 1] > off[A]) m |= 1 << s;
      }
    }
    s_gmask = m;
  }
  for (int r0 = 0; r0 < R; r0 += RCT) {
    __syncthreads();
    for (int l = tid; l < d; l += TPB)
      sX[l] = make_float4(X[3 * l], X[3 * l + 1], X[3 * l + 2], lh[((int64_t)b * R + r0) * dp + l]);
    if (RCT > 1)
      for (int t = tid; t < RCT * d; t += TPB) {
        const int rr = t / d, l = t - rr * d;
        sl[t] = (r0 + rr < R) ? lh[((int64_t)b * R + r0 + rr) * dp + l] : 0.f;
      }
    __syncthreads();
    for (int t0 = beg; t0 < end; t0 += TPB) {
      const int P = min(TPB, end - t0), S = TPB / P;
      const int ti = tid % P, si = tid / P;
      const int p = t0 + ti;
      float acc[RCT];
#pragma unroll
      for (int rr = 0; rr < RCT; ++rr) acc[rr] = 0.f;
      // the output index and (one right-hand side) the near field, loaded
      // before the sum so that their latency overlaps it
      int64_t i_out = 0;
      double fn0 = 0.0;
      if (tid < P && f) {
        i_out = perm[p];
        if (RCT == 1) fn0 = fnear[p + (int64_t)r0 * n];
      }
      if (si < S) {
        const float z0 = lx[p], z1 = ly[p], z2 = lz[p];
#pragma unroll 4
        for (int l = si; l < d; l += S) {
          const float4 x = sX[l];
          const float kv = kern_pt<KERN, ACC>(kern, z0 - x.x, z1 - x.y, z2 - x.z);
#pragma unroll
          for (int rr = 0; rr < RCT; ++rr) acc[rr] = fmaf(kv, RCT == 1 ? x.w : sl[rr * d + l], acc[rr]);
        }
      }
      __syncthreads();
#pragma unroll
      for (int rr = 0; rr < RCT; ++rr) sp[rr * TPB + tid] = acc[rr];
      __syncthreads();
      if (tid < P) {
        const int64_t i = i_out;
#pragma unroll
        for (int rr = 0; rr < RCT; ++rr) {
          if (r0 + rr >= R) break;
          float s = 0.f;
          for (int k = 0; k < S; ++k) s += sp[rr * TPB + ti + k * P];
          const int rg = r0 + rr;
          if (ffar) ffar[p + rg * n] = s;
          if (!f) continue;  // the far field alone; k_combine adds the near field
          double fn = RCT == 1 ? fn0 : fnear[p + rg * n];
          if (gsym) {  // R = 1
            const int m = s_gmask;
            float gs = 0.f;
            for (int q = 0; q < 13; ++q)
              if (m & (1 << q)) gs += gsym[(int64_t)q * n + p];
            fn += (double)gs;
            fnear[p] = fn;
          }
          f[i + rg * ld_f] = (double)s + fn;
        }
      }
    }
  }
}

// f = f_far + f_N in the caller's order, once both are done (the far field
// no longer waits for the near field before its L2P).
__global__ void k_combine(const int32_t* __restrict__ perm, int64_t n, int R, const double* __restrict__ ffar,
                          const double* __restrict__ fnear, double* __restrict__ f, int64_t ld_f) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * R; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n, p = t - r * n;
    f[perm[p] + r * ld_f] = ffar[t] + fnear[t];
  }
}

// Instantiation of a point kernel launch for (kernel, right-hand-side block,
// Newton step); LAUNCH(K, RCT, ACC) expands to the launch.
#define EIFMM_POINT_DISPATCH(LAUNCH)                                        \
  do {                                                                      \
    if (kern == EIFMM_KERNEL_INV_R) {                                       \
      if (R == 1) {                                                         \
        if (acc) LAUNCH(EIFMM_KERNEL_INV_R, 1, true);                       \
        else LAUNCH(EIFMM_KERNEL_INV_R, 1, false);                          \
      } else {                                                              \
        if (acc) LAUNCH(EIFMM_KERNEL_INV_R, RC, true);                      \
        else LAUNCH(EIFMM_KERNEL_INV_R, RC, false);                         \
      }                                                                     \
    } else if (R == 1) {                                                    \
      if (acc) LAUNCH(-1, 1, true);                                         \
      else LAUNCH(-1, 1, false);                                            \
    } else {                                                                \
      if (acc) LAUNCH(-1, RC, true);                                        \
      else LAUNCH(-1, RC, false);                                           \
    }                                                                       \
  } while (0)

// ------------------------------------------------------------ near field --
// One CTA (128 threads) per non-empty target leaf.  The sources of the 27
// neighbour leaves are staged in shared memory (in chunks of P2P_SRC) as
// (x, y, z, sigma) in the frame of the target leaf (exact shift by the
// leaf-centre offset), with the target leaf itself last so that only its
// segment needs the self-pair test; warp w stages segments w, w + 4, ...
// Threads = (target t, slice s), thread = t + P s: P targets of the pass
// (up to 128) times S = 128 / P contiguous slices of the staged list.  Slice
// starts are spaced by L = 2 (mod 8) float4, so the few slices a warp reads
// at once fall in different banks.  The slices of a target are added in FP64
// in a fixed order; FP32 sums run over at most 128 terms before they are
// flushed into a compensated total.
constexpr int P2P_THREADS = 128;
constexpr int P2P_SRC = 1024;
constexpr int P2P_FLUSH = 128;

// Kahan step: (s, c) += v.
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Adds the staged sources jb <= j < je; SELF: position js (the target
// itself) contributes nothing.  ACC: compensated sums of every term and an
// FP64 flush; otherwise plain FP32 sums flushed into FP32 Kahan totals.
template <int KERN, int RCT, bool ACC, bool SELF>
__device__ __forceinline__ void p2p_span(int kern, const float4* __restrict__ src, const float* __restrict__ ssig,
                                         int jb, int je, int js, float x0, float x1, float x2, float (&th)[RCT],
                                         float (&tc)[RCT], double (&td)[RCT]) {
  for (int j0 = jb; j0 < je; j0 += P2P_FLUSH) {
    const int j1 = min(je, j0 + P2P_FLUSH);
    float sa[RCT], ca[RCT];
#pragma unroll
    for (int rr = 0; rr < RCT; ++rr) sa[rr] = ca[rr] = 0.f;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(src);
    auto term = [&](int j) {
      float4 y;  // one 16-byte shared load from a 32-bit shared address
      asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(y.x), "=f"(y.y), "=f"(y.z), "=f"(y.w)
                   : "r"(sbase + 16u * (uint32_t)j));
      float kv = kern_pt<KERN, ACC>(kern, x0 - y.x, x1 - y.y, x2 - y.z);
      if (SELF && j == js) kv = 0.f;
#pragma unroll
      for (int rr = 0; rr < RCT; ++rr) {
        const float sg = RCT == 1 ? y.w : ssig[rr * P2P_SRC + j];
        if (ACC) kahan_add(sa[rr], ca[rr], sg * kv);
        else sa[rr] = fmaf(sg, kv, sa[rr]);
      }
    };
    // ACC: 8 terms at a time summed in plain FP32, each block added to the
    // compensated sum (a Kahan step per block instead of per term)
    auto block8 = [&](int jb8) {
      float bp[RCT];
#pragma unroll
      for (int rr = 0; rr < RCT; ++rr) bp[rr] = 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = jb8 + u;
        float4 y;
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(y.x), "=f"(y.y), "=f"(y.z), "=f"(y.w)
                     : "r"(sbase + 16u * (uint32_t)j));
        float kv = kern_pt<KERN, ACC>(kern, x0 - y.x, x1 - y.y, x2 - y.z);
        if (SELF && j == js) kv = 0.f;
#pragma unroll
        for (int rr = 0; rr < RCT; ++rr) bp[rr] = fmaf(RCT == 1 ? y.w : ssig[rr * P2P_SRC + j], kv, bp[rr]);
      }
#pragma unroll
      for (int rr = 0; rr < RCT; ++rr) kahan_add(sa[rr], ca[rr], bp[rr]);
    };
    int j = j0;
    for (; j + 16 <= j1; j += 16) {
      if (ACC) {
        block8(j);
        block8(j + 8);
      } else {
#pragma unroll
        for (int u = 0; u < 16; ++u) term(j + u);
      }
    }
    for (; j < j1; ++j) term(j);
#pragma unroll
    for (int rr = 0; rr < RCT; ++rr) {
      if (ACC) td[rr] += (double)sa[rr] - (double)ca[rr];
      else kahan_add(th[rr], tc[rr], sa[rr]);
    }
  }
}

template <int KERN, int RCT, bool ACC>
__global__ void __launch_bounds__(P2P_THREADS)
k_p2p32(int kern_rt, const int32_t* __restrict__ leaves, const int32_t* __restrict__ toff,
        const float* __restrict__ tlx, const float* __restrict__ tly, const float* __restrict__ tlz,
        int64_t nt, const int32_t* __restrict__ soff, const float* __restrict__ slx,
        const float* __restrict__ sly, const float* __restrict__ slz, const float* __restrict__ sig,
        int64_t ns, int R, int depth, float two_l, int exclude_self, double* __restrict__ fnear) {
  const int kern = KERN >= 0 ? KERN : kern_rt;
  __shared__ float4 s_src[P2P_SRC + 8];  // x, y, z in the target frame; w = sigma when RCT == 1
  __shared__ float s_sig[RCT > 1 ? RCT * P2P_SRC : 1];
  __shared__ double s_red[RCT][P2P_THREADS];
  __shared__ int s_pos[28];     // prefix of the segment lengths
  __shared__ int s_beg[27];     // first source of each segment
  __shared__ float s_sh[27][3];  // leaf-centre offset of each segment
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int b = leaves[blockIdx.x];
  int c[3];
  morton_decode(b, depth, c);
  const int n = 1 << depth;
  if (tid < 27) {
    // segments 0..25: the neighbours other than the leaf itself, 26: itself
    const int nb = tid < 13 ? tid : (tid < 26 ? tid + 1 : 13);
    const int dx = nb % 3 - 1, dy = (nb / 3) % 3 - 1, dz = nb / 9 - 1;
    const int jx = c[0] + dx, jy = c[1] + dy, jz = c[2] + dz;
    int beg = 0, len = 0;
    if (jx >= 0 && jy >= 0 && jz >= 0 && jx < n && jy < n && jz < n) {
      const int64_t J = morton_encode(jx, jy, jz, depth);
      beg = soff[J];
      len = soff[J + 1] - beg;
    }
    s_beg[tid] = beg;
    s_pos[tid + 1] = len;
    // y - c_I = (y - c_J) + (c_J - c_I)
    s_sh[tid][0] = dx * two_l;
    s_sh[tid][1] = dy * two_l;
    s_sh[tid][2] = dz * two_l;
  }
  __syncthreads();
  if (tid == 0) {
    s_pos[0] = 0;
    for (int i = 1; i <= 27; ++i) s_pos[i] += s_pos[i - 1];
  }
  __syncthreads();
  const int n_other = s_pos[26], n_all = s_pos[27];
  const int beg = toff[b], end = toff[b + 1];
  // Target passes: 128 targets while that many remain, else 32 at a time
  // while more than 32 remain, then the rest, so that P x S fills the block
  // (P = 33 alone would leave 29 threads idle; on uniform leaves this
  // measured neutral, 422 us either way).  With one source chunk and one
  // block of right-hand sides the sources are staged once for all passes,
  // which saves the re-staging for leaves of more than 128 points.
  const bool once = n_all <= P2P_SRC && R <= RCT;
  bool staged = false;
  for (int t0 = beg, P = 0; t0 < end; t0 += P) {
    const int m = end - t0;
    P = m >= P2P_THREADS ? P2P_THREADS : (m > 32 ? 32 : m);
    const int S = P2P_THREADS / P;
    const int ti = tid % P, si = tid / P;
    const bool act = si < S;
    const int p = t0 + ti;
    const float x0 = tlx[p], x1 = tly[p], x2 = tlz[p];
    // the self pair sits at n_other + (p - beg) of the staged list
    const int js_all = exclude_self ? n_other + (p - beg) : -1;
    for (int r0 = 0; r0 < R; r0 += RCT) {
      float th[RCT], tc[RCT];
      double td[RCT];
#pragma unroll
      for (int rr = 0; rr < RCT; ++rr) th[rr] = tc[rr] = 0.f, td[rr] = 0.0;
      for (int c0 = 0; c0 < n_all; c0 += P2P_SRC) {
        const int cn = min(P2P_SRC, n_all - c0);
        if (!(once && staged)) {
          __syncthreads();
          for (int sg = w; sg < 27; sg += P2P_THREADS / 32) {
            const int pb = s_pos[sg], pe = s_pos[sg + 1];
            const int lo = max(pb, c0), hi = min(pe, c0 + cn);
            const float sx = s_sh[sg][0], sy = s_sh[sg][1], sz = s_sh[sg][2];
            for (int pos = lo + lane; pos < hi; pos += 32) {
              const int sj = s_beg[sg] + (pos - pb);
              const int q = pos - c0;
              const float w0 = (RCT == 1 && r0 < R) ? sig[sj + (int64_t)r0 * ns] : 0.f;
              s_src[q] = make_float4(slx[sj] + sx, sly[sj] + sy, slz[sj] + sz, w0);
              if (RCT > 1)
#pragma unroll
                for (int rr = 0; rr < RCT; ++rr)
                  s_sig[rr * P2P_SRC + q] = (r0 + rr < R) ? sig[sj + (int64_t)(r0 + rr) * ns] : 0.f;
            }
          }
          __syncthreads();
          staged = true;
        }
        if (act) {
          // slice si: [si L, min(cn, (si + 1) L)), L = 2 (mod 8)
          int L = (cn + S - 1) / S;
          L += (10 - (L & 7)) & 7;
          const int jb = min(cn, si * L), je = min(cn, jb + L);
          const int a_end = max(jb, min(je, n_other - c0));
          p2p_span<KERN, RCT, ACC, false>(kern, s_src, s_sig, jb, a_end, -1, x0, x1, x2, th, tc, td);
          p2p_span<KERN, RCT, ACC, true>(kern, s_src, s_sig, a_end, je, js_all - c0, x0, x1, x2, th, tc, td);
        }
      }
      __syncthreads();
#pragma unroll
      for (int rr = 0; rr < RCT; ++rr)
        s_red[rr][tid] = act ? (ACC ? td[rr] : (double)th[rr] - (double)tc[rr]) : 0.0;
      __syncthreads();
      if (tid < P)
#pragma unroll
        for (int rr = 0; rr < RCT; ++rr) {
          if (r0 + rr >= R) break;
          double s = 0.0;
          for (int k = 0; k < S; ++k) s += s_red[rr][ti + k * P];
          fnear[p + (int64_t)(r0 + rr) * nt] = s;
        }
    }
  }
}

// -------------------------------------- near field, packed distances ----
// The near field of 1/r with one right-hand side.  One CTA (128 threads)
// per non-empty target leaf.  The sources of the 27 neighbour leaves are
// staged in shared memory in chunks of NF_SRC, in the frame of the target
// leaf, as SoA pairs:
//   pair q: float4 [2q] = (x_2q, x_2q+1 | y_2q, y_2q+1),
//           float4 [2q + 1] = (z_2q, z_2q+1 | sigma_2q, sigma_2q+1),
// the 26 other leaves first, then the leaf itself from the next even
// position; a pad source (far away, sigma = 0, an exact zero) fills an odd
// end.  Threads = (target t, slice s), thread = t + P s: P targets of the
// pass times S = min(128 / P, 32) contiguous slices of about np / S pairs;
// the passes take 128 targets while that many remain, else 32 while more
// than 32 remain, then the rest, so that the lanes stay busy.  Per pair of
// sources the distance is 3 packed differences and 3 packed multiply-adds
// (add/mul/fma.rn.f32x2, operands straight from the shared loads); 1/r is
// the approximate reciprocal square root on each half.  Each half keeps its
// own FP32 sum over the slice (at most 256 pairs) before a compensated
// flush; when ACC, 1/r gets one Newton step and the sum is compensated
// (Kahan) every NF_KBLOCK pairs.  Only the pairs of the leaf
// itself test for the self pair, whose sigma is replaced by 0 (and its zero
// distance by 1).  The slices of a target are added in FP64 in a fixed
// order.  Staging costs about as much as the arithmetic of one target per
// source, so its bookkeeping is kept to a warp scan and two pad writes.
constexpr int NF_THREADS = 128;
constexpr int NF_SRC = 1024;               // sources per chunk
constexpr int NF_MAXS = 32;                // slices per pass
constexpr float NF_FAR = 1.0e4f;
constexpr size_t NF_SMEM = NF_SRC * sizeof(float4);  // NF_SRC / 2 pairs of 32 bytes
constexpr int NF_KBLOCK = 8;               // pairs per plain FP32 block when ACC

// Packed FP32 pairs are float2 values handled by the sm_100 builtins
// __fadd2_rn / __fmul2_rn / __ffma2_rn (the f32x2 add, mul, fma): the halves
// stay ordinary registers, so no moves split or join 64-bit values.  A
// difference a - b is formed as a + (-b) (the same IEEE result), with -b
// negated once outside the loops.

// r2 of the staged pair e[0..1] against the target, given negated as
// (NX, NX), (NY, NY), (NZ, NZ); and the pair's sigma.
__device__ __forceinline__ float2 nf_r2(const float4* e, float2 NX, float2 NY, float2 NZ, float2& sg) {
  const float4 v0 = e[0], v1 = e[1];
  sg = make_float2(v1.z, v1.w);
  const float2 dx = __fadd2_rn(make_float2(v0.x, v0.y), NX);
  const float2 dy = __fadd2_rn(make_float2(v0.z, v0.w), NY);
  const float2 dz = __fadd2_rn(make_float2(v1.x, v1.y), NZ);
  float2 r2 = __fmul2_rn(dx, dx);
  r2 = __ffma2_rn(dy, dy, r2);
  return __ffma2_rn(dz, dz, r2);
}

// sum (+)= sigma / r for one half.
template <bool ACC>
__device__ __forceinline__ void nf_term(float r2, float sg, float& sa, float& ca) {
  float y = rsqrt_approx(r2);
  if (ACC) {
    y = y * fmaf(-0.5f * r2, y * y, 1.5f);
    kahan_add(sa, ca, sg * y);
  } else {
    sa = fmaf(sg, y, sa);
  }
}

// Pairs [qa, qe) of the staged list; SELF: pair qs, half hs is the target
// itself.
// 1/r with one Newton step (ACC)
__device__ __forceinline__ float nf_rsqrt_newton(float r2) {
  const float y = rsqrt_approx(r2);
  return y * fmaf(-0.5f * r2, y * y, 1.5f);
}

template <bool ACC, bool SELF>
__device__ __forceinline__ void nf_span(const float4* s_pair, int qa, int qe, int qs, int hs, float2 NX,
                                        float2 NY, float2 NZ, float& sl, float& sh, float& cl, float& ch) {
  int q = qa;
  if (ACC) {
    // blocks of NF_KBLOCK pairs summed in plain FP32, each block added to
    // the compensated total: the Kahan step once per block instead of once
    // per term
    for (; q + NF_KBLOCK <= qe; q += NF_KBLOCK) {
      float pl = 0.f, ph = 0.f;
#pragma unroll
      for (int u = 0; u < NF_KBLOCK; ++u) {
        float2 sg;
        float2 r2 = nf_r2(s_pair + 2 * (q + u), NX, NY, NZ, sg);
        if (SELF && q + u == qs) {  // the self pair: sigma 0 at distance 1
          if (hs) r2.y = 1.f, sg.y = 0.f;
          else r2.x = 1.f, sg.x = 0.f;
        }
        pl = fmaf(sg.x, nf_rsqrt_newton(r2.x), pl);
        ph = fmaf(sg.y, nf_rsqrt_newton(r2.y), ph);
      }
      kahan_add(sl, cl, pl);
      kahan_add(sh, ch, ph);
    }
  }
#pragma unroll 8
  for (; q < qe; ++q) {
    float2 sg;
    float2 r2 = nf_r2(s_pair + 2 * q, NX, NY, NZ, sg);
    if (SELF && q == qs) {  // the self pair: sigma 0 at distance 1
      if (hs) r2.y = 1.f, sg.y = 0.f;
      else r2.x = 1.f, sg.x = 0.f;
    }
    nf_term<ACC>(r2.x, sg.x, sl, cl);
    nf_term<ACC>(r2.y, sg.y, sh, ch);
  }
}

// (Capping it at 40 registers for 12 CTAs per SM instead of 10 made the
// evaluate slower: 1.053 against 1.045 ms at 2^20 points.)
template <bool ACC>
__global__ void __launch_bounds__(NF_THREADS)
k_p2p32x(const int32_t* __restrict__ leaves, const int32_t* __restrict__ toff, const float* __restrict__ tlx,
         const float* __restrict__ tly, const float* __restrict__ tlz, const int32_t* __restrict__ soff,
         const float* __restrict__ slx, const float* __restrict__ sly, const float* __restrict__ slz,
         const float* __restrict__ sig, int depth, float two_l, int exclude_self, double* __restrict__ fnear) {
  extern __shared__ __align__(16) float4 s_pair[];  // [NF_SRC]: NF_SRC / 2 pairs
  __shared__ double s_red[NF_THREADS];
  __shared__ int s_pos[28];  // logical start of each segment, then the end
  __shared__ int s_len[27];
  __shared__ int s_beg[27];
  __shared__ float s_sh[27][3];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int b = leaves[blockIdx.x];
  if (w == 0) {
    // segment `lane`: 0..25 the neighbours other than the leaf, 26 itself
    int c[3];
    morton_decode(b, depth, c);
    const int n = 1 << depth;
    int beg = 0, len = 0;
    if (lane < 27) {
      const int nb = lane < 13 ? lane : (lane < 26 ? lane + 1 : 13);
      const int dx = nb % 3 - 1, dy = (nb / 3) % 3 - 1, dz = nb / 9 - 1;
      const int jx = c[0] + dx, jy = c[1] + dy, jz = c[2] + dz;
      if (jx >= 0 && jy >= 0 && jz >= 0 && jx < n && jy < n && jz < n) {
        const int64_t J = morton_encode(jx, jy, jz, depth);
        beg = soff[J];
        len = soff[J + 1] - beg;
      }
      s_beg[lane] = beg;
      s_len[lane] = len;
      s_sh[lane][0] = dx * two_l;
      s_sh[lane][1] = dy * two_l;
      s_sh[lane][2] = dz * two_l;
    }
    // exclusive scan of the lengths of segments 0..25; the leaf itself
    // starts at the next even position
    int x = lane < 26 ? len : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const int other = __shfl_sync(0xffffffffu, x, 25);
    const int own = __shfl_sync(0xffffffffu, len, 26);
    if (lane < 26) s_pos[lane] = x - len;
    if (lane == 26) s_pos[26] = (other + 1) & ~1;
    if (lane == 27) s_pos[27] = ((other + 1) & ~1) + own;
  }
  __syncthreads();
  const int n_real_other = s_pos[25] + s_len[25];
  const int n_other = s_pos[26], n_log = s_pos[27];
  const int beg = toff[b], end = toff[b + 1];
  int staged_c0 = -1;
  for (int t0 = beg, P = 0; t0 < end; t0 += P) {
    const int m = end - t0;
    P = m >= NF_THREADS ? NF_THREADS : (m > 32 ? 32 : m);
    const int S = min(NF_THREADS / P, NF_MAXS);
    const int ti = tid % P, si = tid / P;
    const bool act = si < S;
    const int p = t0 + (act ? ti : 0);
    const float x0 = tlx[p], x1 = tly[p], x2 = tlz[p];
    const float2 NX = make_float2(-x0, -x0), NY = make_float2(-x1, -x1), NZ = make_float2(-x2, -x2);
    const int js = exclude_self ? n_other + (p - beg) : -1;  // logical position of the self pair
    float th0 = 0.f, tc0 = 0.f, th1 = 0.f, tc1 = 0.f;      // tier 0: FP32 Kahan totals per half
    double td = 0.0;                                       // ACC: FP64 total
    for (int c0 = 0; c0 < n_log; c0 += NF_SRC) {
      const int cn = min(NF_SRC, n_log - c0);
      const int np = (cn + 1) >> 1;
      if (staged_c0 != c0) {
        __syncthreads();
        // thread tid stages logical positions c0 + tid, c0 + tid + 128, ...
        // of the chunk; the segment of a position is the last one starting
        // at or before it (a binary search over the 26 starts), so the
        // global loads of all of a thread's sources are independent and in
        // flight together
#pragma unroll 4
        for (int lp = tid; lp < cn; lp += NF_THREADS) {
          const int pos = c0 + lp;
          int sg = 26;
          if (pos < n_other) {
            if (pos >= n_real_other) continue;  // the pad before the leaf itself
            sg = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
              if (sg + step < 26 && s_pos[sg + step] <= pos) sg += step;
          }
          const int sj = s_beg[sg] + (pos - s_pos[sg]);
          float* e = reinterpret_cast<float*>(&s_pair[2 * (lp >> 1)]) + (lp & 1);
          e[0] = slx[sj] + s_sh[sg][0];
          e[2] = sly[sj] + s_sh[sg][1];
          e[4] = slz[sj] + s_sh[sg][2];
          e[6] = sig[sj];
        }
        // pads at an odd end of the other leaves and of the chunk
        if (tid < 2) {
          const int g = tid == 0 ? n_real_other : c0 + cn;
          if ((g & 1) && g >= c0 && g < c0 + 2 * np && (tid == 1 || g < n_other)) {
            float* e = reinterpret_cast<float*>(&s_pair[2 * ((g - c0) >> 1)]) + 1;
            e[0] = NF_FAR;
            e[2] = NF_FAR;
            e[4] = NF_FAR;
            e[6] = 0.f;
          }
        }
        __syncthreads();
        staged_c0 = c0;
      }
      if (act) {
        const int L = (np + S - 1) / S;
        const int qb = min(np, si * L), qe = min(np, qb + L);
        const int qown = max(0, n_other - c0) >> 1;  // first pair of the leaf itself
        const int qs = js - c0 >= 0 && js - c0 < cn ? (js - c0) >> 1 : -1, hs = (js - c0) & 1;
        const int qm = qs < 0 ? qe : max(qb, min(qe, qown));
        float sl = 0.f, sh = 0.f, cl = 0.f, ch = 0.f;
        const float4* sp4 = reinterpret_cast<const float4*>(s_pair);
        nf_span<ACC, false>(sp4, qb, qm, -1, 0, NX, NY, NZ, sl, sh, cl, ch);
        nf_span<ACC, true>(sp4, qm, qe, qs, hs, NX, NY, NZ, sl, sh, cl, ch);
        if (ACC) {
          td += ((double)sl - (double)cl) + ((double)sh - (double)ch);
        } else {
          kahan_add(th0, tc0, sl);
          kahan_add(th1, tc1, sh);
        }
      }
    }
    if (!ACC) td = ((double)th0 - (double)tc0) + ((double)th1 - (double)tc1);
    __syncthreads();
    s_red[tid] = act ? td : 0.0;
    __syncthreads();
    if (tid < P) {
      double s = 0.0;
      for (int k = 0; k < S; ++k) s += s_red[ti + k * P];
      fnear[p] = s;
    }
  }
}

// ------------------------------------- P2M and L2P of 1/r, one RHS ------
// Steps 1 and 7 for K = 1/r with one right-hand side, with the distances
// computed two at a time (the packed f32x2 builtins) over pairs of interpolation
// points: one warp per leaf, PT_WARPS leaves per CTA, the level's points
// x_l^{I_0} (= y_l^{J_0}) staged once per CTA as SoA pairs
//   s_xy[q] = (x_2q, x_2q+1 | y_2q, y_2q+1),  s_z[q] = (z_2q, z_2q+1),
// with a far-away pad (and a zero coefficient) past d.  No CTA barrier after
// the staging: each warp owns its leaf.
constexpr int PT_WARPS = 8;
constexpr int PT_MAXQ = 128;  // pairs: dp <= 256

__device__ __forceinline__ void pt_stage_x(const float* __restrict__ X, int d, int nq, float4* s_xy,
                                           float2* s_z) {
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const int a = 2 * q, b = 2 * q + 1;
    const float x0 = a < d ? X[3 * a] : NF_FAR, y0 = a < d ? X[3 * a + 1] : NF_FAR, z0 = a < d ? X[3 * a + 2] : NF_FAR;
    const float x1 = b < d ? X[3 * b] : NF_FAR, y1 = b < d ? X[3 * b + 1] : NF_FAR, z1 = b < d ? X[3 * b + 2] : NF_FAR;
    s_xy[q] = make_float4(x0, x1, y0, y1);
    s_z[q] = make_float2(z0, z1);
  }
}

// (1/r_lo, 1/r_hi) of a packed r^2, with a Newton step when ACC
template <bool ACC>
__device__ __forceinline__ float2 pt_rsqrt2(float2 r2) {
  float yl = rsqrt_approx(r2.x), yh = rsqrt_approx(r2.y);
  if (ACC) {
    yl = yl * fmaf(-0.5f * r2.x, yl * yl, 1.5f);
    yh = yh * fmaf(-0.5f * r2.y, yh * yh, 1.5f);
  }
  return make_float2(yl, yh);
}

// acc (+)= k sigma on each half with scalar FMAs: the two rsqrt results stay
// in registers of their own (joining them into a pair for one packed FMA
// measured slower in the near field)
__device__ __forceinline__ void pt_fma_halves(float2& acc, float2 k, float2 sg) {
  acc.x = fmaf(k.x, sg.x, acc.x);
  acc.y = fmaf(k.y, sg.y, acc.y);
}

// |a - b|^2 of two packed points, b given negated
__device__ __forceinline__ float2 pt_r2(float2 ax, float2 ay, float2 az, float2 nbx, float2 nby, float2 nbz) {
  const float2 dx = __fadd2_rn(ax, nbx);
  const float2 dy = __fadd2_rn(ay, nby);
  const float2 dz = __fadd2_rn(az, nbz);
  float2 r2 = __fmul2_rn(dx, dx);
  r2 = __ffma2_rn(dy, dy, r2);
  return __ffma2_rn(dz, dz, r2);
}

// Step 1: W_m = sum_j sigma_j / |x_m - y_j|.  Lane owns the coefficient
// pairs q = lane + 32 i (at most PT_MAXQ / 32 of them, in registers); the
// leaf's points pass through shared memory 32 at a time, each as two
// broadcast 16-byte words (-x, -x | -y, -y) and (-z, -z | sigma, sigma).
template <bool ACC>
__global__ void __launch_bounds__(32 * PT_WARPS, 4)
k_p2m32x(const int32_t* __restrict__ off, int64_t nleaf, const float* __restrict__ lx,
         const float* __restrict__ ly, const float* __restrict__ lz, const float* __restrict__ sig,
         const float* __restrict__ X, int d, int dp, float* __restrict__ W,
         __nv_bfloat16* __restrict__ planes, int grid_level, const double* __restrict__ sig64,
         const int32_t* __restrict__ perm) {
  constexpr int NI = PT_MAXQ / 32;
  __shared__ float4 s_xy[PT_MAXQ];
  __shared__ float2 s_z[PT_MAXQ];
  __shared__ float4 s_pt[PT_WARPS][32][2];
  const int nq = (d + 1) >> 1, nqi = (nq + 31) >> 5;
  pt_stage_x(X, d, nq, s_xy, s_z);
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.x * PT_WARPS + w;
  if (b >= nleaf) return;
  float2 ax[NI], ay[NI], az[NI], acc[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int q = lane + 32 * i;
    acc[i] = make_float2(0.f, 0.f);
    if (q < nq) {
      const float4 e = s_xy[q];
      ax[i] = make_float2(e.x, e.y);
      ay[i] = make_float2(e.z, e.w);
      az[i] = s_z[q];
    } else {
      ax[i] = ay[i] = az[i] = make_float2(NF_FAR, NF_FAR);
    }
  }
  const int beg = off[b], end = off[b + 1];
  for (int j0 = beg; j0 < end; j0 += 32) {
    const int j = j0 + lane;
    __syncwarp();
    if (j < end) {
      // sigma in sorted order, or (sig64) read through the permutation from
      // the caller's FP64 array and rounded as the gather rounds it
      const float s = sig64 ? (float)sig64[perm[j]] : sig[j];
      const float px = -lx[j], py = -ly[j], pz = -lz[j];
      s_pt[w][lane][0] = make_float4(px, px, py, py);
      s_pt[w][lane][1] = make_float4(pz, pz, s, s);
    }
    __syncwarp();
    const int cnt = min(32, end - j0);
    // two points per step: their distances and 1/r are independent, only
    // the accumulation is sequential (in point order)
    int t = 0;
    for (; t + 1 < cnt; t += 2) {
      const float4 p0 = s_pt[w][t][0], p1 = s_pt[w][t][1];
      const float4 o0 = s_pt[w][t + 1][0], o1 = s_pt[w][t + 1][1];
#pragma unroll
      for (int i = 0; i < NI; ++i)
        if (i < nqi) {  // warp-uniform; lanes past nq work on the far pad
          const float2 kp = pt_rsqrt2<ACC>(pt_r2(ax[i], ay[i], az[i], make_float2(p0.x, p0.y),
                                                 make_float2(p0.z, p0.w), make_float2(p1.x, p1.y)));
          const float2 ko = pt_rsqrt2<ACC>(pt_r2(ax[i], ay[i], az[i], make_float2(o0.x, o0.y),
                                                 make_float2(o0.z, o0.w), make_float2(o1.x, o1.y)));
          pt_fma_halves(acc[i], kp, make_float2(p1.z, p1.w));
          pt_fma_halves(acc[i], ko, make_float2(o1.z, o1.w));
        }
    }
    if (t < cnt) {
      const float4 p0 = s_pt[w][t][0], p1 = s_pt[w][t][1];
#pragma unroll
      for (int i = 0; i < NI; ++i)
        if (i < nqi)
          pt_fma_halves(acc[i],
                        pt_rsqrt2<ACC>(pt_r2(ax[i], ay[i], az[i], make_float2(p0.x, p0.y),
                                             make_float2(p0.z, p0.w), make_float2(p1.x, p1.y))),
                        make_float2(p1.z, p1.w));
    }
  }
  float* row = W + b * dp;
  // step 3's BF16 hi/lo planes of the leaf level too, when given (the same
  // split as k_planes, at the plane row of the box)
  const int64_t prow = planes ? plane_row(b, grid_level, 1) * dp : 0;
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int q = lane + 32 * i;
    if (2 * q < dp) {
      float lo = acc[i].x, hi = acc[i].y;
      if (2 * q >= d) lo = 0.f;
      if (2 * q + 1 >= d) hi = 0.f;
      *reinterpret_cast<float2*>(row + 2 * q) = make_float2(lo, hi);
      if (planes) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        const float2 fh = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(lo - fh.x, hi - fh.y);
        *reinterpret_cast<__nv_bfloat162*>(planes + prow + 2 * q) = h;
        *reinterpret_cast<__nv_bfloat162*>(planes + nleaf * dp + prow + 2 * q) = l;
      }
    }
  }
}

// Step 7 (the far field alone): f_F(x_i) = sum_l lhat_l / |x_i - x_l|.  The
// warp stages the leaf's coefficient pairs beside the z pairs,
// s_zl[q] = (z_2q, z_2q+1 | lhat_2q, lhat_2q+1); lanes = (point, slice):
// 32 points per pass while that many remain, then the rest with
// S = 32 / rest slices of the pairs, added by shuffles.
template <bool ACC>
__global__ void __launch_bounds__(32 * PT_WARPS)
k_l2p32x(const int32_t* __restrict__ leaves, int64_t nl, const int32_t* __restrict__ off,
         const float* __restrict__ lx, const float* __restrict__ ly, const float* __restrict__ lz,
         const float* __restrict__ X, int d, int dp, const float* __restrict__ lh, double* __restrict__ ffar) {
  __shared__ float4 s_xy[PT_MAXQ];
  __shared__ float2 s_z[PT_MAXQ];
  __shared__ float4 s_zl[PT_WARPS][PT_MAXQ];
  const int nq = (d + 1) >> 1;
  pt_stage_x(X, d, nq, s_xy, s_z);
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * PT_WARPS + w;
  if (i >= nl) return;
  const int b = leaves[i];
  const float* lrow = lh + (int64_t)b * dp;
  for (int q = lane; q < nq; q += 32) {
    const float2 c = *reinterpret_cast<const float2*>(lrow + 2 * q);
    const float2 z = s_z[q];
    s_zl[w][q] = make_float4(z.x, z.y, c.x, 2 * q + 1 < d ? c.y : 0.f);
  }
  __syncwarp();
  const int beg = off[b], end = off[b + 1];
  for (int t0 = beg; t0 < end; t0 += 32) {
    const int P = min(32, end - t0), S = 32 / P;
    const int ti = lane % P, si = lane / P;
    const int p = t0 + ti;
    float s = 0.f;
    if (si < S) {
      const float px = -lx[p], py = -ly[p], pz = -lz[p];
      const float2 PX = make_float2(px, px), PY = make_float2(py, py), PZ = make_float2(pz, pz);
      const int L = (nq + S - 1) / S;
      const int qb = min(nq, si * L), qe = min(nq, qb + L);
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int q = qb; q < qe; ++q) {
        const float4 e = s_xy[q], f = s_zl[w][q];
        const float2 k = pt_rsqrt2<ACC>(
            pt_r2(make_float2(e.x, e.y), make_float2(e.z, e.w), make_float2(f.x, f.y), PX, PY, PZ));
        pt_fma_halves(acc, k, make_float2(f.z, f.w));
      }
      s = acc.x + acc.y;
    }
    // slices si = 1..S-1 of point ti sit at lanes ti + P si
    for (int k = 1; k < S; ++k) {
      const float o = __shfl_sync(0xffffffffu, s, min(31, lane + P * k));
      if (lane < P) s += o;
    }
    if (lane < P) ffar[p] = (double)s;
  }
}

// --------------------------------------------------- operator images ----
// K^delta (kdT[slot][l][m'] FP64) -> two planes in the swizzled image used
// by the tensor-core M2L: byte offset of row n, 16-byte unit j inside the
// 128-byte chunk: (n / 8) * 1024 + (n % 8) * 128 + ((j ^ (n % 8)) * 16).
// fmt: PlaneFmt; FP16 rows are scaled by kscale[m'] (a power of two).
__global__ void k_build_img(const double* __restrict__ kdT, int d, int dp, int fmt,
                            const float* __restrict__ kscale, unsigned char* __restrict__ img) {
  const bool tf32 = fmt == kPlaneTF32;
  const int esz = tf32 ? 4 : 2;
  const int E = 128 / esz;  // elements per chunk
  const int nchunk = dp / E;
  const int slot = blockIdx.y;
  const int64_t units = (int64_t)nchunk * dp * 8;  // (chunk, row, 16-byte unit)
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < units;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(u / (dp * 8));
    const int rem = (int)(u - (int64_t)c * dp * 8);
    const int nrow = rem / 8, j = rem % 8;
    const int per = 16 / esz;
    unsigned char* base0 = img + (((size_t)slot * nchunk + c) * 2 + 0) * (size_t)dp * 128;
    unsigned char* base1 = base0 + (size_t)dp * 128;
    const size_t off = (size_t)(nrow / 8) * 1024 + (nrow % 8) * 128 + ((j ^ (nrow % 8)) * 16);
    for (int e = 0; e < per; ++e) {
      const int l = c * E + j * per + e;
      const double v = (l < d && nrow < d) ? kdT[((int64_t)slot * d + l) * d + nrow] : 0.0;
      if (fmt == kPlaneF16) {
        const double vs = v * (double)kscale[nrow];
        const __half hi = __double2half(vs);
        const __half lo = __double2half(vs - (double)__half2float(hi));
        ((__half*)(base0 + off))[e] = hi;
        ((__half*)(base1 + off))[e] = lo;
      } else if (tf32) {
        const float hi = tf32_rn((float)v);
        const float lo = tf32_rn((float)(v - (double)hi));
        ((float*)(base0 + off))[e] = hi;
        ((float*)(base1 + off))[e] = lo;
      } else {
        const __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
        const __nv_bfloat16 lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
        ((__nv_bfloat16*)(base0 + off))[e] = hi;
        ((__nv_bfloat16*)(base1 + off))[e] = lo;
      }
    }
  }
}

// Power-of-two scale of row m' of the FP16 operator image: its largest
// entry over the 316 far offsets and every l lands in [2^14, 2^15).  One
// block per row.
__global__ void k_kd_rowscale(const double* __restrict__ kdT, int d, int dp, float* __restrict__ kscale) {
  const int row = blockIdx.x;
  __shared__ float red[256];
  float m = 0.f;
  if (row < d)
    for (int64_t t = threadIdx.x; t < (int64_t)kNumSlots * d; t += blockDim.x) {
      const int slot = (int)(t / d), l = (int)(t - (int64_t)slot * d);
      const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
      if (max(abs(dx), max(abs(dy), abs(dz))) < 2) continue;  // near offsets: not M2L
      m = fmaxf(m, (float)fabs(kdT[((int64_t)slot * d + l) * d + row]));
    }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) kscale[row] = f16_plane_scale(red[0]);
}

// wmax[k] = bits of max |W| over level k (levels lo..hi, one launch; wmax
// zeroed before): non-negative floats order like their bit patterns.
struct AbsMaxBatch {
  const float* w[kMaxLevel + 1];
  int64_t n[kMaxLevel + 1];
  int lo = 0, hi = -1;
};
__global__ void __launch_bounds__(256) k_absmax(const __grid_constant__ AbsMaxBatch b, uint32_t* __restrict__ wmax) {
  for (int k = b.lo; k <= b.hi; ++k) {
    float m = 0.f;
    const int64_t n4 = b.n[k] / 4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
      const float4 v = reinterpret_cast<const float4*>(b.w[k])[i];
      m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(&wmax[k], __float_as_uint(m));
  }
}

// planes -> FP64 [row][d] (debug export of What)
// The M2L operand planes of W (hi and lo parts, BF16 or TF32) at every
// level in one launch; entries j >= d are zero.  One thread per 4
// consecutive entries (dp is a multiple of 64, so a quad never straddles a
// row).
struct PlaneLevel {
  const float* in;  // [rows][dp]
  void* out;        // [2][rows][dp] at plane_row order
  int64_t rows, q0; // q0: first quad of this level in the launch
  int d, dp, grid_level, R, level;
};
struct PlaneBatch {
  PlaneLevel lv[kMaxLevel + 1];
  int nlev = 0;
  int64_t nq = 0;
  const uint32_t* wmax = nullptr;  // FP16: bits of max |W| per level
};

// FMT: PlaneFmt.  FP16 planes hold W s_W = hi + lo with the level's scale
// s_W = f16_plane_scale(max |W|).
template <int FMT>
__global__ void __launch_bounds__(256) k_planes(const __grid_constant__ PlaneBatch b) {
  constexpr bool TF32 = FMT == kPlaneTF32;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < b.nq;
       q += (int64_t)gridDim.x * blockDim.x) {
    int li = 0;
    while (li + 1 < b.nlev && q >= b.lv[li + 1].q0) ++li;
    const PlaneLevel& L = b.lv[li];
    const int64_t e = (q - L.q0) * 4;
    const int64_t v = e / L.dp;
    const int j = (int)(e - v * L.dp);
    float4 x = *reinterpret_cast<const float4*>(L.in + e);
    if (j + 4 > L.d) {
      if (j + 0 >= L.d) x.x = 0.f;
      if (j + 1 >= L.d) x.y = 0.f;
      if (j + 2 >= L.d) x.z = 0.f;
      if (j + 3 >= L.d) x.w = 0.f;
    }
    const int64_t o = plane_row(v, L.grid_level, L.R) * L.dp + j;
    const int64_t lo_off = L.rows * L.dp;
    if (TF32) {
      const float4 h = make_float4(tf32_rn(x.x), tf32_rn(x.y), tf32_rn(x.z), tf32_rn(x.w));
      const float4 l = make_float4(tf32_rn(x.x - h.x), tf32_rn(x.y - h.y), tf32_rn(x.z - h.z), tf32_rn(x.w - h.w));
      float* p = (float*)L.out;
      *reinterpret_cast<float4*>(p + o) = h;
      *reinterpret_cast<float4*>(p + lo_off + o) = l;
    } else if (FMT == kPlaneF16) {
      const float sw = f16_plane_scale(__uint_as_float(b.wmax[L.level]));
      x.x *= sw; x.y *= sw; x.z *= sw; x.w *= sw;  // exact: a power of two
      const __half2 h01 = __floats2half2_rn(x.x, x.y), h23 = __floats2half2_rn(x.z, x.w);
      const float2 f01 = __half22float2(h01), f23 = __half22float2(h23);
      const __half2 l01 = __floats2half2_rn(x.x - f01.x, x.y - f01.y);
      const __half2 l23 = __floats2half2_rn(x.z - f23.x, x.w - f23.y);
      __half* p = (__half*)L.out;
      uint2 hv, lv;
      hv.x = *reinterpret_cast<const uint32_t*>(&h01); hv.y = *reinterpret_cast<const uint32_t*>(&h23);
      lv.x = *reinterpret_cast<const uint32_t*>(&l01); lv.y = *reinterpret_cast<const uint32_t*>(&l23);
      *reinterpret_cast<uint2*>(p + o) = hv;
      *reinterpret_cast<uint2*>(p + lo_off + o) = lv;
    } else {
      const __nv_bfloat162 h01 = __floats2bfloat162_rn(x.x, x.y), h23 = __floats2bfloat162_rn(x.z, x.w);
      const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
      const __nv_bfloat162 l01 = __floats2bfloat162_rn(x.x - f01.x, x.y - f01.y);
      const __nv_bfloat162 l23 = __floats2bfloat162_rn(x.z - f23.x, x.w - f23.y);
      __nv_bfloat16* p = (__nv_bfloat16*)L.out;
      uint2 hv, lv;
      hv.x = *reinterpret_cast<const uint32_t*>(&h01); hv.y = *reinterpret_cast<const uint32_t*>(&h23);
      lv.x = *reinterpret_cast<const uint32_t*>(&l01); lv.y = *reinterpret_cast<const uint32_t*>(&l23);
      *reinterpret_cast<uint2*>(p + o) = hv;
      *reinterpret_cast<uint2*>(p + lo_off + o) = lv;
    }
  }
}

__global__ void k_f32_to_f64(const float* __restrict__ a, int64_t nvec, int d, int dp,
                             double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nvec * d;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t / d;
    const int j = (int)(t - v * d);
    out[t] = (double)a[v * dp + j];
  }
}

unsigned grid_for(int64_t n, int tpb, unsigned cap = 8192) {
  int64_t g = (n + tpb - 1) / tpb;
  if (g < 1) g = 1;
  return (unsigned)(g > cap ? cap : g);
}

// FP32 copy of the folded M2L operator for the SIMT M2L of tier 2:
// kd32[slot][l][m'] = (K^delta Delta)_{m' l} for l < d, m' < d, zero for
// d <= m' < dp (row stride dp).
__global__ void k_build_kd32(const double* __restrict__ kdT, int d, int dp, float* __restrict__ kd32) {
  const int64_t slot = blockIdx.y;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)d * dp;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(t / dp), mp = (int)(t - (int64_t)l * dp);
    kd32[(slot * d + l) * dp + mp] = mp < d ? (float)kdT[(slot * d + l) * d + mp] : 0.f;
  }
}

// Step 4 of tier 2 on the SIMT pipes: g^I = sum_J (K^delta Delta) W^J with
// FP32 products summed in FP32 over the d terms of one offset, and the
// offsets added with compensated (Kahan) FP32 sums (the plain FP32
// accumulation of the whole sum, about 30,000 terms, is what limits the
// tensor-core tiers; FP64 adds would cost 1/64 of the FP32 rate here).
//
// A block computes 64 target boxes x 64 rows m': the boxes are 64
// consecutive parents of one parity class (a 4x4x4 block of the class grid,
// fewer at level 2), which share the 189 candidate offsets.  Per offset and
// per chunk of 16 terms l, the 64 source rows (gathered, zero outside the
// cube) and 16 x 64 operator entries are staged in shared memory; each of
// the 256 threads accumulates a 4 x 4 block (4 boxes x 4 rows).
constexpr int M2S_BOX = 64, M2S_ROW = 64, M2S_L = 16, M2S_THREADS = 256;

__global__ void __launch_bounds__(M2S_THREADS, 3)
k_m2l32s(int level, int d, int dp, int R, const float* __restrict__ kd32, const int* __restrict__ slot_lists,
         const float* __restrict__ W, float* __restrict__ g, int groups, float* __restrict__ part,
         int64_t part_stride) {
  __shared__ __align__(16) float sW[M2S_L][M2S_BOX];  // [l][box]
  __shared__ __align__(16) float sT[M2S_L][M2S_ROW];  // [l][m']
  __shared__ int64_t s_src[M2S_BOX];                   // source row offset, -1 outside the cube
  __shared__ int s_c[M2S_BOX][3];
  const int tid = threadIdx.x;
  const int r = blockIdx.z;
  const int oct = blockIdx.x & 7;
  const int grp = (int)((blockIdx.x >> 3) % groups);  // offsets [grp, grp+1) * 189 / groups
  const int64_t per_class = (int64_t)1 << (3 * (level - 1));
  const int nb = per_class < M2S_BOX ? (int)per_class : M2S_BOX;  // boxes of this block
  const int64_t p0 = ((blockIdx.x >> 3) / groups) * (int64_t)M2S_BOX;
  float* const dst = groups > 1 ? part + grp * part_stride : g;
  const int m0 = blockIdx.y * M2S_ROW;
  const int n = 1 << level;
  if (tid < M2S_BOX) {
    int c[3] = {0, 0, 0};
    if (tid < nb) morton_decode(8 * (p0 + tid) + oct, level, c);
    s_c[tid][0] = c[0];
    s_c[tid][1] = c[1];
    s_c[tid][2] = c[2];
  }
  // this thread's 4 rows and 4 boxes; the rows come from the warp index, so
  // a warp whose 8 rows all lie at or beyond d (the padding of the last row
  // tile) skips the sums
  const int tm = (tid >> 4) * 4, tb = (tid & 15) * 4;
  const bool rows_live = m0 + (tid >> 5) * 8 < d;
  float acc[4][4], cmp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = cmp[i][j] = 0.f;
  const int* lst = slot_lists + oct * kListLen;
  // staging roles: box lb, 4 consecutive terms 4 lq of the chunk; operator row
  // ll, 4 consecutive m' from 4 lm
  const int lb = tid >> 2, lq = (tid & 3) * 4;
  const int ll = tid >> 4, lm = (tid & 15) * 4;
  const int s_end = (grp + 1) * kListLen / groups;
  for (int s = grp * kListLen / groups; s < s_end; ++s) {
    const int slot = lst[s];
    const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
    __syncthreads();  // s_src and the tiles of the previous offset are free
    if (tid < M2S_BOX) {
      const int jx = s_c[tid][0] + dx, jy = s_c[tid][1] + dy, jz = s_c[tid][2] + dz;
      const bool ok = tid < nb && jx >= 0 && jy >= 0 && jz >= 0 && jx < n && jy < n && jz < n;
      s_src[tid] = ok ? (morton_encode(jx, jy, jz, level) * R + r) * dp : -1;
    }
    __syncthreads();
    const float* K = kd32 + (int64_t)slot * d * dp;
    float part[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[i][j] = 0.f;
    // source coefficients (rows of W are dp long, 16-byte aligned, zero
    // beyond d) and operator entries (rows l >= d do not exist) of the chunk
    // at l0; the next chunk is loaded while the current one is summed
    const int64_t so = s_src[lb];
    auto load_w = [&](int l0) {
      return (so >= 0 && l0 + lq < dp) ? *reinterpret_cast<const float4*>(W + so + l0 + lq)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto load_k = [&](int l0) {
      return (l0 + ll < d && m0 + lm < dp)
                 ? __ldg(reinterpret_cast<const float4*>(K + (int64_t)(l0 + ll) * dp + m0 + lm))
                 : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    float4 wv = load_w(0), kv = load_k(0);
    for (int l0 = 0; l0 < d; l0 += M2S_L) {
      sW[lq + 0][lb] = wv.x;
      sW[lq + 1][lb] = wv.y;
      sW[lq + 2][lb] = wv.z;
      sW[lq + 3][lb] = wv.w;
      *reinterpret_cast<float4*>(&sT[ll][lm]) = kv;
      __syncthreads();
      if (l0 + M2S_L < d) {
        wv = load_w(l0 + M2S_L);
        kv = load_k(l0 + M2S_L);
      }
#pragma unroll
      for (int u = 0; u < M2S_L && rows_live; ++u) {
        const float4 a4 = *reinterpret_cast<const float4*>(&sW[u][tb]);
        const float4 b4 = *reinterpret_cast<const float4*>(&sT[u][tm]);
        const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) part[i][j] = fmaf(av[i], bv[j], part[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) kahan_add(acc[i][j], cmp[i][j], part[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (tb + i >= nb) break;
    const int64_t I = 8 * (p0 + tb + i) + oct;
    float* out = dst + (I * R + r) * dp + m0 + tm;
    if (m0 + tm < dp)
      *reinterpret_cast<float4*>(out) = make_float4(acc[i][0] - cmp[i][0], acc[i][1] - cmp[i][1],
                                                    acc[i][2] - cmp[i][2], acc[i][3] - cmp[i][3]);
  }
}

}  // namespace

eifmm_status build_kd_image(Ops* ops, int fmt, cudaStream_t s) {
  const bool tf32 = fmt == kPlaneTF32;
  for (int k = 2; k <= ops->depth; ++k) {
    LevelOps& v = ops->lv[k];
    if (v.kd_img_fmt == fmt) continue;
    dfree(v.kd_img);
    v.kd_img = nullptr;
    v.kd_img_fmt = -1;
    // the SIMT path serves larger levels (FP16: the drains hold dp <= 256)
    if (v.dp > (fmt == kPlaneF16 ? 256 : kMaxDpTc)) continue;
    if (fmt == kPlaneF16 && !v.kscale) {
      EIFMM_TRY(dalloc(&v.kscale, (size_t)v.dp));
      k_kd_rowscale<<<v.dp, 256, 0, s>>>(v.kdT, v.d, v.dp, v.kscale);
      EIFMM_CHECK_LAUNCH();
    }
    const size_t bytes = (size_t)kNumSlots * 2 * v.dp * (size_t)(v.dp * (tf32 ? 4 : 2));
    EIFMM_TRY(dmalloc(&v.kd_img, bytes));
    const int nchunk = v.dp * (tf32 ? 4 : 2) / 128;
    k_build_img<<<dim3(grid_for((int64_t)nchunk * v.dp * 8, 256, 64), kNumSlots), 256, 0, s>>>(
        v.kdT, v.d, v.dp, fmt, v.kscale, (unsigned char*)v.kd_img);
    EIFMM_CHECK_LAUNCH();
    v.kd_img_fmt = fmt;
  }
  // tier 1 falls back to the SIMT M2L where it has no FP16 tile (dp above
  // 256, or a right-hand-side count without a tile shape)
  if (fmt == kPlaneF16) EIFMM_TRY(build_kd32(ops, s));
  EIFMM_CUDA(cudaStreamSynchronize(s));
  return EIFMM_OK;
}

eifmm_status build_kd32(Ops* ops, cudaStream_t s) {
  for (int k = 2; k <= ops->depth; ++k) {
    LevelOps& v = ops->lv[k];
    if (v.kd32) continue;
    EIFMM_TRY(dalloc(&v.kd32, (size_t)kNumSlots * v.d * v.dp));
    k_build_kd32<<<dim3(grid_for((int64_t)v.d * v.dp, 256, 64), kNumSlots), 256, 0, s>>>(v.kdT, v.d, v.dp,
                                                                                        v.kd32);
    EIFMM_CHECK_LAUNCH();
  }
  EIFMM_CUDA(cudaStreamSynchronize(s));
  return EIFMM_OK;
}

// Step 4 of tier 2 at level k (SIMT, FP64 across offsets).
static int sm_count();

// g = the offset-group partials of the SIMT M2L added in group order with
// a compensated FP32 sum.
__global__ void k_sum_groups(const float* __restrict__ part, int groups, int64_t n, int64_t stride,
                             float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f, c = 0.f;
    for (int q = 0; q < groups; ++q) kahan_add(s, c, part[q * stride + i]);
    out[i] = s - c;
  }
}

static eifmm_status launch_m2l_simt(const Tree* t, const Ops* ops, int k, int R, cudaStream_t s) {
  const LevelOps& v = ops->lv[k];
  if (!v.kd32) {
    set_error("eifmm_evaluate: FP32 M2L operator of tier 2 missing");
    return EIFMM_EUNSUPPORTED;
  }
  const Workspace& ws = t->ws;
  const int64_t per_class = nboxes(k) / 8;
  const int64_t tiles = (per_class + M2S_BOX - 1) / M2S_BOX;
  // every block walks its offsets in sequence, so a level with few blocks
  // splits the offsets into groups (two waves of blocks at least; the leaf
  // level keeps one group)
  const int64_t ctas = tiles * 8 * (v.dp / M2S_ROW) * R;
  const int64_t rows_dp = nboxes(k) * R * v.dp;
  int G = 1;
  if (k < t->depth)
    while (G < 16 && ctas * G < 2 * sm_count() && (size_t)(2 * G) * rows_dp <= ws.m2l_part_cap) G *= 2;
  k_m2l32s<<<dim3((unsigned)(tiles * 8 * G), (unsigned)(v.dp / M2S_ROW), (unsigned)R), M2S_THREADS, 0, s>>>(
      k, v.d, v.dp, R, v.kd32, ops->d_slot_lists, ws.W32[k], ws.g32[k], G, ws.m2l_part, rows_dp);
  EIFMM_CHECK_LAUNCH();
  if (G > 1) {
    k_sum_groups<<<grid_for(rows_dp, 256, 4096), 256, 0, s>>>(ws.m2l_part, G, rows_dp, rows_dp, ws.g32[k]);
    EIFMM_CHECK_LAUNCH();
  }
  return EIFMM_OK;
}

eifmm_status alloc_mixed_workspace(Tree* t, const Ops* ops, int R) {
  Workspace& ws = t->ws;
  const int kap = t->depth;
  if (R == 1 && t->same && t->exclude_self && t->tgt.n > 0 && !ws.gsym)
    EIFMM_TRY(dalloc(&ws.gsym, (size_t)kSymSlots * t->tgt.n));
  for (int k = 2; k <= kap; ++k) {
    const int dp = ops->lv[k].dp;
    const size_t n = (size_t)nboxes(k) * R * dp;
    EIFMM_TRY(dalloc(&ws.W32[k], n));
    EIFMM_TRY(dalloc(&ws.g32[k], n));
    if (k == 2) ws.l32[k] = ws.g32[k];
    else EIFMM_TRY(dalloc(&ws.l32[k], n));
    EIFMM_TRY(dmalloc(&ws.wa[k], 2 * n * 4));
    // TMA-tiled M2L when the rhs count has a tile shape: planes on the
    // per-class grid, one tensor map per plane (tier 0: BF16, tier 1: FP16)
    int bx, by, bz;
    ws.wa_grid[k] = false;
    ws.wa_t256[k] = false;
    const int fmt = ops->tier == 1 ? kPlaneF16 : kPlaneBF16;
    if (ops->tier <= 1 && ops->lv[k].dp <= kMaxDpTc && m2l_tma_block(R, &bx, &by, &bz)) {
      const size_t plane = n * 2;
      EIFMM_TRY(make_plane_map(ws.tmap[k][0], ws.wa[k], k, R, dp, fmt));
      EIFMM_TRY(make_plane_map(ws.tmap[k][1], (char*)ws.wa[k] + plane, k, R, dp, fmt));
      ws.wa_grid[k] = true;
      if (fmt == kPlaneBF16 && dp == 128 && m2l_t256_block(R, &bx, &by, &bz)) {
        EIFMM_TRY(make_plane_map(ws.tmap2[k][0], ws.wa[k], k, R, dp, fmt, 256));
        EIFMM_TRY(make_plane_map(ws.tmap2[k][1], (char*)ws.wa[k] + plane, k, R, dp, fmt, 256));
        ws.wa_t256[k] = true;
      }
    }
  }
  EIFMM_TRY(dalloc(&ws.lh32, (size_t)nboxes(kap) * R * ops->lv[kap].dp));
  if (!ws.blas_ws) EIFMM_TRY(dmalloc(&ws.blas_ws, kXferBlasWorkspace));
  {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    size_t need = 0, need_leaf = 0;
    for (int k = 2; k <= kap; ++k) {
      const int64_t rows = nboxes(k) * R;
      const int64_t tiles = (nboxes(k) / 8 * R + 127) / 128;
      size_t& nd = k == kap ? need_leaf : need;
      const int G = m2l_tc_groups(tiles * 8, nsm, ops->lv[k].dp);
      if (G > 1) nd = std::max(nd, (size_t)G * rows * ops->lv[k].dp);
      const int G2 = m2l_t256_groups(m2l_t256_ctas(k, R), nsm);
      if (G2 > 1) nd = std::max(nd, (size_t)G2 * rows * ops->lv[k].dp);
      const int G3 = ops->tier == 1 ? m2l_h16_groups(m2l_tma_ctas(k, R), nsm) : 1;
      if (G3 > 1) nd = std::max(nd, (size_t)G3 * rows * ops->lv[k].dp);
    }
    // the stream-K form of the leaf level of tier 0 (an autotuner variant
    // and a tree option) when its transposed tiles fill less than two waves
    // of the SMs
    if (ops->tier == 0 && ws.wa_t256[kap] && nboxes(kap) / 8 * R >= 256 && m2l_t256_ctas(kap, R) < 2 * nsm)
      EIFMM_TRY(build_sk_plan(kap, R, nsm, &ws.sk));
    if (need) EIFMM_TRY(dalloc(&ws.m2l_part, need));
    ws.m2l_part_cap = need;
    if (need_leaf) EIFMM_TRY(dalloc(&ws.m2l_part_leaf, need_leaf));
    ws.m2l_part_leaf_cap = need_leaf;
  }
  if (!ws.wmax) EIFMM_TRY(dalloc(&ws.wmax, (size_t)kMaxLevel + 1));
  if (!ws.err) {
    EIFMM_TRY(dalloc(&ws.err, 1));
    EIFMM_CUDA(cudaMemset(ws.err, 0, sizeof(int)));
    EIFMM_CUDA(cudaMallocHost(&ws.err_host, sizeof(int)));
    *ws.err_host = 0;
  }
  return EIFMM_OK;
}

// ---------------------------------------------------------------------------
// Near field with each unordered pair of leaves visited once (tier 0, one
// right-hand side, targets = sources; every kernel of the library is even,
// K(-z) = K(z), so k_ij serves both f_i and f_j).  The CTA of leaf A takes
// A itself and its 13 forward neighbours B = A + o (neighbour index
// (dx+1) + 3(dy+1) + 9(dz+1) above 13).  For i in A and j in B it adds
// sigma_j k_ij to f_i and sigma_i k_ij to the partial g_j, written to
// gsym[s][j] (s = the forward offset); the L2P of B adds the partials of its
// 13 backward neighbours in a fixed order.  The own leaf is done in full
// (f only, i != j).  Every entry of gsym is written by one CTA, so the result
// is deterministic.
//
// Threads: a warp computes 32 targets x 32 sources, lane (ta, sb) =
// (lane / 4, lane % 4) the 4 x 8 block of targets 4 ta .. 4 ta + 3 and
// sources 8 sb .. 8 sb + 7, with f and g partials in registers; the f
// partials are reduce-scattered over the 4 sb lanes and the g partials over
// the 8 ta lanes with shuffles.  Warps share the column tiles of the staged
// source list; targets are staged SYM_TGT at a time.
// ---------------------------------------------------------------------------
constexpr int SYM_THREADS = 128;
constexpr int SYM_WARPS = SYM_THREADS / 32;
constexpr int SYM_SRC = 1024;
constexpr int SYM_TGT = 128;

template <int KERN>
__global__ void __launch_bounds__(SYM_THREADS)
k_p2p32_sym(int kern_rt, const int32_t* __restrict__ leaves, const int32_t* __restrict__ off,
            const float* __restrict__ lx, const float* __restrict__ ly, const float* __restrict__ lz,
            const float* __restrict__ sig, int64_t n, int depth, float two_l, double* __restrict__ fnear,
            float* __restrict__ gsym) {
  const int kern = KERN >= 0 ? KERN : kern_rt;
  __shared__ float4 s_src[SYM_SRC];
  __shared__ int64_t s_out[SYM_SRC];  // gsym index of a forward source, -1 for the leaf's own points
  __shared__ float4 s_tgt[SYM_TGT];
  __shared__ float s_f[SYM_WARPS][SYM_TGT];
  __shared__ int s_pos[15];    // prefix of the segment lengths (0..12 forward, 13 own)
  __shared__ int s_beg[14];
  __shared__ float s_sh[14][3];
  const unsigned full = 0xffffffffu;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int ta = lane >> 2, sb = lane & 3;
  const int b = leaves[blockIdx.x];
  int c[3];
  morton_decode(b, depth, c);
  const int nside = 1 << depth;
  if (tid < 14) {
    const int nb = tid < 13 ? 14 + tid : 13;
    const int dx = nb % 3 - 1, dy = (nb / 3) % 3 - 1, dz = nb / 9 - 1;
    const int jx = c[0] + dx, jy = c[1] + dy, jz = c[2] + dz;
    int beg = 0, len = 0;
    if (jx >= 0 && jy >= 0 && jz >= 0 && jx < nside && jy < nside && jz < nside) {
      const int64_t J = morton_encode(jx, jy, jz, depth);
      beg = off[J];
      len = off[J + 1] - beg;
    }
    s_beg[tid] = beg;
    s_pos[tid + 1] = len;
    s_sh[tid][0] = dx * two_l;
    s_sh[tid][1] = dy * two_l;
    s_sh[tid][2] = dz * two_l;
  }
  __syncthreads();
  if (tid == 0) {
    s_pos[0] = 0;
    for (int i = 1; i <= 14; ++i) s_pos[i] += s_pos[i - 1];
  }
  __syncthreads();
  const int n_fwd = s_pos[13], n_all = s_pos[14];
  const int tbeg = off[b], tend = off[b + 1];
  for (int t0 = tbeg; t0 < tend; t0 += SYM_TGT) {
    const int nt = min(SYM_TGT, tend - t0);
    const int nrt = (nt + 31) >> 5;
    __syncthreads();
    for (int i = tid; i < SYM_TGT; i += SYM_THREADS) {
      // padding targets: sigma 0, far from every source and from the padding sources
      s_tgt[i] = i < nt ? make_float4(lx[t0 + i], ly[t0 + i], lz[t0 + i], sig[t0 + i])
                        : make_float4(1e6f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < SYM_WARPS; ++q) s_f[q][i] = 0.f;
    }
    for (int c0 = 0; c0 < n_all; c0 += SYM_SRC) {
      const int cn = min(SYM_SRC, n_all - c0);
      const int nct = (cn + 31) >> 5;
      __syncthreads();
      for (int sg = w; sg < 14; sg += SYM_WARPS) {
        const int pb = s_pos[sg], pe = s_pos[sg + 1];
        const int lo = max(pb, c0), hi = min(pe, c0 + cn);
        const float sx = s_sh[sg][0], sy = s_sh[sg][1], sz = s_sh[sg][2];
        for (int pos = lo + lane; pos < hi; pos += 32) {
          const int sj = s_beg[sg] + (pos - pb);
          const int q = pos - c0;
          s_src[q] = make_float4(lx[sj] + sx, ly[sj] + sy, lz[sj] + sz, sig[sj]);
          s_out[q] = sg < kSymSlots ? (int64_t)sg * n + sj : -1;
        }
      }
      for (int q = cn + tid; q < nct * 32; q += SYM_THREADS) {
        s_src[q] = make_float4(-1e6f, 0.f, 0.f, 0.f);
        s_out[q] = -1;
      }
      __syncthreads();
      for (int ct = w; ct < nct; ct += SYM_WARPS) {
        const int jb = ct * 32 + sb * 8;
        float4 sj[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) sj[v] = s_src[jb + v];
        // own-leaf sources of this tile start at column own0 (>= 8: none)
        const int own0 = n_fwd - (c0 + jb);
        float gl[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) gl[v] = 0.f;
        for (int rt = 0; rt < nrt; ++rt) {
          const int ib = rt * 32 + ta * 4;
          float4 ti[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) ti[u] = s_tgt[ib + u];
          float fl[4] = {0.f, 0.f, 0.f, 0.f};
          if (own0 >= 8) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 8; ++v) {
                const float kv = kern_pt<KERN, false>(kern, ti[u].x - sj[v].x, ti[u].y - sj[v].y, ti[u].z - sj[v].z);
                fl[u] = fmaf(sj[v].w, kv, fl[u]);
                gl[v] = fmaf(ti[u].w, kv, gl[v]);
              }
          } else {
            // the own leaf: source column v is the own point own_idx = v - own0
            // (when v >= own0); the self pair is target (t0 - tbeg) + ib + u
            const int tself = (t0 - tbeg) + ib;
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 8; ++v) {
                float kv = kern_pt<KERN, false>(kern, ti[u].x - sj[v].x, ti[u].y - sj[v].y, ti[u].z - sj[v].z);
                const bool own = v >= own0;
                if (own && v - own0 == tself + u) kv = 0.f;
                fl[u] = fmaf(sj[v].w, kv, fl[u]);
                if (!own) gl[v] = fmaf(ti[u].w, kv, gl[v]);
              }
          }
          // f: reduce-scatter over the 4 sb lanes; lane (ta, sb) gets target ib + sb
          float k0 = (sb & 1) ? fl[1] : fl[0], k1 = (sb & 1) ? fl[3] : fl[2];
          const float a0 = (sb & 1) ? fl[0] : fl[1], a1 = (sb & 1) ? fl[2] : fl[3];
          k0 += __shfl_xor_sync(full, a0, 1);
          k1 += __shfl_xor_sync(full, a1, 1);
          float fk = (sb & 2) ? k1 : k0;
          fk += __shfl_xor_sync(full, (sb & 2) ? k0 : k1, 2);
          s_f[w][ib + sb] += fk;
        }
        // g: reduce-scatter over the 8 ta lanes; lane (ta, sb) gets source jb + ta
        float y[4], z[2];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const float mine = (ta & 1) ? gl[2 * m + 1] : gl[2 * m];
          const float other = (ta & 1) ? gl[2 * m] : gl[2 * m + 1];
          y[m] = mine + __shfl_xor_sync(full, other, 4);
        }
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          const float mine = (ta & 2) ? y[2 * m + 1] : y[2 * m];
          const float other = (ta & 2) ? y[2 * m] : y[2 * m + 1];
          z[m] = mine + __shfl_xor_sync(full, other, 8);
        }
        const float g = ((ta & 4) ? z[1] : z[0]) + __shfl_xor_sync(full, (ta & 4) ? z[0] : z[1], 16);
        const int64_t o = s_out[jb + ta];
        if (o >= 0) gsym[o] = t0 == tbeg ? g : gsym[o] + g;
      }
    }
    __syncthreads();
    for (int i = tid; i < nt; i += SYM_THREADS) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < SYM_WARPS; ++q) s += (double)s_f[q][i];
      fnear[t0 + i] = s;
    }
  }
}

template <int KERN, int RCT, bool ACC>
static void p2p_launch(const Tree* t, int kern, const float* sig32, int R, double* fnear, float two_l,
                       cudaStream_t s) {
  const PointSet& T = t->tgt;
  const PointSet& S = t->src;
  if (KERN == EIFMM_KERNEL_INV_R && RCT == 1) {  // 1/r, one right-hand side: packed distances
    static bool attr[64][2] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64 || !attr[dev][ACC]) {
      cudaFuncSetAttribute(k_p2p32x<ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NF_SMEM);
      if (dev < 64) attr[dev][ACC] = true;
    }
    k_p2p32x<ACC><<<(unsigned)T.n_nonempty, NF_THREADS, NF_SMEM, s>>>(
        T.nonempty, T.leaf_off, T.lx, T.ly, T.lz, S.leaf_off, S.lx, S.ly, S.lz, sig32, t->depth, two_l,
        t->exclude_self, fnear);
    return;
  }
  k_p2p32<KERN, RCT, ACC><<<(unsigned)T.n_nonempty, P2P_THREADS, 0, s>>>(
      kern, T.nonempty, T.leaf_off, T.lx, T.ly, T.lz, T.n, S.leaf_off, S.lx, S.ly, S.lz,
      sig32, S.n, R, t->depth, two_l, t->exclude_self, fnear);
}

// The pair-symmetric near field can serve tier 0 with one right-hand side
// on a tree whose targets are its sources; it runs when the tree's option
// EIFMM_OPT_P2P_PAIR_SYMMETRIC is on
// (read at every evaluate).  It is not the default: it measured slower than
// the per-target kernel (588 against 423 us at 1M points).
static bool use_p2p_sym(const Tree* t, int R, bool accurate, const float* gsym) {
  return gsym && !accurate && R == 1 && t->same && t->exclude_self &&
         (t->opt[EIFMM_OPT_P2P_PAIR_SYMMETRIC] || t->ws.p2p_sym == 1);
}

eifmm_status launch_p2p32(const Tree* t, int kern, const float* sig32, int R, double* fnear,
                          cudaStream_t s, bool accurate, float* gsym) {
  if (t->tgt.n_nonempty == 0) return EIFMM_OK;
  const float two_l = (float)(t->L * ldexp(1.0, -t->depth));
  if (use_p2p_sym(t, R, accurate, gsym)) {
    const PointSet& T = t->tgt;
    if (kern == EIFMM_KERNEL_INV_R)
      k_p2p32_sym<EIFMM_KERNEL_INV_R><<<(unsigned)T.n_nonempty, SYM_THREADS, 0, s>>>(
          kern, T.nonempty, T.leaf_off, T.lx, T.ly, T.lz, sig32, T.n, t->depth, two_l, fnear, gsym);
    else
      k_p2p32_sym<-1><<<(unsigned)T.n_nonempty, SYM_THREADS, 0, s>>>(
          kern, T.nonempty, T.leaf_off, T.lx, T.ly, T.lz, sig32, T.n, t->depth, two_l, fnear, gsym);
    EIFMM_CHECK_LAUNCH();
    return EIFMM_OK;
  }
  const bool inv = kern == EIFMM_KERNEL_INV_R;
  if (R == 1) {
    if (inv) {
      if (accurate) p2p_launch<EIFMM_KERNEL_INV_R, 1, true>(t, kern, sig32, R, fnear, two_l, s);
      else p2p_launch<EIFMM_KERNEL_INV_R, 1, false>(t, kern, sig32, R, fnear, two_l, s);
    } else {
      if (accurate) p2p_launch<-1, 1, true>(t, kern, sig32, R, fnear, two_l, s);
      else p2p_launch<-1, 1, false>(t, kern, sig32, R, fnear, two_l, s);
    }
  } else {
    if (inv) {
      if (accurate) p2p_launch<EIFMM_KERNEL_INV_R, 4, true>(t, kern, sig32, R, fnear, two_l, s);
      else p2p_launch<EIFMM_KERNEL_INV_R, 4, false>(t, kern, sig32, R, fnear, two_l, s);
    } else {
      if (accurate) p2p_launch<-1, 4, true>(t, kern, sig32, R, fnear, two_l, s);
      else p2p_launch<-1, 4, false>(t, kern, sig32, R, fnear, two_l, s);
    }
  }
  EIFMM_CHECK_LAUNCH();
  return EIFMM_OK;
}

static void record(Workspace& ws, int i, cudaStream_t s) {
  if (timing_enabled()) cudaEventRecord(ws.ev_t[i], s);
}

static int sm_count() {
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm;
}

static int shift_groups(int g, int shift) {
  g = shift >= 0 ? g << shift : g >> -shift;
  return g < 1 ? 1 : (g > 16 ? 16 : g);
}

// Step 4 at level k.  kind 0 follows the built-in rule (the transposed kernel
// where a parity class fills a 256-row tile and dp = 128, else the 128-row
// TMA kernel, else the cp.async one); 1-3 force a variant (autotuner);
// gshift scales the offset-group count.  EUNSUPPORTED when the variant does
// not apply to this level.
eifmm_status launch_m2l_level(Tree* t, const Ops* ops, int k, int R, int kind, int gshift, cudaStream_t s) {
  Workspace& ws = t->ws;
  const bool tf32 = false;
  const int fmt = ops->tier == 1 ? kPlaneF16 : kPlaneBF16;
  const LevelOps& v = ops->lv[k];
  if (ops->tier == 1 && (v.kd_img == nullptr || !ws.wa_grid[k])) {
    // no FP16 tile for this level (dp above 256 or no tile shape for R): the
    // SIMT M2L with its compensated sums serves it
    if (kind != 0) return EIFMM_EUNSUPPORTED;
    return launch_m2l_simt(t, ops, k, R, s);
  }
  if (v.kd_img == nullptr || v.kd_img_fmt != fmt) {
    set_error("eifmm_evaluate: tensor-core M2L operands missing for this level (d too large)");
    return EIFMM_EUNSUPPORTED;
  }
  M2LTcArgs a;
  a.level = k;
  a.nbox = nboxes(k);
  a.R = R;
  a.rows = a.nbox * R;
  a.dp = v.dp;
  a.tmem_cols = v.dp <= 128 ? 128 : (v.dp <= 256 ? 256 : 512);
  a.wa = ws.wa[k];
  a.kd_img = v.kd_img;
  a.slot_lists = ops->d_slot_lists;
  a.g = ws.g32[k];
  a.err = ws.err;
  const bool leaf = k == t->depth;
  a.part = leaf ? ws.m2l_part_leaf : ws.m2l_part;
  const size_t cap = leaf ? ws.m2l_part_leaf_cap : ws.m2l_part_cap;
  const int nsm = sm_count();
  if (ops->tier == 1) {  // FP16 planes, per-offset drains: one variant
    if (kind != 0) return EIFMM_EUNSUPPORTED;
    a.groups = shift_groups(m2l_h16_groups(m2l_tma_ctas(k, R), nsm), gshift);
    if (a.groups > 1 && (size_t)a.groups * a.rows * a.dp > cap) return EIFMM_EUNSUPPORTED;
    return launch_m2l_h16(a, ws.tmap[k][0], ws.tmap[k][1], ws.wmax, v.kscale, s);
  }
  const bool rule = kind == 0;
  if (rule) {
    // the transposed kernel where a parity class fills at least one of its
    // 256-row tiles; the 128-row kernel at the coarse levels
    kind = (ws.wa_t256[k] && nboxes(k) / 8 * R >= 256 && !t->opt[EIFMM_OPT_M2L_128ROW]) ? 1
                                                                                         : (ws.wa_grid[k] ? 2 : 4);
    if (kind == 1 && leaf && ws.sk.tu && t->opt[EIFMM_OPT_M2L_STREAM_K]) kind = 3;
  }
  if (kind == 3) {  // stream-K: one CTA per SM, no offset groups
    if (!leaf || !ws.sk.tu || !ws.wa_t256[k] || gshift != 0) return EIFMM_EUNSUPPORTED;
    return launch_m2l_t256s(a, ws.tmap2[k][0], ws.tmap2[k][1], ws.sk, s);
  }
  if (kind == 1) {
    if (!ws.wa_t256[k]) return EIFMM_EUNSUPPORTED;
    a.groups = shift_groups(m2l_t256_groups(m2l_t256_ctas(k, R), nsm), gshift);
  } else {
    // the 128-row TMA kernel reads the per-class grid planes, the cp.async
    // one the Morton-ordered planes
    if ((kind == 4) == ws.wa_grid[k]) return EIFMM_EUNSUPPORTED;
    a.groups = shift_groups(m2l_tc_groups((a.nbox / 8 * R + 127) / 128 * 8, nsm, a.dp), gshift);
  }
  if (a.groups > 1 && (size_t)a.groups * a.rows * a.dp > cap) return EIFMM_EUNSUPPORTED;
  if (kind == 1) return launch_m2l_t256(a, ws.tmap2[k][0], ws.tmap2[k][1], tf32, s);
  if (kind == 2) return launch_m2l_tma(a, ws.tmap[k][0], ws.tmap[k][1], tf32, s);
  return launch_m2l_tc(a, tf32, s);
}

eifmm_status eval_mixed(Tree* t, const Ops* ops, const double* sigma, int64_t ld_sigma, int R,
                        double* f, int64_t ld_f, cudaStream_t s) {
  if (ops->tier == 3) return eval_fp64(t, ops, sigma, ld_sigma, R, f, ld_f, s, true, true);
  Workspace& ws = t->ws;
  if (*ws.err_host != 0) {
    const int code = *ws.err_host;
    *ws.err_host = 0;
    cudaMemsetAsync(ws.err, 0, sizeof(int), s);
    set_error("eifmm_evaluate: a bounded device wait of the previous call timed out (code " +
              std::to_string(code) + ")");
    return EIFMM_ETIMEOUT;
  }
  // P2M and L2P: the approximate reciprocal square root alone in tier 0
  // (relative error below 2^-22), one Newton step above
  const bool acc = ops->tier >= 1;
  const int kap = t->depth;
  const int kern = (int)ops->kern;
  const PointSet& S = t->src;
  const PointSet& T = t->tgt;
  record(ws, 0, s);
  const LevelOps& vl = ops->lv[kap];
  const bool p2m_x = kern == EIFMM_KERNEL_INV_R && R == 1 && vl.dp <= 2 * PT_MAXQ;
  // the FP32 tiers read only the FP32 copy of the sorted sigma.  The packed
  // P2M reads sigma through the permutation itself, so there only the near
  // field waits for the copy (it is made on the near field's stream)
  if (!p2m_x) EIFMM_TRY(launch_gather_sigma(sigma, ld_sigma, S, R, nullptr, ws.sig32, s));
  EIFMM_CUDA(cudaEventRecord(ws.ev_fork, s));
  EIFMM_CUDA(cudaStreamWaitEvent(ws.side, ws.ev_fork, 0));
  // the far field continues on the high-priority stream; the caller's stream
  // waits for it at the end
  const cudaStream_t caller = s;
  const bool single = t->opt[EIFMM_OPT_SINGLE_STREAM] != 0;
  if (!single) {
    EIFMM_CUDA(cudaStreamWaitEvent(ws.hi, ws.ev_fork, 0));
    s = ws.hi;
  }
  // with the single-stream option every launch below goes to the caller's
  // stream, in submission order
  const cudaStream_t nf_stream = single ? s : ws.side;
  const cudaStream_t coarse_stream = single ? s : ws.side2;
  // when a step fails after the fork, the caller's stream still waits for
  // every stream this call may have used, so that no work of the call is
  // left unordered against the caller's next one
  struct ForkGuard {
    Workspace& w;
    cudaStream_t caller;
    bool armed = true;
    ~ForkGuard() {
      if (!armed) return;
      cudaEventRecord(w.ev_join, w.side);
      cudaStreamWaitEvent(caller, w.ev_join, 0);
      cudaEventRecord(w.ev_join2, w.side2);
      cudaStreamWaitEvent(caller, w.ev_join2, 0);
      cudaEventRecord(w.ev_hi, w.hi);
      cudaStreamWaitEvent(caller, w.ev_hi, 0);
    }
  } guard{ws, caller};
  if (p2m_x) EIFMM_TRY(launch_gather_sigma(sigma, ld_sigma, S, R, nullptr, ws.sig32, nf_stream));
  const bool p2p_sym = use_p2p_sym(t, R, ops->tier >= 1, ws.gsym);
  auto near_field = [&]() -> eifmm_status {
    if (timing_enabled()) cudaEventRecord(ws.ev_nf[0], nf_stream);
    EIFMM_TRY(launch_p2p32(t, kern, ws.sig32, R, ws.fnear, nf_stream, ops->tier >= 1, ws.gsym));
    if (timing_enabled()) cudaEventRecord(ws.ev_nf[1], nf_stream);
    EIFMM_CUDA(cudaEventRecord(ws.ev_join, ws.side));
    return EIFMM_OK;
  };
  // by default the near field starts with the far field; with the option
  // NEAR_FIELD_LATE it starts with the M2L (step 4 below)
  const bool nf_late = !single && t->opt[EIFMM_OPT_NEAR_FIELD_LATE];
  if (!nf_late) EIFMM_TRY(near_field());

  // step 1 (every leaf, empty ones get zeros)
  // tier 0: the packed P2M also writes the leaf level's BF16 planes (step 3)
  const bool leaf_planes_in_p2m = p2m_x && ops->tier == 0 && ws.wa[kap] != nullptr;
  {
    const unsigned nb = (unsigned)nboxes(kap);
#define EIFMM_P2M(K, RC_, A)                                                                   \
  k_p2m32<K, RC_, A><<<nb, TPB, 0, s>>>(kern, S.leaf_off, S.lx, S.ly, S.lz, ws.sig32, S.n, R, vl.X32, \
                                        vl.d, vl.dp, ws.W32[kap])
    if (p2m_x) {
      const unsigned g = (unsigned)((nboxes(kap) + PT_WARPS - 1) / PT_WARPS);
      __nv_bfloat16* lp = leaf_planes_in_p2m ? (__nv_bfloat16*)ws.wa[kap] : nullptr;
      const int gl = ws.wa_grid[kap] ? kap : -1;
      if (acc)
        k_p2m32x<true><<<g, 32 * PT_WARPS, 0, s>>>(S.leaf_off, nboxes(kap), S.lx, S.ly, S.lz, ws.sig32, vl.X32,
                                                   vl.d, vl.dp, ws.W32[kap], lp, gl, sigma, S.perm);
      else
        k_p2m32x<false><<<g, 32 * PT_WARPS, 0, s>>>(S.leaf_off, nboxes(kap), S.lx, S.ly, S.lz, ws.sig32, vl.X32,
                                                    vl.d, vl.dp, ws.W32[kap], lp, gl, sigma, S.perm);
    } else {
      EIFMM_POINT_DISPATCH(EIFMM_P2M);
    }
#undef EIFMM_P2M
    EIFMM_CHECK_LAUNCH();
  }
  record(ws, 1, s);
  // step 2
  for (int k = kap - 1; k >= 2; --k) {
    const LevelOps& a = ops->lv[k];
    const LevelOps& c = ops->lv[k + 1];
    XferGemm x;
    x.mode = 0;
    x.dk = a.d; x.ldk = a.dp; x.dc = c.d; x.ldc = c.dp; x.R = R;
    x.ncol = nboxes(k) * R;
    x.A = a.m2m32; x.B = ws.W32[k + 1]; x.G = nullptr; x.C = ws.W32[k];
    x.P8 = (float*)ws.tmp;  // 8 x nboxes(k) x R x dp floats fit in the scratch
    if (!xfer_blas(true, a, c, nboxes(k), R, ws.W32[k + 1], nullptr, ws.W32[k], ws.blas_ws, s))
      EIFMM_TRY(launch_xfer_gemm(x, s));
  }
  record(ws, 2, s);
  // step 3: What = Delta W is folded into the M2L operator (K^delta Delta,
  // built with the operators), so the M2L reads the planes of W itself
  // (tier 2 reads W in FP32)
  const bool simt = ops->tier == 2;
  if (!simt) {
    PlaneBatch b;
    AbsMaxBatch mb;
    mb.lo = 2;
    mb.hi = kap;
    for (int k = 2; k <= kap; ++k) {
      if (k == kap && leaf_planes_in_p2m) continue;  // written by the P2M
      const LevelOps& v = ops->lv[k];
      PlaneLevel& L = b.lv[b.nlev++];
      L.in = ws.W32[k]; L.out = ws.wa[k];
      L.rows = nboxes(k) * R; L.q0 = b.nq;
      L.d = v.d; L.dp = v.dp; L.grid_level = ws.wa_grid[k] ? k : -1; L.R = R; L.level = k;
      b.nq += L.rows * v.dp / 4;
      mb.w[k] = ws.W32[k];
      mb.n[k] = L.rows * v.dp;
    }
    const unsigned g = grid_for(b.nq > 0 ? b.nq : 1, 256, 152 * 16);
    if (b.nq == 0) {
      // nothing left to split
    } else if (ops->tier == 1) {
      // the FP16 planes need the largest |W| of every level first
      EIFMM_CUDA(cudaMemsetAsync(ws.wmax, 0, (kMaxLevel + 1) * sizeof(uint32_t), s));
      k_absmax<<<152 * 4, 256, 0, s>>>(mb, ws.wmax);
      EIFMM_CHECK_LAUNCH();
      b.wmax = ws.wmax;
      k_planes<kPlaneF16><<<g, 256, 0, s>>>(b);
    } else {
      k_planes<kPlaneBF16><<<g, 256, 0, s>>>(b);
    }
    EIFMM_CHECK_LAUNCH();
  }
  record(ws, 3, s);
  // step 4: the levels are independent.  The coarse levels run on a second
  // stream while the leaf level runs here, so their small grids fill the
  // SMs the leaf level leaves free; each side has its own partial sums.
  EIFMM_CUDA(cudaEventRecord(ws.ev_fork2, s));
  if (kap > 2) EIFMM_CUDA(cudaStreamWaitEvent(ws.side2, ws.ev_fork2, 0));
  if (nf_late) {
    EIFMM_CUDA(cudaStreamWaitEvent(ws.side, ws.ev_fork2, 0));
    EIFMM_TRY(near_field());
  }
  auto m2l = [&](int k, cudaStream_t st) {
    return simt ? launch_m2l_simt(t, ops, k, R, st)
                : launch_m2l_level(t, ops, k, R, ws.m2l_kind[k], ws.m2l_gshift[k], st);
  };
  // The SIMT M2L of tier 2 submits the coarse levels first: each of their
  // few blocks walks all 189 offsets, so they must start early to end
  // within the leaf level.
  auto coarse = [&]() -> eifmm_status {
    for (int k = 2; k < kap; ++k) {
      if (timing_enabled()) cudaEventRecord(ws.ev_m2l[k], coarse_stream);
      EIFMM_TRY(m2l(k, coarse_stream));
      if (timing_enabled()) cudaEventRecord(ws.ev_m2le[k], coarse_stream);
    }
    return EIFMM_OK;
  };
  if (simt) EIFMM_TRY(coarse());
  if (timing_enabled()) cudaEventRecord(ws.ev_m2l[kap], s);
  EIFMM_TRY(m2l(kap, s));
  if (timing_enabled()) cudaEventRecord(ws.ev_m2le[kap], s);
  if (!simt) EIFMM_TRY(coarse());
  if (kap > 2) {
    EIFMM_CUDA(cudaEventRecord(ws.ev_join2, ws.side2));
    EIFMM_CUDA(cudaStreamWaitEvent(s, ws.ev_join2, 0));
  }
  record(ws, 4, s);
  // step 5
  for (int k = 3; k <= kap; ++k) {
    const LevelOps& v = ops->lv[k];
    const LevelOps& pv = ops->lv[k - 1];
    XferGemm x;
    x.mode = 1;
    x.dk = v.d; x.ldk = v.dp; x.dc = pv.d; x.ldc = pv.dp; x.R = R;
    x.ncol = nboxes(k - 1) * R;
    x.A = v.l2l32; x.B = ws.l32[k - 1]; x.G = ws.g32[k]; x.C = ws.l32[k];
    x.P8 = nullptr;
    if (!xfer_blas(false, v, pv, nboxes(k - 1), R, ws.l32[k - 1], ws.g32[k], ws.l32[k], ws.blas_ws, s))
      EIFMM_TRY(launch_xfer_gemm(x, s));
  }
  record(ws, 5, s);
  // step 6: lhat = Delta^t l (B z = l, then Gamma^t lhat = z)
  {
    DeltaBatch b;
    b.nlev = 1;
    b.lv[0] = delta_level(vl.d, delta_ops32(vl), true, ws.l32[kap], vl.dp, ws.lh32, vl.dp, nullptr,
                          nboxes(kap) * R);
    EIFMM_TRY((launch_delta_batch<float, float, float, 0>(b, true, s)));
  }
  record(ws, 6, s);
  // step 7.  The L2P of the far field does not wait for the near field
  // (which runs at the lower priority and ends last); a short kernel then
  // adds the two in the caller's order.  The pair-symmetric near field needs
  // the L2P's per-leaf neighbour test, so it keeps the combined L2P.
  auto l2p = [&](double* fout) -> eifmm_status {
    if (T.n_nonempty == 0) return EIFMM_OK;
    const unsigned nl = (unsigned)T.n_nonempty;
    if (!fout && !p2p_sym && kern == EIFMM_KERNEL_INV_R && R == 1 && vl.dp <= 2 * PT_MAXQ) {
      const unsigned g = (unsigned)((T.n_nonempty + PT_WARPS - 1) / PT_WARPS);
      if (acc)
        k_l2p32x<true><<<g, 32 * PT_WARPS, 0, s>>>(T.nonempty, T.n_nonempty, T.leaf_off, T.lx, T.ly, T.lz,
                                                   vl.X32, vl.d, vl.dp, ws.lh32, ws.ffar);
      else
        k_l2p32x<false><<<g, 32 * PT_WARPS, 0, s>>>(T.nonempty, T.n_nonempty, T.leaf_off, T.lx, T.ly, T.lz,
                                                    vl.X32, vl.d, vl.dp, ws.lh32, ws.ffar);
      EIFMM_CHECK_LAUNCH();
      return EIFMM_OK;
    }
    const int rct = R == 1 ? 1 : RC;
    const size_t sm = (size_t)vl.d * sizeof(float4) + (size_t)((rct > 1 ? rct * vl.d : 0) + rct * TPB) * sizeof(float);
#define EIFMM_L2P(K, RC_, A)                                                                     \
  k_l2p32<K, RC_, A><<<nl, TPB, sm, s>>>(kern, T.nonempty, T.leaf_off, T.perm, T.lx, T.ly, T.lz, T.n, R, \
                                         vl.X32, vl.d, vl.dp, ws.lh32, ws.fnear, ws.ffar, fout, ld_f,       \
                                         p2p_sym ? ws.gsym : nullptr, kap)
    EIFMM_POINT_DISPATCH(EIFMM_L2P);
#undef EIFMM_L2P
    EIFMM_CHECK_LAUNCH();
    return EIFMM_OK;
  };
  if (!p2p_sym) EIFMM_TRY(l2p(nullptr));
  EIFMM_CUDA(cudaStreamWaitEvent(s, ws.ev_join, 0));
  record(ws, 7, s);
  if (p2p_sym) {
    EIFMM_TRY(l2p(f));
  } else if (T.n > 0) {
    k_combine<<<grid_for(T.n * R, 256, 8192), 256, 0, s>>>(T.perm, T.n, R, ws.ffar, ws.fnear, f, ld_f);
    EIFMM_CHECK_LAUNCH();
  }
  EIFMM_CUDA(cudaMemcpyAsync(ws.err_host, ws.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  record(ws, 8, s);
  if (s != caller) {
    EIFMM_CUDA(cudaEventRecord(ws.ev_hi, s));
    EIFMM_CUDA(cudaStreamWaitEvent(caller, ws.ev_hi, 0));
  }
  guard.armed = false;
  return EIFMM_OK;
}

eifmm_status export_mixed(const Tree& t, const Ops& o, int what, int level, double* out, int64_t n) {
  const Workspace& ws = t.ws;
  const LevelOps& v = o.lv[level];
  const int64_t nvec = nboxes(level) * ws.nrhs;
  const int64_t cnt = nvec * v.d;
  if (n < cnt) {
    set_error("eifmm_debug_export: output too small");
    return EIFMM_EINVAL;
  }
  double* tmp = nullptr;
  EIFMM_TRY(dalloc(&tmp, cnt));
  if (what == 1) {
    // What = Delta W, from the FP32 W of the evaluation (FP64 solves)
    k_f32_to_f64<<<grid_for(cnt, 256), 256>>>(ws.W32[level], nvec, v.d, v.dp, tmp);
    EIFMM_CHECK_LAUNCH();
    DeltaBatch b;
    b.nlev = 1;
    b.lv[0] = delta_level(v.d, delta_ops64(v), false, tmp, v.d, tmp, v.d, nullptr, nvec);
    const eifmm_status rc = launch_delta_batch<double, double, double, 0>(b, false, 0);
    if (rc != EIFMM_OK) {
      dfree(tmp);
      return rc;
    }
  } else {
    const float* src = what == 0 ? ws.W32[level] : what == 2 ? ws.g32[level] : what == 3 ? ws.l32[level] : ws.lh32;
    k_f32_to_f64<<<grid_for(cnt, 256), 256>>>(src, nvec, v.d, v.dp, tmp);
  }
  EIFMM_CHECK_LAUNCH();
  EIFMM_CUDA(cudaMemcpy(out, tmp, cnt * sizeof(double), cudaMemcpyDeviceToHost));
  dfree(tmp);
  return EIFMM_OK;
}

}  // namespace eifmm
