// fmm32.cu -- the mixed-precision EIFMM (Algorithm 3 + near field).
//
// Tier 0 (EIM tolerance >= 1e-5): P2M, M2M, the Delta solves, L2L and L2P in
// FP32 on coordinates local to each leaf; M2L on tcgen05 with BF16 hi + lo
// operand planes (m2l_tc.cu).  Tier 1 (>= 1e-6): the Delta solves in FP64 and
// M2L with TF32 hi + lo planes.  Tier 2 (< 1e-6): the FP64 far field of
// fmm64.cu.  Every tier evaluates the near field here in FP32 with Kahan
// compensated summation.
//
// Far-field arrays: [row = box * R + r][dp] FP32, dp = d rounded up to 64,
// padding columns zero.
#include <algorithm>

#include "internal.h"
#include "m2l_tc.h"
#include "transfer.cuh"
#include "solve.cuh"

namespace eifmm {

eifmm_status launch_gather_sigma(const double* sigma, int64_t ld, const PointSet& src, int R,
                                 double* s64, float* s32, cudaStream_t s);

namespace {

constexpr int TPB = 128;
constexpr int RC = 4;

__host__ __device__ inline int64_t nboxes(int k) { return (int64_t)1 << (3 * k); }

// ---------------------------------------------------------------- step 1 --
// W_m^I = sum_{y_j in I} sigma_j K(x_m^{I_0}, y_j - c_I), FP32, local coords.
template <int KERN>
__global__ void __launch_bounds__(TPB)
k_p2m32(int kern_rt, const int32_t* __restrict__ off, const float* __restrict__ lx,
        const float* __restrict__ ly, const float* __restrict__ lz,
        const float* __restrict__ sig, int64_t n, int R, const float* __restrict__ X, int d,
        int dp, float* __restrict__ W) {
  const int kern = KERN >= 0 ? KERN : kern_rt;
  __shared__ float sz[3][TPB];
  __shared__ float ss[RC][TPB];
  const int64_t b = blockIdx.x;
  const int beg = off[b], end = off[b + 1];
  for (int r0 = 0; r0 < R; r0 += RC) {
    for (int m0 = 0; m0 < dp; m0 += TPB) {
      const int m = m0 + threadIdx.x;
      float x0 = 0.f, x1 = 0.f, x2 = 0.f;
      if (m < d) { x0 = X[3 * m]; x1 = X[3 * m + 1]; x2 = X[3 * m + 2]; }
      float acc[RC] = {0.f, 0.f, 0.f, 0.f};
      for (int j0 = beg; j0 < end; j0 += TPB) {
        const int j = j0 + threadIdx.x;
        __syncthreads();
        if (j < end) {
          sz[0][threadIdx.x] = lx[j];
          sz[1][threadIdx.x] = ly[j];
          sz[2][threadIdx.x] = lz[j];
#pragma unroll
          for (int rr = 0; rr < RC; ++rr) ss[rr][threadIdx.x] = (r0 + rr < R) ? sig[j + (r0 + rr) * n] : 0.f;
        }
        __syncthreads();
        const int cnt = min(TPB, end - j0);
        if (m < d)
          for (int t = 0; t < cnt; ++t) {
            const float kv = kern_f32(kern, x0 - sz[0][t], x1 - sz[1][t], x2 - sz[2][t]);
#pragma unroll
            for (int rr = 0; rr < RC; ++rr) acc[rr] = fmaf(ss[rr][t], kv, acc[rr]);
          }
      }
      if (m < dp)
        for (int rr = 0; rr < RC && r0 + rr < R; ++rr) W[(b * R + r0 + rr) * dp + m] = acc[rr];
    }
  }
}


// ---------------------------------------------------------------- step 7 --
template <int KERN>
__global__ void __launch_bounds__(TPB)
k_l2p32(int kern_rt, const int32_t* __restrict__ leaves, const int32_t* __restrict__ off,
        const int32_t* __restrict__ perm, const float* __restrict__ lx,
        const float* __restrict__ ly, const float* __restrict__ lz, int64_t n, int R,
        const float* __restrict__ X, int d, int dp, const float* __restrict__ lh,
        const double* __restrict__ fnear, double* __restrict__ ffar, double* __restrict__ f,
        int64_t ld_f) {
  const int kern = KERN >= 0 ? KERN : kern_rt;
  extern __shared__ float smf[];  // X (3d) then lhat (RC d)
  float* sX = smf;
  float* sl = smf + 3 * d;
  const int b = leaves[blockIdx.x];
  const int beg = off[b], end = off[b + 1];
  for (int t = threadIdx.x; t < 3 * d; t += TPB) sX[t] = X[t];
  for (int r0 = 0; r0 < R; r0 += RC) {
    __syncthreads();
    for (int t = threadIdx.x; t < RC * d; t += TPB) {
      const int rr = t / d, l = t - rr * d;
      sl[t] = (r0 + rr < R) ? lh[((int64_t)b * R + r0 + rr) * dp + l] : 0.f;
    }
    __syncthreads();
    for (int p = beg + threadIdx.x; p < end; p += TPB) {
      const float z0 = lx[p], z1 = ly[p], z2 = lz[p];
      float acc[RC] = {0.f, 0.f, 0.f, 0.f};
      for (int l = 0; l < d; ++l) {
        const float kv = kern_f32(kern, z0 - sX[3 * l], z1 - sX[3 * l + 1], z2 - sX[3 * l + 2]);
#pragma unroll
        for (int rr = 0; rr < RC; ++rr) acc[rr] = fmaf(kv, sl[rr * d + l], acc[rr]);
      }
      const int64_t i = perm[p];
      for (int rr = 0; rr < RC && r0 + rr < R; ++rr) {
        const int rg = r0 + rr;
        if (ffar) ffar[p + rg * n] = acc[rr];
        f[i + rg * ld_f] = (double)acc[rr] + fnear[p + rg * n];
      }
    }
  }
}

// ------------------------------------------------------------ near field --
// One warp per target leaf.  Lanes = (target, slice): a chunk of up to 32
// targets is spread over Tp = next power of two >= count lanes and the
// sources over 32/Tp slices, so leaves of 8 points keep every lane busy.
// Sources are staged per warp in shared memory, expressed in the frame of
// the target leaf (exact shift by the leaf-centre offset); FP32 kernel,
// Kahan-compensated FP32 sums, slices combined in FP64.
constexpr int P2P_WARPS = 4;
constexpr int P2P_CHUNK = 64;

// ACC: Newton-refined 1/r and Kahan summation of every term (tiers 1, 2);
// otherwise the hardware rsqrt and plain FP32 sums per neighbour leaf, the
// 27 leaf sums combined with Kahan summation (tier 0).  RCT: right-hand
// sides per pass (the kernel value is reused across them).
template <int KERN, int RCT, bool ACC>
__global__ void __launch_bounds__(32 * P2P_WARPS)
k_p2p32(int kern_rt, const int32_t* __restrict__ leaves, int nleaves,
        const int32_t* __restrict__ toff, const float* __restrict__ tlx,
        const float* __restrict__ tly, const float* __restrict__ tlz, int64_t nt,
        const int32_t* __restrict__ soff, const float* __restrict__ slx,
        const float* __restrict__ sly, const float* __restrict__ slz,
        const float* __restrict__ sig, int64_t ns, int R, int depth, float two_l,
        int exclude_self, double* __restrict__ fnear) {
  const int kern = KERN >= 0 ? KERN : kern_rt;
  __shared__ float4 src[P2P_WARPS][P2P_CHUNK];        // xyz in the target frame
  __shared__ float ssig[P2P_WARPS][RCT][P2P_CHUNK];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * P2P_WARPS + w;
  if (gw >= nleaves) return;
  const int b = leaves[gw];
  int c[3];
  morton_decode(b, depth, c);
  const int n = 1 << depth;
  const int beg = toff[b], end = toff[b + 1];
  for (int t0 = beg; t0 < end; t0 += 32) {
    const int nT = min(32, end - t0);
    int Tp = 1;
    while (Tp < nT) Tp <<= 1;
    const int S = 32 / Tp;
    const int ti = lane & (Tp - 1), si = lane / Tp;
    const bool act = ti < nT;
    const int p = t0 + (act ? ti : 0);
    const int pself = (exclude_self && act) ? p : -1;
    const float x0 = tlx[p], x1 = tly[p], x2 = tlz[p];
    for (int r0 = 0; r0 < R; r0 += RCT) {
      float sum[RCT], comp[RCT];
#pragma unroll
      for (int rr = 0; rr < RCT; ++rr) sum[rr] = comp[rr] = 0.f;
      for (int nb = 0; nb < 27; ++nb) {
        const int dx = nb % 3 - 1, dy = (nb / 3) % 3 - 1, dz = nb / 9 - 1;
        const int jx = c[0] + dx, jy = c[1] + dy, jz = c[2] + dz;
        if (jx < 0 || jy < 0 || jz < 0 || jx >= n || jy >= n || jz >= n) continue;
        const int64_t J = morton_encode(jx, jy, jz, depth);
        const int sb = soff[J], se = soff[J + 1];
        // y - c_I = (y - c_J) + (c_J - c_I)
        const float s0 = dx * two_l, s1 = dy * two_l, s2 = dz * two_l;
        float part[RCT];
#pragma unroll
        for (int rr = 0; rr < RCT; ++rr) part[rr] = 0.f;
        for (int q0 = sb; q0 < se; q0 += P2P_CHUNK) {
          __syncwarp();
          for (int t = lane; t < P2P_CHUNK; t += 32) {
            const int q = q0 + t;
            if (q < se) {
              src[w][t] = make_float4(slx[q] + s0, sly[q] + s1, slz[q] + s2, 0.f);
#pragma unroll
              for (int rr = 0; rr < RCT; ++rr)
                ssig[w][rr][t] = (r0 + rr < R) ? sig[q + (int64_t)(r0 + rr) * ns] : 0.f;
            }
          }
          __syncwarp();
          const int cnt = min(P2P_CHUNK, se - q0);
          const int jself = pself - q0;  // the self pair, if it is in this chunk
          if (act)
            for (int j = si; j < cnt; j += S) {
              const float4 y = src[w][j];
              float kv = ACC ? kern_f32(kern, x0 - y.x, x1 - y.y, x2 - y.z)
                             : kern_f32_fast(kern, x0 - y.x, x1 - y.y, x2 - y.z);
              if (j == jself) kv = 0.f;
#pragma unroll
              for (int rr = 0; rr < RCT; ++rr) {
                const float term = ssig[w][rr][j] * kv;
                if (ACC) {
                  const float yk = term - comp[rr];
                  const float tk = sum[rr] + yk;
                  comp[rr] = (tk - sum[rr]) - yk;
                  sum[rr] = tk;
                } else {
                  part[rr] += term;
                }
              }
            }
        }
        if (!ACC) {
#pragma unroll
          for (int rr = 0; rr < RCT; ++rr) {
            const float yk = part[rr] - comp[rr];
            const float tk = sum[rr] + yk;
            comp[rr] = (tk - sum[rr]) - yk;
            sum[rr] = tk;
          }
        }
      }
#pragma unroll
      for (int rr = 0; rr < RCT; ++rr) {
        double tot = act ? (double)sum[rr] - (double)comp[rr] : 0.0;
        for (int o = Tp; o < 32; o <<= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        if (act && si == 0 && r0 + rr < R) fnear[p + (int64_t)(r0 + rr) * nt] = tot;
      }
    }
  }
}

// --------------------------------------------------- operator images ----
// K^delta (kdT[slot][l][m'] FP64) -> two planes in the swizzled image used
// by the tensor-core M2L: byte offset of row n, 16-byte unit j inside the
// 128-byte chunk: (n / 8) * 1024 + (n % 8) * 128 + ((j ^ (n % 8)) * 16).
__global__ void k_build_img(const double* __restrict__ kdT, int d, int dp, int tf32,
                            unsigned char* __restrict__ img) {
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
      if (tf32) {
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

// planes -> FP64 [row][d] (debug export of What)
__global__ void k_planes_to_f64(const void* __restrict__ planes, int tf32, int64_t nvec, int d, int dp,
                                int grid_level, int R, double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nvec * d;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v0 = t / d;
    const int j = (int)(t - v0 * d);
    const int64_t v = plane_row(v0, grid_level, R);
    double x;
    if (tf32) {
      const float* p = (const float*)planes;
      x = (double)p[v * dp + j] + (double)p[nvec * dp + v * dp + j];
    } else {
      const __nv_bfloat16* p = (const __nv_bfloat16*)planes;
      x = (double)__bfloat162float(p[v * dp + j]) + (double)__bfloat162float(p[nvec * dp + v * dp + j]);
    }
    out[t] = x;
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

}  // namespace

eifmm_status build_kd_image(Ops* ops, bool tf32, cudaStream_t s) {
  for (int k = 2; k <= ops->depth; ++k) {
    LevelOps& v = ops->lv[k];
    if (v.kd_img_tf32 == (int)tf32) continue;
    dfree(v.kd_img);
    v.kd_img = nullptr;
    v.kd_img_tf32 = -1;
    if (v.dp > kMaxDpTc) continue;  // the SIMT path serves these levels
    const size_t bytes = (size_t)kNumSlots * 2 * v.dp * (size_t)(v.dp * (tf32 ? 4 : 2));
    EIFMM_TRY(dmalloc(&v.kd_img, bytes));
    const int nchunk = v.dp * (tf32 ? 4 : 2) / 128;
    k_build_img<<<dim3(grid_for((int64_t)nchunk * v.dp * 8, 256, 64), kNumSlots), 256, 0, s>>>(
        v.kdT, v.d, v.dp, tf32 ? 1 : 0, (unsigned char*)v.kd_img);
    EIFMM_CHECK_LAUNCH();
    v.kd_img_tf32 = tf32 ? 1 : 0;
  }
  EIFMM_CUDA(cudaStreamSynchronize(s));
  return EIFMM_OK;
}

eifmm_status alloc_mixed_workspace(Tree* t, const Ops* ops, int R) {
  Workspace& ws = t->ws;
  const int kap = t->depth;
  for (int k = 2; k <= kap; ++k) {
    const int dp = ops->lv[k].dp;
    const size_t n = (size_t)nboxes(k) * R * dp;
    EIFMM_TRY(dalloc(&ws.W32[k], n));
    EIFMM_TRY(dalloc(&ws.g32[k], n));
    if (k == 2) ws.l32[k] = ws.g32[k];
    else EIFMM_TRY(dalloc(&ws.l32[k], n));
    EIFMM_TRY(dmalloc(&ws.wa[k], 2 * n * 4));
    // TMA-tiled M2L when the rhs count has a tile shape: planes on the
    // per-class grid, one tensor map per plane
    int bx, by, bz;
    ws.wa_grid[k] = false;
    const bool tf32 = ops->tier == 1;
    if (ops->tier <= 1 && ops->lv[k].dp <= kMaxDpTc && m2l_tma_block(R, &bx, &by, &bz)) {
      const size_t plane = n * (tf32 ? 4 : 2);
      EIFMM_TRY(make_plane_map(ws.tmap[k][0], ws.wa[k], k, R, dp, tf32));
      EIFMM_TRY(make_plane_map(ws.tmap[k][1], (char*)ws.wa[k] + plane, k, R, dp, tf32));
      ws.wa_grid[k] = true;
    }
  }
  EIFMM_TRY(dalloc(&ws.lh32, (size_t)nboxes(kap) * R * ops->lv[kap].dp));
  {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    size_t need = 0;
    for (int k = 2; k <= kap; ++k) {
      const int64_t rows = nboxes(k) * R;
      const int64_t tiles = (nboxes(k) / 8 * R + 127) / 128;
      const int G = m2l_tc_groups(tiles * 8, nsm, ops->lv[k].dp);
      if (G > 1) need = std::max(need, (size_t)G * rows * ops->lv[k].dp);
    }
    if (need) EIFMM_TRY(dalloc(&ws.m2l_part, need));
  }
  if (!ws.err) {
    EIFMM_TRY(dalloc(&ws.err, 1));
    EIFMM_CUDA(cudaMemset(ws.err, 0, sizeof(int)));
    EIFMM_CUDA(cudaMallocHost(&ws.err_host, sizeof(int)));
    *ws.err_host = 0;
  }
  return EIFMM_OK;
}

template <int KERN, int RCT, bool ACC>
static void p2p_launch(const Tree* t, int kern, const float* sig32, int R, double* fnear, float two_l,
                       cudaStream_t s) {
  const PointSet& T = t->tgt;
  const PointSet& S = t->src;
  const unsigned grid = (unsigned)((T.n_nonempty + P2P_WARPS - 1) / P2P_WARPS);
  k_p2p32<KERN, RCT, ACC><<<grid, 32 * P2P_WARPS, 0, s>>>(
      kern, T.nonempty, T.n_nonempty, T.leaf_off, T.lx, T.ly, T.lz, T.n, S.leaf_off, S.lx, S.ly, S.lz,
      sig32, S.n, R, t->depth, two_l, t->exclude_self, fnear);
}

eifmm_status launch_p2p32(const Tree* t, int kern, const float* sig32, int R, double* fnear,
                          cudaStream_t s, bool accurate) {
  if (t->tgt.n_nonempty == 0) return EIFMM_OK;
  const float two_l = (float)(t->L * ldexp(1.0, -t->depth));
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

eifmm_status eval_mixed(Tree* t, const Ops* ops, const double* sigma, int64_t ld_sigma, int R,
                        double* f, int64_t ld_f, cudaStream_t s) {
  if (ops->tier == 2) return eval_fp64(t, ops, sigma, ld_sigma, R, f, ld_f, s, true);
  Workspace& ws = t->ws;
  if (*ws.err_host != 0) {
    const int code = *ws.err_host;
    *ws.err_host = 0;
    cudaMemsetAsync(ws.err, 0, sizeof(int), s);
    set_error("eifmm_evaluate: a bounded device wait of the previous call timed out (code " +
              std::to_string(code) + ")");
    return EIFMM_ETIMEOUT;
  }
  const bool tf32 = ops->tier == 1;
  const int kap = t->depth;
  const int kern = (int)ops->kern;
  const PointSet& S = t->src;
  const PointSet& T = t->tgt;
  record(ws, 0, s);
  EIFMM_TRY(launch_gather_sigma(sigma, ld_sigma, S, R, ws.sig, ws.sig32, s));
  EIFMM_CUDA(cudaEventRecord(ws.ev_fork, s));
  EIFMM_CUDA(cudaStreamWaitEvent(ws.side, ws.ev_fork, 0));
  EIFMM_TRY(launch_p2p32(t, kern, ws.sig32, R, ws.fnear, ws.side, ops->tier >= 1));
  EIFMM_CUDA(cudaEventRecord(ws.ev_join, ws.side));

  // step 1 (every leaf, empty ones get zeros)
  const LevelOps& vl = ops->lv[kap];
  if (kern == EIFMM_KERNEL_INV_R)
    k_p2m32<EIFMM_KERNEL_INV_R><<<(unsigned)nboxes(kap), TPB, 0, s>>>(
        kern, S.leaf_off, S.lx, S.ly, S.lz, ws.sig32, S.n, R, vl.X32, vl.d, vl.dp, ws.W32[kap]);
  else
    k_p2m32<-1><<<(unsigned)nboxes(kap), TPB, 0, s>>>(kern, S.leaf_off, S.lx, S.ly, S.lz, ws.sig32,
                                                      S.n, R, vl.X32, vl.d, vl.dp, ws.W32[kap]);
  EIFMM_CHECK_LAUNCH();
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
    EIFMM_TRY(launch_xfer_gemm(x, s));
  }
  record(ws, 2, s);
  // step 3: What = Delta W (Gamma z = W, then B^t What = z), written as the
  // two M2L operand planes
  {
    DeltaBatch b;
    for (int k = 2; k <= kap; ++k) {
      const LevelOps& v = ops->lv[k];
      const int gl = ws.wa_grid[k] ? k : -1;
      b.lv[b.nlev++] = tf32 ? delta_level(v.d, delta_ops64(v), false, ws.W32[k], v.dp, nullptr, v.dp, ws.wa[k],
                                          nboxes(k) * R, gl, R)
                            : delta_level(v.d, delta_ops32(v), false, ws.W32[k], v.dp, nullptr, v.dp, ws.wa[k],
                                          nboxes(k) * R, gl, R);
    }
    if (tf32) EIFMM_TRY((launch_delta_batch<double, float, float, 2>(b, false, s)));
    else EIFMM_TRY((launch_delta_batch<float, float, float, 1>(b, false, s)));
  }
  record(ws, 3, s);
  // step 4
  for (int k = 2; k <= kap; ++k) {
    if (timing_enabled()) cudaEventRecord(ws.ev_m2l[k], s);
    const LevelOps& v = ops->lv[k];
    if (v.kd_img == nullptr || v.kd_img_tf32 != (int)tf32) {
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
    {
      int dev = 0, nsm = 148;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      a.groups = m2l_tc_groups((a.nbox / 8 * R + 127) / 128 * 8, nsm, a.dp);
      a.part = ws.m2l_part;
    }
    if (ws.wa_grid[k]) EIFMM_TRY(launch_m2l_tma(a, ws.tmap[k][0], ws.tmap[k][1], tf32, s));
    else EIFMM_TRY(launch_m2l_tc(a, tf32, s));
  }
  if (timing_enabled()) cudaEventRecord(ws.ev_m2l[kap + 1], s);
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
    EIFMM_TRY(launch_xfer_gemm(x, s));
  }
  record(ws, 5, s);
  // step 6: lhat = Delta^t l (B z = l, then Gamma^t lhat = z)
  {
    DeltaBatch b;
    b.nlev = 1;
    if (tf32) {
      b.lv[0] = delta_level(vl.d, delta_ops64(vl), true, ws.l32[kap], vl.dp, ws.lh32, vl.dp, nullptr,
                            nboxes(kap) * R);
      EIFMM_TRY((launch_delta_batch<double, float, float, 0>(b, true, s)));
    } else {
      b.lv[0] = delta_level(vl.d, delta_ops32(vl), true, ws.l32[kap], vl.dp, ws.lh32, vl.dp, nullptr,
                            nboxes(kap) * R);
      EIFMM_TRY((launch_delta_batch<float, float, float, 0>(b, true, s)));
    }
  }
  record(ws, 6, s);
  EIFMM_CUDA(cudaStreamWaitEvent(s, ws.ev_join, 0));
  record(ws, 7, s);
  if (T.n_nonempty > 0) {
    const size_t sm = (size_t)(3 * vl.d + RC * vl.d) * sizeof(float);
    if (kern == EIFMM_KERNEL_INV_R)
      k_l2p32<EIFMM_KERNEL_INV_R><<<T.n_nonempty, TPB, sm, s>>>(
          kern, T.nonempty, T.leaf_off, T.perm, T.lx, T.ly, T.lz, T.n, R, vl.X32, vl.d, vl.dp,
          ws.lh32, ws.fnear, ws.ffar, f, ld_f);
    else
      k_l2p32<-1><<<T.n_nonempty, TPB, sm, s>>>(kern, T.nonempty, T.leaf_off, T.perm, T.lx, T.ly,
                                                T.lz, T.n, R, vl.X32, vl.d, vl.dp, ws.lh32, ws.fnear,
                                                ws.ffar, f, ld_f);
    EIFMM_CHECK_LAUNCH();
  }
  EIFMM_CUDA(cudaMemcpyAsync(ws.err_host, ws.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  record(ws, 8, s);
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
    k_planes_to_f64<<<grid_for(cnt, 256), 256>>>(ws.wa[level], ws.tier == 1, nvec, v.d, v.dp,
                                                 ws.wa_grid[level] ? level : -1, ws.nrhs, tmp);
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
