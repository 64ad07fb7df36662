// solve.cuh -- the Delta applications of Algorithm 3 (steps 3 and 6) as two
// triangular solves (Section 4.1: Delta = B^-t Gamma^-1 is applied by solving
// with Gamma and with B^t rather than through an explicit inverse).
//
//   Delta v   : Gamma z = v (lower, forward), B^t w = z (upper, backward)
//   Delta^t v : B z = v (lower, forward),     Gamma^t w = z (upper, backward)
//
// Both solves of one application run in one kernel.  A warp owns
// kDeltaVpw = 16 vectors, kDeltaLpv = 2 lanes per vector, kept transposed in
// shared memory ([entry][vector], row stride 17 so that both the transposing
// copy and the lane-wise access are free of bank conflicts).  Each solve
// walks 32-row blocks (blocked left-looking substitution): lane half h
// holds rows 16h .. 16h+15 of the block in registers, every earlier block
// contributes a dense 32 x 32 tile product (16 FMAs per lane for each solved
// entry read back from shared memory), and the diagonal 32 x 32 block is
// solved in registers, each solved entry passed from its owner to the other
// half by a shuffle.  The tile entries are broadcast loads, so there is no
// synchronisation inside a solve: the cost is the d^2/2 FMAs per vector and
// solve.  (At the 1M-point leaf level: 66 us with one lane per vector, 63
// with two, 68 with four.)
//
// The backward (upper) solve is run as a forward solve in reversed entry
// order: with p(a) = dpad-1-a, U w = z becomes L' w' = z' with
// L'[a][b] = U[p(a)][p(b)] lower triangular; the host stores L' tiles and
// the kernel maps logical to physical entries.
#pragma once
#include <type_traits>

#include "internal.h"

namespace eifmm {

constexpr int kDeltaTile = 32;
constexpr int kDeltaLpv = 2;                    // lanes per vector
constexpr int kDeltaVpw = 32 / kDeltaLpv;       // vectors per warp
constexpr int kDeltaRl = kDeltaTile / kDeltaLpv;  // rows of a block per lane
constexpr int kDeltaLd = kDeltaVpw + 1;         // shared row stride (floats or doubles)
constexpr int kDeltaMaxWarps = 8;               // warps per CTA

// Tiles of one solve: tile (J, K), K <= J, at (J(J+1)/2 + K) * 1024, entry
// [k][i] = L'[32J + i][32K + k]; the diagonal tiles are zero on and above
// the diagonal.  Pivots: FP32 stores 1/L'[a][a], FP64 stores L'[a][a].
inline int64_t delta_tiles_elems(int d) {
  const int nb = (d + kDeltaTile - 1) / kDeltaTile;
  return (int64_t)nb * (nb + 1) / 2 * kDeltaTile * kDeltaTile;
}

__device__ __forceinline__ float tf32_rn(float v) {
  uint32_t u = __float_as_uint(v);
  u = (u + 0x1000u) & ~0x1FFFu;
  return __uint_as_float(u);
}

// Destination row of vector v = box * R + r in the What planes: Morton order,
// or (grid_level >= 0) the per-parity-class grid [class][Z][Y][X*R + r] of
// that level read by the TMA M2L.
__device__ __forceinline__ int64_t plane_row(int64_t v, int grid_level, int R) {
  if (grid_level < 0) return v;
  const int64_t box = v / R;
  const int r = (int)(v - box * R);
  int c[3];
  morton_decode(box, grid_level, c);
  const int64_t h = (int64_t)1 << (grid_level - 1);
  const int cls = (int)(box & 7);
  return ((((int64_t)cls * h + (c[2] >> 1)) * h + (c[1] >> 1)) * h + (c[0] >> 1)) * R + r;
}

// acc[i] -= col[i] * z for the lane's rows of one tile column (16-byte
// loads of a half-warp-uniform address: shared memory when SH, else global
// through L1).
template <bool SH>
__device__ __forceinline__ void tile_col_update(float (&acc)[kDeltaRl], const float* __restrict__ col,
                                                float z) {
#pragma unroll
  for (int q = 0; q < kDeltaRl / 4; ++q) {
    const float4 m = SH ? reinterpret_cast<const float4*>(col)[q] : __ldg(reinterpret_cast<const float4*>(col) + q);
    acc[4 * q + 0] -= m.x * z;
    acc[4 * q + 1] -= m.y * z;
    acc[4 * q + 2] -= m.z * z;
    acc[4 * q + 3] -= m.w * z;
  }
}
template <bool SH>
__device__ __forceinline__ void tile_col_update(double (&acc)[kDeltaRl], const double* __restrict__ col,
                                                double z) {
#pragma unroll
  for (int q = 0; q < kDeltaRl / 2; ++q) {
    const double2 m =
        SH ? reinterpret_cast<const double2*>(col)[q] : __ldg(reinterpret_cast<const double2*>(col) + q);
    acc[2 * q + 0] -= m.x * z;
    acc[2 * q + 1] -= m.y * z;
  }
}

__device__ __forceinline__ float apply_pivot(float v, float rp) { return v * rp; }
__device__ __forceinline__ double apply_pivot(double v, double p) { return v / p; }

// One forward solve L' x = v over the warp's kDeltaVpw vectors held in sz
// (physical entry e of vector c at sz[e * kDeltaLd + c]); lane = c + kDeltaVpw h
// works on rows kDeltaRl h .. of every block.  REV maps logical entry a to
// physical dpad-1-a.  The solution overwrites sz.
template <typename T, bool DIAG, bool REV, bool SH>
__device__ __forceinline__ void tiled_solve(T* __restrict__ sz, int nb, const T* __restrict__ tiles,
                                            const T* __restrict__ piv, int lane) {
  constexpr int TL = kDeltaTile, RL = kDeltaRl;
  const int c = lane % kDeltaVpw, h = lane / kDeltaVpw;
  for (int J = 0; J < nb; ++J) {
    const int pj = REV ? nb - 1 - J : J;
    T acc[RL];
#pragma unroll
    for (int i = 0; i < RL; ++i) {
      const int row = h * RL + i;
      acc[i] = sz[(pj * TL + (REV ? TL - 1 - row : row)) * kDeltaLd + c];
    }
    const T* tJ = tiles + (int64_t)(J * (J + 1) / 2) * TL * TL;
    for (int K = 0; K < J; ++K) {
      const T* tk = tJ + (int64_t)K * TL * TL + h * RL;
      const T* zK = sz + (REV ? (nb - 1 - K) * TL + TL - 1 : K * TL) * kDeltaLd + c;
#pragma unroll
      for (int k = 0; k < TL; ++k) {
        const T zk = zK[(REV ? -k : k) * kDeltaLd];
        tile_col_update<SH>(acc, tk + k * TL, zk);
      }
    }
    const T* td = tJ + (int64_t)J * TL * TL;
#pragma unroll
    for (int k = 0; k < TL; ++k) {
      const int owner = k / RL;  // the half that holds entry k
      T mine = acc[k % RL];
      if (DIAG && h == owner) mine = apply_pivot(mine, __ldg(piv + J * TL + k));
      const T zk = kDeltaLpv == 1 ? mine : __shfl_sync(0xffffffffu, mine, c + owner * kDeltaVpw);
      if (h == owner) acc[k % RL] = zk;
      // the tile holds zeros on and above its diagonal, so the update of
      // every row leaves the rows up to k as they are
      tile_col_update<SH>(acc, td + k * TL + h * RL, zk);
    }
#pragma unroll
    for (int i = 0; i < RL; ++i) {
      const int row = h * RL + i;
      sz[(pj * TL + (REV ? TL - 1 - row : row)) * kDeltaLd + c] = acc[i];
    }
  }
}

// One level of a batched application: vectors `in` (row v at v * ldi, d
// entries) -> rows of `out` (ldo; entries d..ldo-1 written as zeros) or the
// two M2L operand planes at plane_row(v).  Blocks block0.. serve this level.
struct DeltaLevel {
  const void* t1 = nullptr;  // tiles and pivots of the first solve
  const void* p1 = nullptr;
  const void* t2 = nullptr;  // and of the second (reversed) solve
  const void* p2 = nullptr;
  const void* in = nullptr;
  void* out = nullptr;
  void* planes = nullptr;
  int64_t nvec = 0;
  int d = 0, nb = 0, ldi = 0, ldo = 0, grid_level = -1, R = 1;
  int block0 = 0;
};
struct DeltaBatch {
  DeltaLevel lv[kMaxLevel + 1];
  int nlev = 0;
};

__device__ __forceinline__ void copy_tiles(void* dst, const void* src, int64_t bytes) {
  const int4* s4 = (const int4*)src;
  int4* d4 = (int4*)dst;
  for (int64_t i = threadIdx.x; i < bytes / 16; i += blockDim.x) d4[i] = __ldg(s4 + i);
}

// out = M2^-1 M1^-1 in, both solves in one pass over the vectors.  SH: the
// tiles of the running solve are staged in shared memory (one copy per CTA,
// read by all its warps); otherwise they are read through L1.
template <typename T, bool DIAG1, bool DIAG2, typename Ti, typename To, int PLANES, bool SH>
__global__ void __launch_bounds__(32 * kDeltaMaxWarps)
k_delta(const __grid_constant__ DeltaBatch b) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  int li = 0;
  while (li + 1 < b.nlev && (int)blockIdx.x >= b.lv[li + 1].block0) ++li;
  const DeltaLevel& L = b.lv[li];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = L.nb, d = L.d;
  const int dpad = nb * kDeltaTile;
  const int64_t tile_elems = (int64_t)nb * (nb + 1) / 2 * kDeltaTile * kDeltaTile;
  T* s_tiles = reinterpret_cast<T*>(s_raw);
  T* sz = s_tiles + (SH ? tile_elems : 0) + (int64_t)w * dpad * kDeltaLd;
  const int64_t v0 = ((int64_t)(blockIdx.x - L.block0) * (blockDim.x >> 5) + w) * kDeltaVpw;
  const int64_t nvec = L.nvec;
  const bool live = v0 < nvec;
  const Ti* __restrict__ in = (const Ti*)L.in;
  if (live) {
    // transposing load: row v0+vv -> column vv (four rows' loads in flight
    // before their shared stores)
    for (int vv0 = 0; vv0 < kDeltaVpw; vv0 += 4) {
      for (int j = lane; j < dpad; j += 32) {
        T x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t v = v0 + vv0 + u;
          x[u] = (v < nvec && j < d) ? (T)__ldg(in + v * L.ldi + j) : (T)0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) sz[j * kDeltaLd + vv0 + u] = x[u];
      }
    }
  }
  const T* t1 = (const T*)L.t1;
  const T* t2 = (const T*)L.t2;
  if (SH) {
    copy_tiles(s_tiles, t1, tile_elems * (int64_t)sizeof(T));
    __syncthreads();
    t1 = s_tiles;
  } else {
    __syncwarp();
  }
  if (live) tiled_solve<T, DIAG1, false, SH>(sz, nb, t1, (const T*)L.p1, lane);
  if (SH) {
    __syncthreads();
    copy_tiles(s_tiles, t2, tile_elems * (int64_t)sizeof(T));
    __syncthreads();
    t2 = s_tiles;
  }
  if (!live) return;
  tiled_solve<T, DIAG2, true, SH>(sz, nb, t2, (const T*)L.p2, lane);
  __syncwarp();
  To* out = (To*)L.out;
  const int ldo = L.ldo;
  for (int vv = 0; vv < kDeltaVpw; ++vv) {
    const int64_t v = v0 + vv;
    if (v >= nvec) break;
    if (PLANES == 0) {
      for (int j = lane; j < ldo; j += 32) out[v * ldo + j] = j < d ? (To)sz[j * kDeltaLd + vv] : (To)0;
    } else {
      const int64_t prow = plane_row(v, L.grid_level, L.R);
      for (int j = lane; j < ldo; j += 32) {
        const T x = j < d ? sz[j * kDeltaLd + vv] : (T)0;
        if (PLANES == 1) {
          __nv_bfloat16* pl = (__nv_bfloat16*)L.planes;
          const __nv_bfloat16 hi = __float2bfloat16_rn((float)x);
          const __nv_bfloat16 lo = __float2bfloat16_rn((float)(x - (T)__bfloat162float(hi)));
          pl[prow * ldo + j] = hi;
          pl[nvec * ldo + prow * ldo + j] = lo;
        } else {
          float* pl = (float*)L.planes;
          const float hi = tf32_rn((float)x);
          const float lo = tf32_rn((float)(x - (T)hi));
          pl[prow * ldo + j] = hi;
          pl[nvec * ldo + prow * ldo + j] = lo;
        }
      }
    }
  }
}

// Tiled operands of one level in precision T: [0] Gamma, [1] B^t reversed
// (Delta); [2] B, [3] Gamma^t reversed (Delta^t); pivots [0] of Gamma,
// [1] of Gamma^t reversed.
template <typename T>
struct DeltaOps {
  const T* tiles[4];
  const T* piv[2];
};
inline DeltaOps<double> delta_ops64(const LevelOps& v) {
  return {{v.dt64[0], v.dt64[1], v.dt64[2], v.dt64[3]}, {v.piv64[0], v.piv64[1]}};
}
inline DeltaOps<float> delta_ops32(const LevelOps& v) {
  return {{v.dt32[0], v.dt32[1], v.dt32[2], v.dt32[3]}, {v.piv32[0], v.piv32[1]}};
}

// One level's entry of a batch (Delta, or Delta^t when `transpose`).
template <typename T>
DeltaLevel delta_level(int d, const DeltaOps<T>& op, bool transpose, const void* in, int ldi, void* out,
                       int ldo, void* planes, int64_t nvec, int grid_level = -1, int R = 1) {
  DeltaLevel L;
  L.t1 = op.tiles[transpose ? 2 : 0];
  L.p1 = transpose ? nullptr : op.piv[0];
  L.t2 = op.tiles[transpose ? 3 : 1];
  L.p2 = transpose ? op.piv[1] : nullptr;
  L.in = in; L.out = out; L.planes = planes;
  L.nvec = nvec; L.d = d; L.nb = (d + kDeltaTile - 1) / kDeltaTile;
  L.ldi = ldi; L.ldo = ldo; L.grid_level = grid_level; L.R = R;
  return L;
}

template <auto KFN>
eifmm_status delta_launch(const DeltaBatch& b, int blocks, int warps, size_t sm, cudaStream_t s) {
  constexpr int kDev = 64;
  static bool attr[kDev] = {};  // the attribute is per device
  int dev = 0;
  EIFMM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kDev || !attr[dev]) {
    EIFMM_CUDA(cudaFuncSetAttribute(KFN, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    if (dev >= 0 && dev < kDev) attr[dev] = true;
  }
  KFN<<<(unsigned)blocks, 32 * warps, sm, s>>>(b);
  EIFMM_CHECK_LAUNCH();
  return EIFMM_OK;
}

// All levels of `b` in one launch (Delta if !transpose, else Delta^t).  The
// warps per CTA and the staging of the tiles follow the largest level.
template <typename T, typename Ti, typename To, int PLANES>
eifmm_status launch_delta_batch(DeltaBatch& b, bool transpose, cudaStream_t s) {
  int nbmax = 0;
  for (int i = 0; i < b.nlev; ++i) nbmax = b.lv[i].nvec > 0 && b.lv[i].nb > nbmax ? b.lv[i].nb : nbmax;
  if (nbmax == 0) return EIFMM_OK;
  const size_t per_warp = (size_t)nbmax * kDeltaTile * kDeltaLd * sizeof(T);
  const size_t tiles = (size_t)nbmax * (nbmax + 1) / 2 * kDeltaTile * kDeltaTile * sizeof(T);
  const size_t cap = 227 * 1024;
  bool sh = tiles + per_warp <= cap;
  int warps = kDeltaMaxWarps;
  while (warps > 1 && (sh ? tiles : 0) + warps * per_warp > cap) --warps;
  if ((sh ? tiles : 0) + warps * per_warp > cap) {
    set_error("Delta application: d too large for one warp's vectors in shared memory");
    return EIFMM_EUNSUPPORTED;
  }
  int blocks = 0;
  for (int i = 0; i < b.nlev; ++i) {
    b.lv[i].block0 = blocks;
    const int64_t nw = (b.lv[i].nvec + kDeltaVpw - 1) / kDeltaVpw;
    blocks += (int)((nw + warps - 1) / warps);
  }
  if (blocks == 0) return EIFMM_OK;
  const size_t sm = (sh ? tiles : 0) + warps * per_warp;
  if (!transpose)
    return sh ? delta_launch<k_delta<T, true, false, Ti, To, PLANES, true>>(b, blocks, warps, sm, s)
              : delta_launch<k_delta<T, true, false, Ti, To, PLANES, false>>(b, blocks, warps, sm, s);
  return sh ? delta_launch<k_delta<T, false, true, Ti, To, PLANES, true>>(b, blocks, warps, sm, s)
            : delta_launch<k_delta<T, false, true, Ti, To, PLANES, false>>(b, blocks, warps, sm, s);
}

}  // namespace eifmm
