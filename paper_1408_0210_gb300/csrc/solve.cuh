// solve.cuh -- the Delta applications of Algorithm 3 (steps 3 and 6) as two
// triangular sweeps (Section 4.1: Delta = B^-t Gamma^-1 applied by solving
// with Gamma and with B^t rather than through an explicit inverse).
//
//   Delta v   : Gamma z = v (forward, columns of Gamma), B^t w = z (backward,
//               rows of B)
//   Delta^t v : B z = v (forward, columns of B), Gamma^t w = z (backward, rows
//               of Gamma)
//
// One sweep per launch: the packed triangle of one matrix (d(d+1)/2 entries)
// is staged once in shared memory and reused by every warp of the CTA; each
// warp runs the substitution of one vector at a time (lanes own strided
// entries, one __syncwarp per column), grid-striding over the vectors.
#pragma once
#include "internal.h"

namespace eifmm {

constexpr int kSolveWarps = 8;

// Packed layouts (diagonal always stored; ignored for the unit B):
//   column-packed: column k holds rows k..d-1 at offset k*d - k*(k-1)/2
//   row-packed:    row k holds columns 0..k at offset k*(k+1)/2
__host__ __device__ inline int64_t colp_off(int k, int d) { return (int64_t)k * d - (int64_t)k * (k - 1) / 2; }
__host__ __device__ inline int64_t rowp_off(int k) { return (int64_t)k * (k + 1) / 2; }

inline size_t solve_smem_bytes(int d, size_t elem) {
  return ((size_t)d * (d + 1) / 2 + (size_t)kSolveWarps * d) * elem;
}

// FWD: for k = 0..d-1: z_k = v_k (/ M_kk if DIAG); v_j -= M_jk z_k, j > k.
// BWD: for k = d-1..0: w_k = v_k (/ M_kk if DIAG); v_j -= M_kj w_k, j < k.
// Input `in` (element type Ti, row stride ldi), output `out` (To, ldo): the
// entries d..ldo-1 of each output row are written as zeros.  When PLANES is
// 1 or 2 the result is written as the two M2L operand planes (BF16 or TF32
// hi + lo) of `planes` instead.
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

template <typename T, bool FWD, bool DIAG, typename Ti, typename To, int PLANES>
__global__ void __launch_bounds__(32 * kSolveWarps)
k_tri_sweep(int d, const T* __restrict__ Mp, const Ti* __restrict__ in, int ldi,
            To* __restrict__ out, int ldo, void* __restrict__ planes, int64_t nvec, int grid_level,
            int R) {
  extern __shared__ unsigned char s_raw[];
  T* sM = (T*)s_raw;
  const int64_t np = (int64_t)d * (d + 1) / 2;
  for (int64_t t = threadIdx.x; t < np; t += blockDim.x) sM[t] = Mp[t];
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* sv = sM + np + (int64_t)w * d;
  for (int64_t v = (int64_t)blockIdx.x * kSolveWarps + w; v < nvec;
       v += (int64_t)gridDim.x * kSolveWarps) {
    for (int j = lane; j < d; j += 32) sv[j] = (T)in[v * ldi + j];
    __syncwarp();
    if (FWD) {
      for (int k = 0; k < d; ++k) {
        const T* col = sM + colp_off(k, d);  // col[j - k] = M_jk
        const T zk = DIAG ? sv[k] / col[0] : sv[k];
        __syncwarp();
        if (DIAG && lane == 0) sv[k] = zk;
        for (int j = k + 1 + lane; j < d; j += 32) sv[j] -= col[j - k] * zk;
        __syncwarp();
      }
    } else {
      for (int k = d - 1; k >= 0; --k) {
        const T* row = sM + rowp_off(k);  // row[j] = M_kj
        const T wk = DIAG ? sv[k] / row[k] : sv[k];
        __syncwarp();
        if (DIAG && lane == 0) sv[k] = wk;
        for (int j = lane; j < k; j += 32) sv[j] -= row[j] * wk;
        __syncwarp();
      }
    }
    if (PLANES == 0) {
      for (int j = lane; j < ldo; j += 32) out[v * ldo + j] = j < d ? (To)sv[j] : (To)0;
    } else {
      const int64_t prow = plane_row(v, grid_level, R);
      for (int j = lane; j < ldo; j += 32) {
        const T x = j < d ? sv[j] : (T)0;
        if (PLANES == 1) {
          __nv_bfloat16* pl = (__nv_bfloat16*)planes;
          const __nv_bfloat16 hi = __float2bfloat16_rn((float)x);
          const __nv_bfloat16 lo = __float2bfloat16_rn((float)(x - (T)__bfloat162float(hi)));
          pl[prow * ldo + j] = hi;
          pl[nvec * ldo + prow * ldo + j] = lo;
        } else {
          float* pl = (float*)planes;
          const float hi = tf32_rn((float)x);
          const float lo = tf32_rn((float)(x - (T)hi));
          pl[prow * ldo + j] = hi;
          pl[nvec * ldo + prow * ldo + j] = lo;
        }
      }
    }
    __syncwarp();
  }
}

template <typename T, bool FWD, bool DIAG, typename Ti, typename To, int PLANES>
eifmm_status launch_tri_sweep(int d, const T* Mp, const Ti* in, int ldi, To* out, int ldo,
                              void* planes, int64_t nvec, cudaStream_t s, int grid_level = -1,
                              int R = 1) {
  static bool attr = false;
  const size_t sm = solve_smem_bytes(d, sizeof(T));
  if (!attr) {
    EIFMM_CUDA(cudaFuncSetAttribute(k_tri_sweep<T, FWD, DIAG, Ti, To, PLANES>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr = true;
  }
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = (int)((200 * 1024) / (sm > 0 ? sm : 1));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2048 / (32 * kSolveWarps)) per_sm = 2048 / (32 * kSolveWarps);
  int64_t blocks = (nvec + kSolveWarps - 1) / kSolveWarps;
  if (blocks > (int64_t)nsm * per_sm) blocks = (int64_t)nsm * per_sm;
  k_tri_sweep<T, FWD, DIAG, Ti, To, PLANES><<<(unsigned)blocks, 32 * kSolveWarps, sm, s>>>(
      d, Mp, in, ldi, out, ldo, planes, nvec, grid_level, R);
  EIFMM_CHECK_LAUNCH();
  return EIFMM_OK;
}

}  // namespace eifmm
