// m2l_tc.h -- launcher of the tensor-core M2L (step 4 of Algorithm 3).
#pragma once
#include <cmath>

#include "internal.h"

namespace eifmm {

struct M2LTcArgs {
  int level;
  int64_t nbox;          // 8^level
  int R;                 // right-hand sides; rows = nbox * R
  int64_t rows;
  int dp;                // padded rank (multiple of 64), <= kMaxDpTc
  int tmem_cols;         // power of two >= dp
  const void* wa;        // A planes [2][rows][dp] (BF16 or TF32 bit patterns)
  const void* kd_img;    // B image [343][dp*esz/128][2][dp rows x 128 B], swizzled
  const int* slot_lists; // [8][189]
  float* g;              // [rows][dp] FP32 output
  int* err;              // device error word (0 = ok)
  int groups = 1;        // CTAs sharing one tile, each over 189/groups offsets
  float* part = nullptr; // [groups][rows][dp] partial sums when groups > 1
  // set by the launcher
  float* out = nullptr;
  int64_t part_stride = 0;
  int stages = 2;
  int chains = 1;        // accumulators in TMEM (round-robin over offsets)
  int h = 0;             // TMA variant: boxes per axis per parity class
  int bx = 0, by = 0, bz = 0;  // TMA variant: tile block
};

constexpr int kMaxDpTc = 320;
size_t m2l_tc_smem_bytes(int dp, bool tf32);
int m2l_tc_groups(int64_t tiles8, int nsm, int dp);
bool m2l_tma_block(int R, int* bx, int* by, int* bz);
bool m2l_t256_block(int R, int* bx, int* by, int* bz);
int m2l_t256_groups(int64_t ctas, int nsm);
int64_t m2l_t256_ctas(int level, int R);  // CTAs of one offset group
size_t m2l_t256_smem_bytes();
// Tensor map (a 128-byte CUtensorMap, 64-byte aligned) of one What plane in
// the per-class grid layout [class][Z][Y][X*R + r][dp].
eifmm_status make_plane_map(void* map, void* base, int level, int R, int dp, int fmt, int rows = 128);
eifmm_status launch_m2l_tma(const M2LTcArgs& a, const void* map0, const void* map1, bool tf32,
                            cudaStream_t s);
eifmm_status launch_m2l_tc(const M2LTcArgs& a, bool tf32, cudaStream_t s);
// Stream-K transposed M2L (dp = 128): one CTA per SM over (tile, offset)
// units, split tiles summed by a fix-up kernel (plan: SkPlanDev).
eifmm_status build_sk_plan(int level, int R, int nsm, SkPlanDev* p);
void free_sk_plan(SkPlanDev* p);
eifmm_status launch_m2l_t256s(const M2LTcArgs& a, const void* map0, const void* map1, const SkPlanDev& p,
                              cudaStream_t s);

// FP16 hi + lo planes, per-offset drains (dp in {64, 128, 192, 256}): W
// planes scaled by f16_plane_scale(max |W| of the level) (wmax: the bits of
// that maximum per level), K^delta Delta rows by kscale[m'].
size_t m2l_h16_smem_bytes(int dp);
int64_t m2l_tma_ctas(int level, int R);   // CTAs of one offset group, 128-row tiles
int m2l_h16_groups(int64_t ctas, int nsm);
eifmm_status launch_m2l_h16(const M2LTcArgs& a, const void* map0, const void* map1, const uint32_t* wmax,
                            const float* kscale, cudaStream_t s);

// Power of two s with maxabs * s in [2^14, 2^15): the scale of an FP16
// operand plane whose largest magnitude is maxabs (1 when maxabs is 0).  The
// split x s = hi + lo then keeps hi and lo in FP16's normal range for every
// entry within 2^-24 of the largest.
__host__ __device__ inline float f16_plane_scale(float maxabs) {
  if (!(maxabs > 0.0f) || maxabs > 3.0e38f) return 1.0f;
  int e = 0;
  frexpf(maxabs, &e);  // maxabs = m 2^e, m in [0.5, 1)
  e = 15 - e;
  e = e < -100 ? -100 : (e > 100 ? 100 : e);
  return ldexpf(1.0f, e);
}
// Transposed variant (dp = 128): M = 128 (m'), N = 256 target rows per MMA.
eifmm_status launch_m2l_t256(const M2LTcArgs& a, const void* map0, const void* map1, bool tf32,
                             cudaStream_t s);

}  // namespace eifmm
