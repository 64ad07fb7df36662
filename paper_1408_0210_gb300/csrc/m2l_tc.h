// m2l_tc.h -- launcher of the tensor-core M2L (step 4 of Algorithm 3).
#pragma once
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
eifmm_status make_plane_map(void* map, void* base, int level, int R, int dp, bool tf32, int rows = 128);
eifmm_status launch_m2l_tma(const M2LTcArgs& a, const void* map0, const void* map1, bool tf32,
                            cudaStream_t s);
eifmm_status launch_m2l_tc(const M2LTcArgs& a, bool tf32, cudaStream_t s);
// Transposed variant (dp = 128): M = 128 (m'), N = 256 target rows per MMA.
eifmm_status launch_m2l_t256(const M2LTcArgs& a, const void* map0, const void* map1, bool tf32,
                             cudaStream_t s);

}  // namespace eifmm
