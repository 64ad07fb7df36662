// internal.h -- shared declarations of the EIFMM GPU library (sm_103a).
// Not part of the ABI; include/eifmm.h is.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>

#include "../../include/eifmm.h"

namespace eifmm {

constexpr int kMaxLevel = 10;
constexpr int kMaxD = 512;
constexpr int kMaxRhs = 256;
constexpr int kNumSlots = 343;  // 7^3 offsets delta/(2 l_k) in [-3, 3]^3
constexpr int kListLen = 189;   // interaction-list length of an interior box

// ---------------------------------------------------------------- errors --
void set_error(const std::string& msg);
#define EIFMM_CUDA(call)                                                     \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      ::eifmm::set_error(std::string(#call) + ": " + cudaGetErrorString(e_)); \
      return EIFMM_ECUDA;                                                    \
    }                                                                        \
  } while (0)
void count_launch();
#define EIFMM_CHECK_LAUNCH()          \
  do {                                \
    ::eifmm::count_launch();          \
    EIFMM_CUDA(cudaGetLastError());   \
  } while (0)
#define EIFMM_TRY(call)                 \
  do {                                  \
    eifmm_status s_ = (call);           \
    if (s_ != EIFMM_OK) return s_;      \
  } while (0)

eifmm_status dmalloc(void** p, size_t bytes);
template <class T>
eifmm_status dalloc(T** p, size_t count) {
  return dmalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}
void dfree(void* p);

// ------------------------------------------------------------- kernels --
// k(z) in FP64, contracted arithmetic (evaluation path).
__host__ __device__ inline double kern_f64(int kern, double z0, double z1, double z2);

// ------------------------------------------------------------ operators --
struct LevelOps {
  int d = 0;          // EIM rank of the level
  int dp = 0;         // d padded to a multiple of 64 (tensor-core layouts)
  double eps_est = 0;
  double* X = nullptr;     // d x 3, x_m^{I_0^k}
  double* Y = nullptr;     // d x 3, y_l^{J_0^k}
  double* G_rm = nullptr;  // Gamma row-major
  double* B_rm = nullptr;  // B row-major
  double* m2mT = nullptr;  // [8][q < d_{k+1}][m < d]: (K_M2M^i)^t, levels 2..depth-1
  double* l2lT = nullptr;  // [8][q' < d_{k-1}][m' < d]: (K_L2L^i)^t, levels 3..depth
  double* kdT = nullptr;   // [343][l < d][m' < d]: (K^delta Delta)_{m'l}, applied to W
  double* m2m = nullptr;   // [8][m < d][q < d_{k+1}]: K_M2M^i row-major
  double* l2l = nullptr;   // [8][m' < d][q' < d_{k-1}]: K_L2L^i row-major
  float* m2m32 = nullptr;
  float* l2l32 = nullptr;
  float* m2m_cb = nullptr;  // [K_M2M^0 .. K_M2M^7] col-major dp x 8 dp_child, zero-padded (library GEMM)
  float* l2l_cb = nullptr;  // [K_L2L^0; ..; K_L2L^7] col-major 8 dp x dp_parent, zero-padded
  // Delta and Delta^t as tiled triangular solves (solve.cuh): tiles [0]
  // Gamma, [1] B^t reversed, [2] B, [3] Gamma^t reversed; pivots [0] of
  // Gamma, [1] of Gamma^t reversed (FP64: the pivots, FP32: reciprocals)
  double* dt64[4] = {};
  float* dt32[4] = {};
  double* piv64[2] = {};
  float* piv32[2] = {};
  // reduced-precision copies
  float* m2mT32 = nullptr;
  float* l2lT32 = nullptr;
  float* X32 = nullptr;    // d x 3
  // M2L operands of the tensor-core kernel: K^delta split in two planes
  // (hi, lo) in the K-major 128B-swizzled layout,
  // [slot][chunk of 128 B of l][plane][row m' < dp][128 B].
  void* kd_img = nullptr;
  float* kd32 = nullptr;   // [343][l < d][m' < dp] FP32 folded operator (SIMT M2L of tier 2)
  // M2L compression (Section 4.2, first stage), FP64 far field only
  double* U = nullptr;     // d x r row-major: the kept left singular vectors of K_fat
  double* Ct = nullptr;    // [343][l < r][m' < r]: C^delta_{m'l} = (U^t K^delta U)_{m'l}
  int r = 0, r_i = 0, r_ii = 0;     // kept rank and the counts of the two filters
  double s_kept = 0.0, s_next = 0.0;  // last kept and first dropped singular value / s_0
  int kd_img_fmt = -1;     // -1 none, else the PlaneFmt of the image
  float* kscale = nullptr; // [dp] power-of-two scale of row m' (FP16 image)
};

struct Ops {
  eifmm_kernel kern;
  double L = 1.0;
  int depth = 0;
  int tier = 0;        // arithmetic tier of the mixed path
  double calib_err[4] = {-1.0, -1.0, -1.0, -1.0};  // last calibration, per tier
  int calib_tier = -1;
  bool compressed = false;  // the FP64 far field runs the compressed M2L
  double compress_eps = 0.0;
  uint64_t uid = 0;    // unique per loaded operator set: workspaces are keyed on it, not
                       // on the handle's address, which a later load may reuse
  LevelOps lv[kMaxLevel + 1];
  int* d_slot_lists = nullptr;  // [8][189] slot ids per parity class
};

// ------------------------------------------------------------------ tree --
struct PointSet {
  int64_t n = 0;
  void* slab = nullptr;         // one device allocation holding every array below
  int32_t* perm = nullptr;      // sorted position -> input index
  uint32_t* keys = nullptr;     // sorted Morton keys
  int32_t* leaf_off = nullptr;  // 8^depth + 1
  int32_t* nonempty = nullptr;  // non-empty leaves
  int32_t n_nonempty = 0;
  double* x = nullptr;          // sorted coordinates (SoA)
  double* y = nullptr;
  double* z = nullptr;
  float* lx = nullptr;          // coordinates relative to the leaf centre
  float* ly = nullptr;
  float* lz = nullptr;
};

// Device arrays of the stream-K plan of the leaf-level tensor-core M2L.
struct SkPlanDev {
  int* tu = nullptr;        // [ntiles + 1] units (active offsets) before each tile
  int* fix_t = nullptr;     // split tiles
  int* fix_b = nullptr;     // [nfix + 1] their first slot in fix_slot
  int* fix_slot = nullptr;  // partial slots, CTA order
  float* part = nullptr;    // [2 nctas][256][128] partial tiles
  int ntiles = 0, tpc = 0, nctas = 0, nfix = 0;
};
void free_sk_plan(SkPlanDev* p);
eifmm_status wait_selftest(long long limit, int* code);  // m2l_tc.cu

struct Workspace {
  const void* ops_id = nullptr;
  uint64_t ops_uid = 0;
  int nrhs = 0;
  int prec = -1;
  int tier = -1;
  // FP64 far field, [box][r][d] per level
  double* W[kMaxLevel + 1] = {};
  double* Wh[kMaxLevel + 1] = {};
  double* g[kMaxLevel + 1] = {};   // step 4 output
  double* l[kMaxLevel + 1] = {};   // step 5 output (l[2] aliases g[2])
  double* lh = nullptr;            // leaf level
  // FP32 far field
  float* W32[kMaxLevel + 1] = {};
  float* Wh32[kMaxLevel + 1] = {};
  float* g32[kMaxLevel + 1] = {};
  float* l32[kMaxLevel + 1] = {};  // l32[2] aliases g32[2]
  float* lh32 = nullptr;
  // tensor-core M2L A operand planes: [plane][box*R + r][dp] (BF16 or TF32)
  void* wa[kMaxLevel + 1] = {};
  bool wa_grid[kMaxLevel + 1] = {};  // planes in the per-class grid layout (TMA M2L)
  alignas(64) unsigned char tmap[kMaxLevel + 1][2][128] = {};  // CUtensorMap per plane
  // 256-row boxes of the transposed M2L (dp = 128)
  bool wa_t256[kMaxLevel + 1] = {};
  // M2L variant per level set by eifmm_autotune (0: built-in rule, 1:
  // transposed, 2: 128-row, 3: transposed stream-K) and the shift of its
  // offset-group count (groups << shift, or >> -shift)
  int m2l_kind[kMaxLevel + 1] = {};
  int m2l_gshift[kMaxLevel + 1] = {};
  int p2p_sym = 0;  // near-field kernel chosen by eifmm_autotune: 1 pair-symmetric
  size_t m2l_part_cap = 0;  // floats in m2l_part (levels below the leaves)
  float* m2l_part_leaf = nullptr;  // partial sums of the leaf level
  size_t m2l_part_leaf_cap = 0;
  alignas(64) unsigned char tmap2[kMaxLevel + 1][2][128] = {};
  float* m2l_part = nullptr;    // partial M2L sums of the split offset lists
  double* part64 = nullptr;     // the same for the FP64 far field (FP64 and FP32-pair M2L)
  size_t part64_cap = 0;        // doubles in part64
  int nsm = 0;                  // SMs of the workspace's device
  uint32_t* wmax = nullptr;     // [kMaxLevel + 1] bits of max |W| per level (FP16 planes)
  SkPlanDev sk;                 // stream-K plan of the leaf level (tier 0), when it pays
  int* err = nullptr;           // device error word of bounded waits
  int* err_host = nullptr;      // pinned copy, read at the next call
  void* tmp = nullptr;          // intermediate of the two Delta sweeps
  void* blas_ws = nullptr;      // the library GEMMs' workspace of this tree (kXferBlasWorkspace bytes)
  double* sig = nullptr;        // sorted sigma, n_src x R (col-major, ld n_src)
  float* sig32 = nullptr;
  double* fnear = nullptr;      // n_tgt x R, sorted order
  double* ffar = nullptr;       // n_tgt x R, sorted order (debug only)
  float* gsym = nullptr;        // 13 x n: pair-symmetric near-field partials (R = 1, targets = sources)
  double* host_sig = nullptr;   // device staging for evaluate_host
  double* host_f = nullptr;
  size_t host_cap = 0;
  cudaStream_t side = nullptr;  // near field runs here, concurrent with far
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // step 4: the coarse levels run here, concurrent with the leaf level
  cudaStream_t side2 = nullptr;
  cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;
  // the far field of the mixed path runs here at the highest stream priority
  // (side2 too), so the near field, at the default priority, fills the SMs
  // it leaves free
  cudaStream_t hi = nullptr;
  cudaEvent_t ev_hi = nullptr;
  cudaEvent_t ev_t[10] = {};
  cudaEvent_t ev_m2l[kMaxLevel + 2] = {};   // start of the M2L launch of level k
  cudaEvent_t ev_m2le[kMaxLevel + 2] = {};  // and its end (on the stream that ran it)
  cudaEvent_t ev_nf[2] = {};  // the near-field launch on the side stream
  bool evaluated = false;
  float step_ms[20] = {};
};

constexpr int kNumOptions = 6;  // eifmm_option

struct Tree {
  int depth = 0;
  double lo[3] = {0, 0, 0};
  double L = 1.0;
  int exclude_self = 0;
  bool same = false;  // targets are the sources
  PointSet src, tgt;  // tgt aliases src when `same`
  Workspace ws;
  int opt[kNumOptions] = {};  // eifmm_option values (all 0 by default)
};

// ------------------------------------------------------------ launchers --
eifmm_status build_pointset(const double* xyz, int64_t n, const double lo[3],
                            double L, int depth, cudaStream_t s, PointSet* ps);
void free_pointset(PointSet* ps);

eifmm_status assemble_ops(Ops* ops, cudaStream_t s);
void free_ops(Ops* ops);

eifmm_status eval_fp64(Tree* t, const Ops* ops, const double* sigma,
                       int64_t ld_sigma, int R, double* f, int64_t ld_f,
                       cudaStream_t s, bool near32 = false,
                       bool pair_m2l = false);
eifmm_status launch_p2p32(const Tree* t, int kern, const float* sig32, int R,
                          double* fnear, cudaStream_t s, bool accurate, float* gsym = nullptr);
// Element format of the tensor-core M2L operand planes.
enum PlaneFmt { kPlaneBF16 = 0, kPlaneTF32 = 1, kPlaneF16 = 2 };
eifmm_status build_kd_image(Ops* ops, int fmt, cudaStream_t s);
eifmm_status build_kd32(Ops* ops, cudaStream_t s);
// M2M / L2L as library GEMMs (xfer_blas.cu): one per level with one right-hand
// side, 8 strided-batched ones per level with several
eifmm_status build_xfer_blas(Ops* ops, cudaStream_t s);
// wsp: the calling tree's workspace for the library (kXferBlasWorkspace
// bytes), so that the GEMMs of trees evaluated on concurrent streams never
// share one; null: the per-device one
constexpr size_t kXferBlasWorkspace = 32u << 20;
bool xfer_blas(bool m2m, const LevelOps& out, const LevelOps& in, int64_t n_par, int R, const float* B,
               const float* G, float* C, void* wsp, cudaStream_t s);
// M2L compression (sarcmp.cu): eps <= 0 removes it.
eifmm_status compress_ops(Ops* ops, double eps, cudaStream_t s);
void free_compression(LevelOps& v);
eifmm_status launch_m2l_level(Tree* t, const Ops* ops, int k, int R, int kind, int gshift, cudaStream_t s);
eifmm_status eval_mixed(Tree* t, const Ops* ops, const double* sigma,
                        int64_t ld_sigma, int R, double* f, int64_t ld_f,
                        cudaStream_t s);
eifmm_status ensure_workspace(Tree* t, const Ops* ops, int R, int prec);
// Step 4 of level k with the compressed operators (sarcmp.cu) on the FP64
// far field; pair: FP32-pair arithmetic, else FP64.
// FP64 far-field M2L (fmm64.cu): offset groups split the offset list of a
// level with few blocks; `part` (part_cap doubles) holds their partial sums.
int m2l64_groups(int64_t blocks, int nsm);
int64_t m2l_df_blocks(int level, int d, int R);
int64_t m2l64_blocks(int level, int R);
eifmm_status launch_m2l_df(int level, int d, int R, const double* kdT, const int* slot_lists, const double* W,
                           double* g, double* part, size_t part_cap, int nsm, cudaStream_t s);
eifmm_status launch_m2l64(int level, int d, int R, const double* kdT, const int* slot_lists, const double* W,
                          double* g, double* part, size_t part_cap, int nsm, cudaStream_t s);
eifmm_status m2l_compressed(Workspace& ws, const Ops* ops, int k, int R, bool pair, cudaStream_t s);
void free_workspace(Workspace* ws);
bool timing_enabled();

// ----------------------------------------------------------- device util --
// spread the low 10 bits of v to every third bit (bit b -> bit 3b)
__host__ __device__ inline uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
// Morton key of box (x, y, z) with `bits` <= 10 bits per axis, x bit lowest.
__host__ __device__ inline int64_t morton_encode(int64_t x, int64_t y, int64_t z, int bits) {
  (void)bits;
  return (int64_t)(spread3((uint32_t)x) | (spread3((uint32_t)y) << 1) | (spread3((uint32_t)z) << 2));
}
__host__ __device__ inline void morton_decode(int64_t key, int bits, int* c) {
  int x = 0, y = 0, z = 0;
  for (int b = 0; b < bits; ++b) {
    x |= (int)((key >> (3 * b)) & 1) << b;
    y |= (int)((key >> (3 * b + 1)) & 1) << b;
    z |= (int)((key >> (3 * b + 2)) & 1) << b;
  }
  c[0] = x;
  c[1] = y;
  c[2] = z;
}

}  // namespace eifmm

// ------------------------------------------------------ kernel functions --
namespace eifmm {
__host__ __device__ inline double kern_f64(int kern, double z0, double z1, double z2) {
  const double r2 = z0 * z0 + z1 * z1 + z2 * z2;
  switch (kern) {
    case EIFMM_KERNEL_INV_R:
#ifdef __CUDA_ARCH__
      return rsqrt(r2);
#else
      return 1.0 / sqrt(r2);
#endif
    case EIFMM_KERNEL_CONFIG3: {
      const double r = sqrt(r2);
      const double a = z0 * z0 + 0.01 * (z1 * z1) + z2 * z2 + 1e-3;
#ifdef __CUDA_ARCH__
      return exp(-r) / r + rsqrt(a);
#else
      return exp(-r) / r + 1.0 / sqrt(a);
#endif
    }
    case EIFMM_KERNEL_QUAD:
      return r2;
    case EIFMM_KERNEL_ONE:
      return 1.0;
    case EIFMM_KERNEL_EXP_R2:
      return exp(-r2);
    case EIFMM_KERNEL_COS20R_R: {
      const double r = sqrt(r2);
      return cos(20.0 * r) / r;
    }
    case EIFMM_KERNEL_SQRT_R2P1:
      return sqrt(r2 + 1.0);
    default:
      return 0.0;
  }
}

// k(z) with IEEE-exact operations (no contraction) for the pivot search.
__device__ inline double kern_f64_ieee(int kern, double z0, double z1, double z2) {
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(z0, z0), __dmul_rn(z1, z1)), __dmul_rn(z2, z2));
  switch (kern) {
    case EIFMM_KERNEL_INV_R:
      return __ddiv_rn(1.0, __dsqrt_rn(r2));
    case EIFMM_KERNEL_CONFIG3: {
      const double r = __dsqrt_rn(r2);
      const double a = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(z0, z0), __dmul_rn(0.01, __dmul_rn(z1, z1))),
                                           __dmul_rn(z2, z2)), 1e-3);
      return __dadd_rn(__ddiv_rn(exp(-r), r), __ddiv_rn(1.0, __dsqrt_rn(a)));
    }
    case EIFMM_KERNEL_QUAD:
      return r2;
    case EIFMM_KERNEL_ONE:
      return 1.0;
    case EIFMM_KERNEL_EXP_R2:
      return exp(-r2);
    case EIFMM_KERNEL_COS20R_R: {
      const double r = __dsqrt_rn(r2);
      return __ddiv_rn(cos(__dmul_rn(20.0, r)), r);
    }
    case EIFMM_KERNEL_SQRT_R2P1:
      return __dsqrt_rn(__dadd_rn(r2, 1.0));
    default:
      return 0.0;
  }
}

// FP32 evaluation (mixed path): one Newton step after the hardware rsqrt.
__device__ inline float rsqrt_nr(float a) {
  float y = rsqrtf(a);
  // y (3 - a y^2) / 2
  return y * fmaf(-0.5f * a, y * y, 1.5f);
}
__device__ inline float kern_f32(int kern, float z0, float z1, float z2) {
  const float r2 = fmaf(z0, z0, fmaf(z1, z1, z2 * z2));
  switch (kern) {
    case EIFMM_KERNEL_INV_R:
      return rsqrt_nr(r2);
    case EIFMM_KERNEL_CONFIG3: {
      const float ir = rsqrt_nr(r2);
      const float r = r2 * ir;
      const float a = fmaf(z0, z0, fmaf(0.01f * z1, z1, fmaf(z2, z2, 1e-3f)));
      return expf(-r) * ir + rsqrt_nr(a);
    }
    case EIFMM_KERNEL_QUAD:
      return r2;
    case EIFMM_KERNEL_ONE:
      return 1.0f;
    case EIFMM_KERNEL_EXP_R2:
      return expf(-r2);
    case EIFMM_KERNEL_COS20R_R: {
      const float ir = rsqrt_nr(r2);
      return cosf(20.0f * r2 * ir) * ir;
    }
    case EIFMM_KERNEL_SQRT_R2P1:
      return sqrtf(r2 + 1.0f);
    default:
      return 0.0f;
  }
}
// Without the Newton step (about 2 ulp for 1/r); used where the tolerance
// allows it.
__device__ inline float kern_f32_fast(int kern, float z0, float z1, float z2) {
  if (kern == EIFMM_KERNEL_INV_R) return rsqrtf(fmaf(z0, z0, fmaf(z1, z1, z2 * z2)));
  return kern_f32(kern, z0, z1, z2);
}
}  // namespace eifmm
