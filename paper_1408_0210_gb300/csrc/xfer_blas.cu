// xfer_blas.cu -- steps 2 and 5 of Algorithm 3 (M2M, L2L) of the mixed path
// with one right-hand side as one GEMM per level in cuBLAS, FP32 emulated
// on the tensor cores (CUBLAS_COMPUTE_32F_EMULATED_16BFX9: each FP32 input
// split into three BF16 values, FP32 accuracy).
//
// In Morton order the 8 children of parent P are the boxes 8P .. 8P + 7,
// whose coefficient rows [box][dp] are contiguous; so, column-major,
//   M2M:  W_parent (dp_k x n_par) = [K_M2M^0 ... K_M2M^7] (dp_k x 8 dp_c)
//                                   x W_child (8 dp_c x n_par, ld 8 dp_c)
//   L2L:  l_child (8 dp_k x n_par, ld 8 dp_k) = g_child
//             + [K_L2L^0; ...; K_L2L^7] (8 dp_k x dp_p) x l_parent (dp_p x n_par)
// with the operators zero-padded to dp (so the padding columns stay zero).
// These are plain GEMMs, so a library GEMM serves them; any failure of the
// library leaves the SIMT kernel of transfer.cuh to do the step.  With
// several right-hand sides each level is 8 strided-batched GEMMs (below).
#include <cublas_v2.h>

#include <mutex>

#include "internal.h"

namespace eifmm {
namespace {

constexpr int kMaxDev = 64;
constexpr size_t kBlasWorkspace = kXferBlasWorkspace;  // set up front: no allocation inside a capture
cublasHandle_t g_handle[kMaxDev] = {};
void* g_ws[kMaxDev] = {};
bool g_failed[kMaxDev] = {};
std::mutex g_mu;

// A_m2m (dp_k x 8 dp_c, col-major) from m2m32 ([8][dk][dc] row-major)
__global__ void k_m2m_cb(const float* __restrict__ m2m, int dk, int dc, int dpk, int dpc, float* __restrict__ A) {
  const int64_t n = (int64_t)dpk * 8 * dpc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(t % dpk);
    const int64_t col = t / dpk;
    const int i = (int)(col / dpc), q = (int)(col % dpc);
    A[t] = (m < dk && q < dc) ? m2m[((int64_t)i * dk + m) * dc + q] : 0.f;
  }
}

// A_l2l (8 dp_k x dp_p, col-major) from l2l32 ([8][dk][dpar] row-major)
__global__ void k_l2l_cb(const float* __restrict__ l2l, int dk, int dpar, int dpk, int dpp, float* __restrict__ A) {
  const int64_t n = (int64_t)8 * dpk * dpp;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = t % (8 * dpk);
    const int q = (int)(t / (8 * dpk));
    const int i = (int)(row / dpk), m = (int)(row % dpk);
    A[t] = (m < dk && q < dpar) ? l2l[((int64_t)i * dk + m) * dpar + q] : 0.f;
  }
}

unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024); }

cublasHandle_t handle_here() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev || g_failed[dev]) return nullptr;
  if (!g_handle[dev]) {
    if (cublasCreate(&g_handle[dev]) != CUBLAS_STATUS_SUCCESS || cudaMalloc(&g_ws[dev], kBlasWorkspace) != cudaSuccess ||
        cublasSetWorkspace(g_handle[dev], g_ws[dev], kBlasWorkspace) != CUBLAS_STATUS_SUCCESS) {
      g_failed[dev] = true;
      return nullptr;
    }
    // the operands are finite (sigma is required finite), so the emulation
    // needs no scan of its inputs for infinities and NaNs nor the patch
    // passes that follow one; a library without the switch keeps its default
    cublasSetEmulationSpecialValuesSupport(g_handle[dev], CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_NONE);
  }
  return g_handle[dev];
}

// the handle on stream s with the workspace wsp (else the device's own):
// kernels of the library that run at the same time on different streams
// must not share a workspace
bool bind(cublasHandle_t h, void* wsp, cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return false;
  return cublasSetStream(h, s) == CUBLAS_STATUS_SUCCESS &&
         cublasSetWorkspace(h, wsp ? wsp : g_ws[dev], kBlasWorkspace) == CUBLAS_STATUS_SUCCESS;
}

}  // namespace

eifmm_status build_xfer_blas(Ops* ops, cudaStream_t s) {
  for (int k = 2; k <= ops->depth; ++k) {
    LevelOps& v = ops->lv[k];
    if (k < ops->depth && v.m2m32 && !v.m2m_cb) {
      const LevelOps& c = ops->lv[k + 1];
      EIFMM_TRY(dalloc(&v.m2m_cb, (size_t)v.dp * 8 * c.dp));
      k_m2m_cb<<<blocks((int64_t)v.dp * 8 * c.dp), 256, 0, s>>>(v.m2m32, v.d, c.d, v.dp, c.dp, v.m2m_cb);
      EIFMM_CHECK_LAUNCH();
    }
    if (k > 2 && v.l2l32 && !v.l2l_cb) {
      const LevelOps& p = ops->lv[k - 1];
      EIFMM_TRY(dalloc(&v.l2l_cb, (size_t)8 * v.dp * p.dp));
      k_l2l_cb<<<blocks((int64_t)8 * v.dp * p.dp), 256, 0, s>>>(v.l2l32, v.d, p.d, v.dp, p.dp, v.l2l_cb);
      EIFMM_CHECK_LAUNCH();
    }
  }
  return EIFMM_OK;
}

// Several right-hand sides (rows [box R + r][dp]): the rows of one octant i
// and one column r are a matrix with a constant leading dimension, so each
// level is 8 strided-batched GEMMs (one per octant, batched over r):
//   M2M: W_parent[:, P R + r] (+)= K_M2M^i W_child[:, (8P + i) R + r]
//   L2L: l_child[:, (8P + i) R + r] = g_child[...] + K_L2L^i l_parent[:, P R + r]
// (column-major, as above).  Below kBatchedMinParents parents the SIMT
// kernel is left the level: 8 library calls cost more there.
constexpr int64_t kBatchedMinParents = 512;
bool g_batched_failed[kMaxDev] = {};

bool xfer_blas_rhs(bool m2m, const LevelOps& out, const LevelOps& in, int64_t n_par, int R, const float* B,
                   const float* G, float* C, void* wsp, cudaStream_t s) {
  const float* A = m2m ? out.m2m_cb : out.l2l_cb;
  if (!A || n_par < kBatchedMinParents || n_par > 2147483647LL || R < 2) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev || g_batched_failed[dev]) return false;
  std::lock_guard<std::mutex> lk(g_mu);
  cublasHandle_t h = handle_here();
  if (!h || !bind(h, wsp, s)) return false;
  const float one = 1.f, zero = 0.f;
  const int dk = out.dp, dc = in.dp;
  const int n = (int)n_par;
  if (!m2m &&
      cudaMemcpyAsync(C, G, (size_t)n_par * 8 * R * dk * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return false;
  for (int i = 0; i < 8; ++i) {
    cublasStatus_t st;
    if (m2m) {
      st = cublasGemmStridedBatchedEx(h, CUBLAS_OP_N, CUBLAS_OP_N, dk, n, dc, &one, A + (size_t)i * dc * dk,
                                      CUDA_R_32F, dk, 0, B + (size_t)dc * i * R, CUDA_R_32F, 8 * R * dc, dc,
                                      i == 0 ? &zero : &one, C, CUDA_R_32F, R * dk, dk, R,
                                      CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT);
    } else {
      st = cublasGemmStridedBatchedEx(h, CUBLAS_OP_N, CUBLAS_OP_N, dk, n, dc, &one, A + (size_t)i * dk, CUDA_R_32F,
                                      8 * dk, 0, B, CUDA_R_32F, R * dc, dc, &one, C + (size_t)dk * i * R,
                                      CUDA_R_32F, 8 * R * dk, dk, R, CUBLAS_COMPUTE_32F_EMULATED_16BFX9,
                                      CUBLAS_GEMM_DEFAULT);
    }
    if (st != CUBLAS_STATUS_SUCCESS) {
      // the SIMT kernel then writes the whole level afresh (it stores, it
      // does not add), whatever the octants before this one left there
      g_batched_failed[dev] = true;
      return false;
    }
  }
  return true;
}

// true when the library took the step; false: the caller runs its own kernel
bool xfer_blas(bool m2m, const LevelOps& out, const LevelOps& in, int64_t n_par, int R, const float* B,
               const float* G, float* C, void* wsp, cudaStream_t s) {
  if (R > 1) return xfer_blas_rhs(m2m, out, in, n_par, R, B, G, C, wsp, s);
  const float* A = m2m ? out.m2m_cb : out.l2l_cb;
  if (!A || n_par <= 0 || n_par > 2147483647LL) return false;
  std::lock_guard<std::mutex> lk(g_mu);
  cublasHandle_t h = handle_here();
  if (!h || !bind(h, wsp, s)) return false;
  const float one = 1.f, zero = 0.f;
  cublasStatus_t st;
  if (m2m) {
    st = cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, out.dp, (int)n_par, 8 * in.dp, &one, A, CUDA_R_32F, out.dp, B,
                      CUDA_R_32F, 8 * in.dp, &zero, C, CUDA_R_32F, out.dp, CUBLAS_COMPUTE_32F_EMULATED_16BFX9,
                      CUBLAS_GEMM_DEFAULT);
  } else {
    // l_child = g_child, then += A l_parent
    if (cudaMemcpyAsync(C, G, (size_t)n_par * 8 * out.dp * sizeof(float), cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
      return false;
    st = cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, 8 * out.dp, (int)n_par, in.dp, &one, A, CUDA_R_32F, 8 * out.dp,
                      B, CUDA_R_32F, in.dp, &one, C, CUDA_R_32F, 8 * out.dp, CUBLAS_COMPUTE_32F_EMULATED_16BFX9,
                      CUBLAS_GEMM_DEFAULT);
  }
  if (st != CUBLAS_STATUS_SUCCESS) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < kMaxDev) g_failed[dev] = true;  // the SIMT kernel from now on
    return false;
  }
  return true;
}

}  // namespace eifmm
