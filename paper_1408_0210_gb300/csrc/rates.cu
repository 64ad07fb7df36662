// rates.cu -- measured per-GPU rates of the arithmetic the point kernels and
// the FP64 path are bound by (FP32 FMA, the approximate reciprocal square
// root, FP64 FMA), used as roofline denominators next to the measured
// HBM and BF16 peaks.  Register loops: 8 independent dependency chains per
// thread, every SM filled, timed with CUDA events; no memory traffic beyond
// one store per thread.
#include "internal.h"

namespace eifmm {
namespace {

constexpr int kRateIters = 4096;
constexpr int kRateChains = 8;

__device__ __forceinline__ float rsqrt_approx_r(float x) {
  float y;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void __launch_bounds__(256) k_rate_ffma(float a, float b, float* out) {
  float v[kRateChains];
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) v[c] = a + (float)(threadIdx.x + c);
  for (int i = 0; i < kRateIters; ++i)
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) v[c] = fmaf(v[c], b, a);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) s += v[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_rate_rsqrt(float a, float* out) {
  float v[kRateChains];
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) v[c] = a + (float)(threadIdx.x + c);
  for (int i = 0; i < kRateIters; ++i)
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) v[c] = rsqrt_approx_r(v[c]);  // x -> x^-1/2 stays finite
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) s += v[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_rate_dfma(double a, double b, double* out) {
  double v[kRateChains];
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) v[c] = a + (double)(threadIdx.x + c);
  for (int i = 0; i < kRateIters; ++i)
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) v[c] = fma(v[c], b, a);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) s += v[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace eifmm

using namespace eifmm;

extern "C" eifmm_status eifmm_measure_rates(eifmm_stream stream, double* rates) {
  if (!rates) {
    set_error("eifmm_measure_rates: null output");
    return EIFMM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 148;
  EIFMM_CUDA(cudaGetDevice(&dev));
  EIFMM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const unsigned blocks = (unsigned)nsm * 8;  // 2048 threads per SM
  const size_t nthr = (size_t)blocks * 256;
  double* buf = nullptr;
  EIFMM_TRY(dalloc(&buf, nthr));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  eifmm_status rc = EIFMM_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_error("eifmm_measure_rates: event creation failed");
    rc = EIFMM_ECUDA;
  }
  const double ops = (double)nthr * kRateIters * kRateChains;
  for (int which = 0; which < 3 && rc == EIFMM_OK; ++which) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {  // the first run warms up
      cudaEventRecord(e0, s);
      if (which == 0) k_rate_ffma<<<blocks, 256, 0, s>>>(0.5f, 0.999f, (float*)buf);
      else if (which == 1) k_rate_rsqrt<<<blocks, 256, 0, s>>>(1.5f, (float*)buf);
      else k_rate_dfma<<<blocks, 256, 0, s>>>(0.5, 0.999, buf);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        set_error("eifmm_measure_rates: a rate kernel failed");
        rc = EIFMM_ECUDA;
        break;
      }
      eifmm::count_launch();
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best) best = ms;
    }
    if (rc == EIFMM_OK) rates[which] = ops / (best * 1e-3);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dfree(buf);
  return rc;
}
