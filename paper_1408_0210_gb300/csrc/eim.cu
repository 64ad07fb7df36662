// eim.cu -- Algorithm 1 (the EIM greedy of Section 2) on the GPU, FP64.
//
// The residual delta_k K is kept on the training grid as an nx x ny matrix R.
// Step k: the pivot (x_{k+1}, y_{k+1}) is the first maximiser of |R| in
// row-major order (the x-argmax of the L-infinity norm, then the y-argmax);
// q_{k+1} = R(x_{k+1}, .) / R(x_{k+1}, y_{k+1}); R <- R - R(., y_{k+1}) q_{k+1}
// with the pivot row and column set to exact zeros.  B_{l,m} = q_m(y_l) and
// the rows of Gamma (pivot on the diagonal, alpha of the recursion of
// Section 2 below it) are formed once the greedy has stopped.
//
// The update and the next argmax are fused in one pass over R.  Every
// operation that decides a pivot is IEEE-exact (explicit _rn intrinsics, no
// fused multiply-add, correctly rounded sqrt and divide) so that, for the
// kernels without transcendental functions, the pivots and factors are the
// exact results of the stated operations.
#include <math.h>

#include <vector>

#include "internal.h"

namespace eifmm {
namespace {

constexpr double kTrainRatio = 1.35;
constexpr double kTrainUniform = 7.0;

int nodes_1d(int level, double* out) {
  const double M = ldexp(1.0, level + 1) - 1.0;  // (L - l_k) / l_k
  double pos[256];
  int np = 0;
  pos[np++] = 0.0;
  double t = 1.0;
  while (t <= kTrainUniform && t <= M) {
    pos[np++] = t;
    t += 1.0;
  }
  t = pos[np - 1];
  while (t < M) {
    t = t * kTrainRatio;
    if (t > M) t = M;
    pos[np++] = t;
  }
  int n = 0;
  for (int i = np - 1; i >= 1; --i) out[n++] = -pos[i];
  for (int i = 0; i < np; ++i) out[n++] = pos[i];
  return n;
}

struct ArgMax {
  double v;
  long long i;
};

__device__ __forceinline__ void am_merge(ArgMax& a, double v, long long i) {
  if (v > a.v || (v == a.v && i < a.i)) {
    a.v = v;
    a.i = i;
  }
}

__device__ ArgMax am_block_reduce(ArgMax a) {
  __shared__ double sv[32];
  __shared__ long long si[32];
  for (int o = 16; o > 0; o >>= 1) {
    const double v = __shfl_down_sync(0xffffffffu, a.v, o);
    const long long i = __shfl_down_sync(0xffffffffu, a.i, o);
    am_merge(a, v, i);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sv[w] = a.v;
    si[w] = a.i;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    a.v = lane < nw ? sv[lane] : -1.0;
    a.i = lane < nw ? si[lane] : 0x7fffffffffffffffLL;
    for (int o = 16; o > 0; o >>= 1) {
      const double v = __shfl_down_sync(0xffffffffu, a.v, o);
      const long long i = __shfl_down_sync(0xffffffffu, a.i, o);
      am_merge(a, v, i);
    }
  }
  return a;  // valid in thread 0
}

struct EimState {
  double g11;
  double p;        // signed pivot of the current step
  double eps_est;
  long long a, b;  // pivot row / column of the current step
  int done;
  int d;
};

__global__ void k_eim_init(int kern, const double* __restrict__ X, long long nx,
                           const double* __restrict__ Y, long long ny,
                           double* __restrict__ R, ArgMax* __restrict__ part) {
  ArgMax a{-1.0, 0x7fffffffffffffffLL};
  const long long nn = nx * ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / ny, j = t - i * ny;
    const double v = kern_f64_ieee(kern, __dsub_rn(X[3 * i], Y[3 * j]), __dsub_rn(X[3 * i + 1], Y[3 * j + 1]),
                                __dsub_rn(X[3 * i + 2], Y[3 * j + 2]));
    R[t] = v;
    am_merge(a, fabs(v), t);
  }
  a = am_block_reduce(a);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// One block: reduce the partial argmaxes, decide, snapshot the pivot row
// (divided by the pivot) and the pivot column.
__global__ void k_eim_pivot(const ArgMax* __restrict__ part, int nparts,
                            const double* __restrict__ R, long long nx,
                            long long ny, int step, double eps, int d_max,
                            EimState* __restrict__ st, long long* __restrict__ ia,
                            long long* __restrict__ ib, double* __restrict__ piv,
                            double* __restrict__ pval, double* __restrict__ q,
                            double* __restrict__ col) {
  __shared__ int s_done;
  __shared__ long long s_a, s_b;
  __shared__ double s_p;
  ArgMax a{-1.0, 0x7fffffffffffffffLL};
  for (int t = threadIdx.x; t < nparts; t += blockDim.x) am_merge(a, part[t].v, part[t].i);
  a = am_block_reduce(a);
  if (threadIdx.x == 0) {
    const long long idx = (a.v >= 0.0) ? a.i : 0;
    const long long pa = idx / ny, pb = idx - pa * ny;
    const double p = R[idx];
    if (step == 0) st->g11 = fabs(p);
    const double g11 = st->g11;
    piv[step] = fabs(p);
    int done = 0;
    if (step == d_max || p == 0.0 || fabs(p) <= eps * g11) {
      done = 1;
      st->eps_est = g11 > 0.0 ? fabs(p) / g11 : 0.0;
      st->d = step;
    } else {
      ia[step] = pa;
      ib[step] = pb;
      pval[step] = p;
    }
    st->done = done;
    st->a = pa;
    st->b = pb;
    st->p = p;
    s_done = done;
    s_a = pa;
    s_b = pb;
    s_p = p;
  }
  __syncthreads();
  if (s_done) return;
  for (long long j = threadIdx.x; j < ny; j += blockDim.x)
    q[(long long)step * ny + j] = __ddiv_rn(R[s_a * ny + j], s_p);
  for (long long i = threadIdx.x; i < nx; i += blockDim.x) col[i] = R[i * ny + s_b];
}

// delta_{k+1} K = delta_k K - col (x) q_{k+1}, pivot row/column zeroed,
// fused with the partial argmax of the new residual.
__global__ void k_eim_update(double* __restrict__ R, long long nx, long long ny,
                             const double* __restrict__ col,
                             const double* __restrict__ q,
                             const EimState* __restrict__ st,
                             ArgMax* __restrict__ part) {
  ArgMax a{-1.0, 0x7fffffffffffffffLL};
  const long long pa = st->a, pb = st->b;
  const long long nn = nx * ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / ny, j = t - i * ny;
    double v = 0.0;
    if (i != pa && j != pb) v = __dsub_rn(R[t], __dmul_rn(col[i], q[j]));
    R[t] = v;
    am_merge(a, fabs(v), t);
  }
  a = am_block_reduce(a);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// B_{l,m} = q_m(y_l) for m < l, B_{l,l} = 1 (row-major, ld = d_max).
__global__ void k_eim_B(int d, int d_max, long long ny, const double* __restrict__ q,
                        const long long* __restrict__ ib, double* __restrict__ B) {
  const int l = blockIdx.x;
  for (int m = threadIdx.x; m < d_max; m += blockDim.x) {
    double v = 0.0;
    if (m < l) v = q[(long long)m * ny + ib[l]];
    else if (m == l) v = 1.0;
    B[(long long)l * d_max + m] = v;
  }
}

// Gamma row k: pivot on the diagonal, alpha_m (m < k) with
// sum_{m' <= m} B_{m m'} alpha_{m'} = K(x_k, y_m).
__global__ void k_eim_Gamma(int kern, int d, int d_max, const double* __restrict__ X,
                            const double* __restrict__ Y,
                            const long long* __restrict__ ia,
                            const long long* __restrict__ ib,
                            const double* __restrict__ B,
                            const double* __restrict__ pval,
                            double* __restrict__ G) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d) return;
  double* row = G + (long long)k * d_max;
  for (int m = 0; m < d_max; ++m) row[m] = 0.0;
  const double* x = X + 3 * ia[k];
  for (int m = 0; m < k; ++m) {
    const double* y = Y + 3 * ib[m];
    double s = kern_f64_ieee(kern, __dsub_rn(x[0], y[0]), __dsub_rn(x[1], y[1]), __dsub_rn(x[2], y[2]));
    for (int mm = 0; mm < m; ++mm) s = __dsub_rn(s, __dmul_rn(B[(long long)m * d_max + mm], row[mm]));
    row[m] = s;
  }
  row[k] = pval[k];
}

}  // namespace
}  // namespace eifmm

using namespace eifmm;

extern "C" eifmm_status eifmm_training_sets(int level, double L, int nJ, double* X,
                                            int64_t* nx, double* Y, int64_t* ny) {
  if (level < 2 || level > kMaxLevel || nJ < 2 || !(L > 0.0) || !nx || !ny) {
    set_error("eifmm_training_sets: invalid level, nJ, L or count pointer");
    return EIFMM_EINVAL;
  }
  double u[512];
  const int n = nodes_1d(level, u);
  const double l = L * ldexp(1.0, -(level + 1));
  int64_t cnt = 0;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c) {
        double m = fabs(u[a]);
        if (fabs(u[b]) > m) m = fabs(u[b]);
        if (fabs(u[c]) > m) m = fabs(u[c]);
        if (m < 3.0) continue;
        if (X) {
          X[3 * cnt + 0] = u[a] * l;
          X[3 * cnt + 1] = u[b] * l;
          X[3 * cnt + 2] = u[c] * l;
        }
        ++cnt;
      }
  *nx = cnt;
  cnt = 0;
  for (int a = 0; a < nJ; ++a)
    for (int b = 0; b < nJ; ++b)
      for (int c = 0; c < nJ; ++c) {
        if (Y) {
          Y[3 * cnt + 0] = ((double)(2 * a - (nJ - 1)) / (double)(nJ - 1)) * l;
          Y[3 * cnt + 1] = ((double)(2 * b - (nJ - 1)) / (double)(nJ - 1)) * l;
          Y[3 * cnt + 2] = ((double)(2 * c - (nJ - 1)) / (double)(nJ - 1)) * l;
        }
        ++cnt;
      }
  *ny = cnt;
  return EIFMM_OK;
}

extern "C" eifmm_status eifmm_eim_build(eifmm_kernel kern, const double* X, int64_t nx,
                                        const double* Y, int64_t ny, double eps,
                                        int d_max, int* d, int64_t* ia, int64_t* ib,
                                        double* Gamma, double* B, double* piv,
                                        double* eps_est, eifmm_stream stream) {
  if (!X || !Y || !d || !ia || !ib || !Gamma || !B || !piv || !eps_est || nx < 1 || ny < 1 ||
      !(eps > 0.0) || d_max < 1 || d_max > 1024 || (int)kern < 0 || (int)kern > 6) {
    set_error("eifmm_eim_build: invalid argument");
    return EIFMM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const long long nn = (long long)nx * ny;
  int dev = 0, nsm = 1;
  EIFMM_CUDA(cudaGetDevice(&dev));
  EIFMM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  long long want = (nn + 255) / 256;
  const int nparts = (int)(want < (long long)nsm * 8 ? want : (long long)nsm * 8);

  double *dX = nullptr, *dY = nullptr, *R = nullptr, *q = nullptr, *col = nullptr;
  double *dpiv = nullptr, *dpval = nullptr, *dG = nullptr, *dB = nullptr;
  long long *dia = nullptr, *dib = nullptr;
  ArgMax* part = nullptr;
  EimState* st = nullptr;
  eifmm_status rc = EIFMM_OK;
  auto cleanup = [&]() {
    dfree(dX); dfree(dY); dfree(R); dfree(q); dfree(col); dfree(dpiv); dfree(dpval);
    dfree(dG); dfree(dB); dfree(dia); dfree(dib); dfree(part); dfree(st);
  };
#define EIM_TRY(call) do { rc = (call); if (rc != EIFMM_OK) { cleanup(); return rc; } } while (0)
#define EIM_CUDA(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { \
    set_error(std::string("eifmm_eim_build: ") + cudaGetErrorString(e_)); cleanup(); return EIFMM_ECUDA; } } while (0)
  EIM_TRY(dalloc(&dX, 3 * nx));
  EIM_TRY(dalloc(&dY, 3 * ny));
  EIM_TRY(dalloc(&R, nn));
  EIM_TRY(dalloc(&q, (size_t)d_max * ny));
  EIM_TRY(dalloc(&col, nx));
  EIM_TRY(dalloc(&dpiv, d_max + 1));
  EIM_TRY(dalloc(&dpval, d_max));
  EIM_TRY(dalloc(&dG, (size_t)d_max * d_max));
  EIM_TRY(dalloc(&dB, (size_t)d_max * d_max));
  EIM_TRY(dalloc(&dia, d_max));
  EIM_TRY(dalloc(&dib, d_max));
  EIM_TRY(dalloc(&part, nparts));
  EIM_TRY(dalloc(&st, 1));
  EIM_CUDA(cudaMemcpyAsync(dX, X, 3 * nx * sizeof(double), cudaMemcpyHostToDevice, s));
  EIM_CUDA(cudaMemcpyAsync(dY, Y, 3 * ny * sizeof(double), cudaMemcpyHostToDevice, s));
  EIM_CUDA(cudaMemsetAsync(st, 0, sizeof(EimState), s));

  k_eim_init<<<nparts, 256, 0, s>>>((int)kern, dX, nx, dY, ny, R, part);
  EIM_CUDA(cudaGetLastError());
  EimState hs{};
  int step = 0;
  for (;; ++step) {
    k_eim_pivot<<<1, 1024, 0, s>>>(part, nparts, R, nx, ny, step, eps, d_max, st, dia, dib, dpiv,
                                   dpval, q, col);
    EIM_CUDA(cudaGetLastError());
    EIM_CUDA(cudaMemcpyAsync(&hs, st, sizeof(EimState), cudaMemcpyDeviceToHost, s));
    EIM_CUDA(cudaStreamSynchronize(s));
    if (hs.done) break;
    k_eim_update<<<nparts, 256, 0, s>>>(R, nx, ny, col, q + (long long)step * ny, st, part);
    EIM_CUDA(cudaGetLastError());
  }
  const int dd = hs.d;
  if (dd > 0) {
    k_eim_B<<<dd, 128, 0, s>>>(dd, d_max, ny, q, dib, dB);
    EIM_CUDA(cudaGetLastError());
    k_eim_Gamma<<<(dd + 63) / 64, 64, 0, s>>>((int)kern, dd, d_max, dX, dY, dia, dib, dB, dpval, dG);
    EIM_CUDA(cudaGetLastError());
  }
  std::vector<long long> hia(d_max), hib(d_max);
  EIM_CUDA(cudaMemcpyAsync(hia.data(), dia, d_max * sizeof(long long), cudaMemcpyDeviceToHost, s));
  EIM_CUDA(cudaMemcpyAsync(hib.data(), dib, d_max * sizeof(long long), cudaMemcpyDeviceToHost, s));
  EIM_CUDA(cudaMemcpyAsync(piv, dpiv, (dd + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (dd > 0) {
    EIM_CUDA(cudaMemcpyAsync(Gamma, dG, (size_t)d_max * dd * sizeof(double), cudaMemcpyDeviceToHost, s));
    EIM_CUDA(cudaMemcpyAsync(B, dB, (size_t)d_max * dd * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  EIM_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < dd; ++k) {
    ia[k] = hia[k];
    ib[k] = hib[k];
  }
  *d = dd;
  *eps_est = hs.eps_est;
  cleanup();
  return EIFMM_OK;
#undef EIM_TRY
#undef EIM_CUDA
}
