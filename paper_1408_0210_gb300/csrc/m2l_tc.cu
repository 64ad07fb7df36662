// m2l_tc.cu -- step 4 of Algorithm 3 (M2L, Eq. M2Lstep) on the tcgen05 tensor
// cores of sm_103a.
//
//   g^I = sum_{J in I(I)} K^delta What^J,   delta = c_J - c_I
//
// is computed as a chain of GEMMs accumulated in TMEM.  A CTA owns a tile of
// 128 rows = (target box I, rhs r) of one parity class (all boxes with the
// same child octant share the 189 candidate offsets delta).  For every delta
// and every 128-byte chunk of the reduction index l:
//   A (128 x chunk, K-major)  = What rows of the source boxes I + delta,
//                               gathered with cp.async (zero-filled outside
//                               the cube), 128B-swizzled in shared memory;
//   B (dp x chunk, K-major)   = K^delta, a pre-swizzled image in HBM copied
//                               with one cp.async.bulk;
//   D (128 x dp, FP32, TMEM) += A B^t  via tcgen05.mma issued by one thread.
// The operands are split into precision planes (BF16 hi + lo, or TF32 hi + lo)
// and the products hi*hi + hi*lo + lo*hi are accumulated, which keeps about
// 16 (BF16) or 21 (TF32) significant bits per product with FP32 accumulation.
// Two stages of shared memory let the copies of one chunk overlap the MMAs of
// the previous one; tcgen05.commit on an mbarrier releases a stage.  Every
// wait is bounded: on time-out the kernel records an error code, drains its
// copies, frees its TMEM and returns.
#include "internal.h"
#include "m2l_tc.h"

namespace eifmm {
namespace {

constexpr int kRows = 128;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok;
}
// Bounded wait; returns false (and records `code`) on time-out.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int* err, int code) {
  const long long t0 = clock64();
  while (!mbar_try(a, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      atomicExch(err, code);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes stacked along M/N (SBO = 1024), version 1 (sm_100 family).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // LBO (ignored for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // SBO
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // SWIZZLE_128B
  return d;
}

// Instruction descriptor: D = F32, A/B format `fmt` (BF16 = 1 in kind::f16,
// TF32 = 2 in kind::tf32), both K-major, N, M = 128.
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, uint32_t n) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (TF32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Template parameters: TF32 selects kind::tf32 (4-byte elements) instead of
// kind::f16 with BF16 (2-byte elements).  Two operand planes on each side.
template <bool TF32>
__global__ void __launch_bounds__(kRows, 1)
k_m2l_tc(M2LTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzle atoms
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x;
  const int esz = TF32 ? 4 : 2;
  const int dp = a.dp;
  const int nchunk = dp * esz / 128;
  const uint32_t a_bytes = 16384u;                  // 128 rows x 128 B per plane
  const uint32_t b_bytes = (uint32_t)dp * 128u;     // dp rows x 128 B per plane
  const uint32_t stage = 2 * a_bytes + 2 * b_bytes;
  uint64_t* bars = (uint64_t*)(smem + 2 * stage);   // [0,1] loads, [2,3] mma
  uint32_t* tslot = (uint32_t*)(bars + 4);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar_ld[2] = {smem_u32(&bars[0]), smem_u32(&bars[1])};
  const uint32_t bar_mma[2] = {smem_u32(&bars[2]), smem_u32(&bars[3])};

  // tile -> rows
  const int oct = blockIdx.x % 8;
  const int64_t tile = blockIdx.x / 8;
  const int64_t q = tile * kRows + tid;  // row within the parity class
  const int64_t nclass = a.nbox / 8 * a.R;
  const bool valid = q < nclass;
  const int64_t p = valid ? q / a.R : 0;
  const int r = valid ? (int)(q % a.R) : 0;
  const int64_t I = 8 * p + oct;
  int ci[3];
  morton_decode(I, a.level, ci);
  const int n = 1 << a.level;

  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(smem_u32(&bars[i]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"((uint32_t)a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const char* wbase = (const char*)a.wa;
  const size_t plane_stride = (size_t)a.rows * dp * esz;  // bytes between A planes
  const int* lst = a.slot_lists + oct * kListLen;
  const uint32_t id_lo = idesc(TF32 ? 2u : 1u, dp > 256 ? 256u : (uint32_t)dp);
  const uint32_t id_hi = idesc(TF32 ? 2u : 1u, dp > 256 ? (uint32_t)(dp - 256) : 16u);

  int it = 0;
  bool accum = false;
  bool ok = true;
  for (int s = 0; s <= kListLen && ok; ++s) {
    int slot = -1;
    int64_t src_row = -1;
    if (s < kListLen) {
      slot = lst[s];
      const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
      const int jx = ci[0] + dx, jy = ci[1] + dy, jz = ci[2] + dz;
      if (valid && jx >= 0 && jy >= 0 && jz >= 0 && jx < n && jy < n && jz < n)
        src_row = morton_encode(jx, jy, jz, a.level) * a.R + r;
      if (!__syncthreads_or(src_row >= 0)) continue;  // no row of the tile reaches this delta
    }
    const int nc = (s < kListLen) ? nchunk : 1;
    for (int c = 0; c < nc && ok; ++c) {
      // ---- issue the copies of iteration `it` (skip on the drain pass) ----
      if (s < kListLen) {
        const int b = it & 1;
        if (it >= 2) ok = mbar_wait(bar_mma[b], ((it >> 1) - 1) & 1, a.err, 1);
        if (!__syncthreads_and(ok)) { ok = false; break; }
        const uint32_t sA = sbase + b * stage;
        const uint32_t sB = sA + 2 * a_bytes;
        if (tid == 0) {
          const char* src = (const char*)a.kd_img + (((size_t)slot * nchunk + c) * 2) * b_bytes;
          mbar_expect_tx(bar_ld[b], 2 * b_bytes);
          bulk_g2s(sB, src, 2 * b_bytes, bar_ld[b]);
        }
        const uint32_t rowoff = (uint32_t)(tid >> 3) * 1024u + (uint32_t)(tid & 7) * 128u;
        const char* gsrc = wbase + (size_t)(src_row >= 0 ? src_row : 0) * dp * esz + (size_t)c * 128;
        const uint32_t nb = src_row >= 0 ? 16u : 0u;
#pragma unroll
        for (int pl = 0; pl < 2; ++pl)
#pragma unroll
          for (int j = 0; j < 8; ++j)
            cp16(sA + pl * a_bytes + rowoff + (uint32_t)((j ^ (tid & 7)) << 4), gsrc + pl * plane_stride + j * 16, nb);
        cp_commit();
      }
      // ---- MMAs of iteration it - 1 ----
      if (it >= 1) {
        if (s < kListLen) cp_wait1(); else cp_wait0();
        fence_async_smem();
        __syncthreads();
        const int bp = (it - 1) & 1;
        if (tid == 0) {
          if (!mbar_wait(bar_ld[bp], ((it - 1) >> 1) & 1, a.err, 2)) {
            ok = false;
          } else {
            tc_fence_after();
            const uint32_t sA = sbase + bp * stage;
            const uint32_t sB = sA + 2 * a_bytes;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              // hi*hi, hi*lo, lo*hi
#pragma unroll
              for (int pr = 0; pr < 3; ++pr) {
                const int pa = (pr == 2) ? 1 : 0, pb = (pr == 1) ? 1 : 0;
                const uint64_t ad = sdesc(sA + pa * a_bytes + kk * 32);
                const uint32_t bB = sB + pb * b_bytes + kk * 32;
                mma<TF32>(tmem, ad, sdesc(bB), id_lo, accum ? 1u : 0u);
                if (dp > 256) mma<TF32>(tmem + 256, ad, sdesc(bB + 32 * 1024), id_hi, accum ? 1u : 0u);
                accum = true;
              }
            }
            mma_commit(bar_mma[bp]);
          }
        }
        ok = __syncthreads_and(ok);
      }
      if (s < kListLen) ++it;
    }
  }
  cp_wait0();
  // wait for the last commit (it tracks every earlier MMA of the thread)
  bool done = ok;
  if (it >= 1 && ok) done = mbar_wait(bar_mma[(it - 1) & 1], ((it - 1) >> 1) & 1, a.err, 3);
  done = __syncthreads_and(done);
  tc_fence_after();
  // ---- epilogue: TMEM lane tid -> row; FP32 out.  The TMEM loads are
  // warp-collective, so every thread executes them; only stores are masked.
  const bool has_acc = it >= 1;  // uniform: some MMA was issued
  if (done) {
    float* out = a.g + (size_t)(I * a.R + r) * dp;
    const uint32_t lane_base = (uint32_t)((tid & ~31) << 16);
    for (int c0 = 0; c0 < dp; c0 += 16) {
      float v[16];
      if (has_acc) {
        tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
      }
      if (valid) {
        float4* o4 = (float4*)(out + c0);
#pragma unroll
        for (int i = 0; i < 4; ++i) o4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)a.tmem_cols));
}

}  // namespace

size_t m2l_tc_smem_bytes(int dp, bool tf32) {
  (void)tf32;
  return 2 * (2 * 16384 + 2 * (size_t)dp * 128) + 64 + 1024;
}

eifmm_status launch_m2l_tc(const M2LTcArgs& a, bool tf32, cudaStream_t s) {
  const size_t sm = m2l_tc_smem_bytes(a.dp, tf32);
  static bool attr[2] = {false, false};
  if (!attr[tf32]) {
    if (tf32)
      EIFMM_CUDA(cudaFuncSetAttribute(k_m2l_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    else
      EIFMM_CUDA(cudaFuncSetAttribute(k_m2l_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr[tf32] = true;
  }
  const int64_t tiles = (a.nbox / 8 * a.R + kRows - 1) / kRows;
  const unsigned grid = (unsigned)(tiles * 8);
  if (tf32) k_m2l_tc<true><<<grid, kRows, sm, s>>>(a);
  else k_m2l_tc<false><<<grid, kRows, sm, s>>>(a);
  EIFMM_CHECK_LAUNCH();
  return EIFMM_OK;
}

}  // namespace eifmm
