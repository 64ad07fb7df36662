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
#include <cuda.h>
#include <stdlib.h>

#include <algorithm>
#include <cstdlib>
#include <vector>

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
// Bounded wait; returns false (and records `code`) after `limit` cycles.
__device__ __forceinline__ bool mbar_wait_lim(uint32_t a, uint32_t parity, int* err, int code, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try(a, parity)) {
    if (clock64() - t0 > limit) {
      atomicExch(err, code);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int* err, int code) {
  return mbar_wait_lim(a, parity, err, code, kWaitCycles);
}

// The producer's last act: every copy it issued has landed (each stage's
// last fill completed its phase) before the CTA may exit, also after an
// abort.  it = fills issued so far, ring of `stages`.  Bounded like every
// wait.
__device__ __forceinline__ void drain_fills(int it, int stages, const uint64_t* bars_full, int* err) {
  for (int k = 0; k < stages && k < it; ++k) {
    const int i = it - 1 - k;  // a recent fill
    mbar_wait(smem_u32(&bars_full[i % stages]), (uint32_t)((i / stages) & 1), err, 5);
  }
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

// The 4 k-steps x 3 split products of one 128-byte chunk of l:
//   D (+)= A_hi B_hi^t + A_hi B_lo^t + A_lo B_hi^t.
// da / db: descriptors of plane 0 of the stage's A and B; plane 1 sits
// pa16 / pb16 descriptor units (16 bytes) further and k-step kk at 2 kk (32
// bytes), which never carries out of the 14-bit address field.  `wide`: a
// second MMA covers accumulator columns 256.. (dp > 256).
template <bool TF32>
__device__ __forceinline__ void issue_chunk(uint32_t dacc, uint64_t da, uint64_t db, uint32_t pa16, uint32_t pb16,
                                            uint32_t id_lo, uint32_t id_hi, bool wide, bool first) {
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
#pragma unroll
    for (int pr = 0; pr < 3; ++pr) {
      const uint64_t ad = da + (pr == 2 ? pa16 : 0u) + 2u * kk;
      const uint64_t bd = db + (pr == 1 ? pb16 : 0u) + 2u * kk;
      const uint32_t acc = (first && kk == 0 && pr == 0) ? 0u : 1u;
      mma<TF32>(dacc, ad, bd, id_lo, acc);
      if (wide) mma<TF32>(dacc + 256, ad, bd + 2048u, id_hi, acc);
    }
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

// Template parameter TF32 selects kind::tf32 (4-byte elements) instead of
// kind::f16 with BF16 (2-byte elements); two operand planes on each side.
//
// Warps 0-3 (threads 0..127) gather the A rows (thread t = tile row t) with
// cp.async and, at the end, read the accumulator (TMEM lane t = row t); warp
// 4 issues the MMAs.  An S-stage ring of shared memory with `full` barriers
// (128 producer arrivals after their copies landed and were fenced for the
// async proxy, plus the expect-tx arrival of the bulk copy of B) and `empty`
// barriers (tcgen05.commit of the MMAs that read the stage).
constexpr int kMaxStages = 3;

template <bool TF32>
__global__ void __launch_bounds__(160, 1)
k_m2l_tc(M2LTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x;
  const int esz = TF32 ? 4 : 2;
  const int dp = a.dp;
  const int S = a.stages;
  const int nchunk = dp * esz / 128;
  const uint32_t a_bytes = 16384u;               // 128 rows x 128 B per plane
  const uint32_t b_bytes = (uint32_t)dp * 128u;  // dp rows x 128 B per plane
  const uint32_t stage = 2 * a_bytes + 2 * b_bytes;
  uint64_t* bars = (uint64_t*)(smem + S * stage);  // full[S], empty[S], done
  uint32_t* tslot = (uint32_t*)(bars + 2 * kMaxStages + 1);
  int* flags = (int*)(tslot + 1);                    // [kListLen]
  short* act = (short*)(flags + kListLen);           // active slot ids
  int* nact_p = (int*)(act + kListLen + 1);
  const uint32_t sbase = smem_u32(smem);
  auto full = [&](int st) { return smem_u32(&bars[st]); };
  auto empty = [&](int st) { return smem_u32(&bars[kMaxStages + st]); };
  const uint32_t done_bar = smem_u32(&bars[2 * kMaxStages]);

  // ---- tile rows and the offset group of this CTA ----
  const int oct = blockIdx.x % 8;
  const int grp = (blockIdx.x / 8) % a.groups;
  const int64_t tile = blockIdx.x / (8 * a.groups);
  const int s_beg = grp * kListLen / a.groups, s_end = (grp + 1) * kListLen / a.groups;
  const int64_t q = tile * kRows + (tid < kRows ? tid : 0);
  const int64_t nclass = a.nbox / 8 * a.R;
  const bool valid = tid < kRows && q < nclass;
  const int64_t p = valid ? q / a.R : 0;
  const int r = valid ? (int)(q % a.R) : 0;
  const int64_t I = 8 * p + oct;
  int ci[3];
  morton_decode(I, a.level, ci);
  const int n = 1 << a.level;
  const int* lst = a.slot_lists + oct * kListLen;

  for (int i = tid; i < kListLen; i += blockDim.x) flags[i] = 0;
  if (tid == 0) {
    for (int i = 0; i < kMaxStages; ++i) {
      mbar_init(full(i), kRows + 1);
      mbar_init(empty(i), 1);
    }
    mbar_init(done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid >= 128) {  // warp 4 owns the TMEM allocation
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"((uint32_t)a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  // offsets of the group that reach at least one row of the tile
  if (valid)
    for (int s = s_beg; s < s_end; ++s) {
      const int slot = lst[s];
      const int jx = ci[0] + slot % 7 - 3, jy = ci[1] + (slot / 7) % 7 - 3, jz = ci[2] + slot / 49 - 3;
      if (jx >= 0 && jy >= 0 && jz >= 0 && jx < n && jy < n && jz < n) flags[s] = 1;
    }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) {
    int na = 0;
    for (int s = s_beg; s < s_end; ++s)
      if (flags[s]) act[na++] = (short)s;
    *nact_p = na;
  }
  __syncthreads();
  const uint32_t tmem = *tslot;
  const int nit = *nact_p * nchunk;
  bool ok = true;

  if (tid < kRows) {
    // ------------------------------------------------------- producers --
    const char* wbase = (const char*)a.wa;
    const size_t plane_stride = (size_t)a.rows * dp * esz;
    const uint32_t rowoff = (uint32_t)(tid >> 3) * 1024u + (uint32_t)(tid & 7) * 128u;
    for (int it = 0; it < nit && ok; ++it) {
      const int st = it % S, u = it / S;
      if (it >= S) ok = mbar_wait(empty(st), (u - 1) & 1, a.err, 1);
      if (!ok) break;
      const int s = act[it / nchunk], c = it % nchunk;
      const int slot = lst[s];
      const int jx = ci[0] + slot % 7 - 3, jy = ci[1] + (slot / 7) % 7 - 3, jz = ci[2] + slot / 49 - 3;
      int64_t src_row = -1;
      if (valid && jx >= 0 && jy >= 0 && jz >= 0 && jx < n && jy < n && jz < n)
        src_row = morton_encode(jx, jy, jz, a.level) * a.R + r;
      const uint32_t sA = sbase + st * stage;
      if (tid == 0) {
        const char* src = (const char*)a.kd_img + (((size_t)slot * nchunk + c) * 2) * b_bytes;
        mbar_expect_tx(full(st), 2 * b_bytes);
        bulk_g2s(sA + 2 * a_bytes, src, 2 * b_bytes, full(st));
      }
      const char* gsrc = wbase + (size_t)(src_row >= 0 ? src_row : 0) * dp * esz + (size_t)c * 128;
      const uint32_t nb = src_row >= 0 ? 16u : 0u;
#pragma unroll
      for (int pl = 0; pl < 2; ++pl)
#pragma unroll
        for (int j = 0; j < 8; ++j)
          cp16(sA + pl * a_bytes + rowoff + (uint32_t)((j ^ (tid & 7)) << 4), gsrc + pl * plane_stride + j * 16, nb);
      cp_commit();
      if (it >= 1) {  // the previous stage has landed: make it visible to the MMAs
        cp_wait1();
        fence_async_smem();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(full((it - 1) % S)) : "memory");
      }
    }
    cp_wait0();
    if (ok && nit >= 1) {
      fence_async_smem();
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(full((nit - 1) % S)) : "memory");
    }
  } else if (tid == kRows) {
    // ----------------------------------------------------- MMA issuer --
    const uint32_t id_lo = idesc(TF32 ? 2u : 1u, dp > 256 ? 256u : (uint32_t)dp);
    const uint32_t id_hi = idesc(TF32 ? 2u : 1u, dp > 256 ? (uint32_t)(dp - 256) : 16u);
    // descriptors of the stages' A and B plane 0 (S <= 3), counters instead
    // of divisions in this single-thread loop
    const uint64_t dA0 = sdesc(sbase), dA1 = sdesc(sbase + stage), dA2 = sdesc(sbase + 2 * stage);
    const uint64_t dB0 = dA0 + (2 * a_bytes >> 4), dB1 = dA1 + (2 * a_bytes >> 4), dB2 = dA2 + (2 * a_bytes >> 4);
    int st = 0, c = 0, e = 0, ch = 0;
    uint32_t ph = 0;
    for (int it = 0; it < nit; ++it) {
      if (!mbar_wait(full(st), ph, a.err, 2)) {
        ok = false;
        break;
      }
      tc_fence_after();
      // offsets go round-robin to `chains` accumulators: shorter FP32
      // accumulation chains, summed in FP64 by the epilogue
      const uint32_t dacc = tmem + (uint32_t)(ch * dp);
      const bool first = e < a.chains && c == 0;
      const uint64_t da = st == 0 ? dA0 : (st == 1 ? dA1 : dA2);
      const uint64_t db = st == 0 ? dB0 : (st == 1 ? dB1 : dB2);
      issue_chunk<TF32>(dacc, da, db, a_bytes >> 4, b_bytes >> 4, id_lo, id_hi, dp > 256, first);
      mma_commit(empty(st));
      if (++st == S) st = 0, ph ^= 1u;
      if (++c == nchunk) {
        c = 0;
        ++e;
        if (++ch == a.chains) ch = 0;
      }
    }
    if (ok && nit >= 1) mma_commit(done_bar);
  }
  // ---------------------------------------------------------- epilogue --
  if (tid < kRows) {
    bool have = nit >= 1 && ok;
    if (have) have = mbar_wait(done_bar, 0, a.err, 3);
    have = __all_sync(0xffffffffu, have);  // uniform per warp for tcgen05.ld
    tc_fence_after();
    float* out = a.out + (size_t)grp * a.part_stride + (size_t)(I * a.R + r) * dp;
    const uint32_t lane_base = (uint32_t)((tid & ~31) << 16);
    const int used = min(a.chains, *nact_p);
    for (int c0 = 0; c0 < dp; c0 += 16) {
      double v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.0;
      if (have)
        for (int ch = 0; ch < used; ++ch) {
          float t[16];
          tmem_ld16(tmem + lane_base + (uint32_t)(ch * dp + c0), t);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] += (double)t[i];
        }
      if (valid) {
        float4* o4 = (float4*)(out + c0);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          o4[i] = make_float4((float)v[4 * i], (float)v[4 * i + 1], (float)v[4 * i + 2], (float)v[4 * i + 3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid >= 128)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)a.tmem_cols));
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            int c3, int c4, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(mbar)
      : "memory");
}

// TMA variant.  What is stored per parity class on a grid,
// [plane][class][Z][Y][X*R + r][dp] with (X, Y, Z) = box coordinates / 2, so
// the 128 source rows of a tile for one offset form a regular box of that
// grid: one 5-D TMA tile load per plane brings them in, zero-filled outside
// the cube.  Warp 4 produces (TMA for A, bulk copy for B), warp 5 issues the
// MMAs, warps 0-3 drain the accumulators.  CTAs that share an offset read
// the same K^delta image; they find it in L2.
template <bool TF32>
__global__ void __launch_bounds__(192, 1)
k_m2l_tma(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1, M2LTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x;
  const int esz = TF32 ? 4 : 2;
  const int E = 128 / esz;
  const int dp = a.dp;
  const int S = a.stages;
  const int nchunk = dp * esz / 128;
  const uint32_t a_bytes = 16384u;
  const uint32_t b_bytes = (uint32_t)dp * 128u;
  const uint32_t stage = 2 * a_bytes + 2 * b_bytes;
  uint64_t* bars = (uint64_t*)(smem + S * stage);
  uint32_t* tslot = (uint32_t*)(bars + 2 * kMaxStages + 1);
  const uint32_t sbase = smem_u32(smem);
  auto full = [&](int st) { return smem_u32(&bars[st]); };
  auto empty = [&](int st) { return smem_u32(&bars[kMaxStages + st]); };
  const uint32_t done_bar = smem_u32(&bars[2 * kMaxStages]);

  const int h = a.h, R = a.R;
  const int bxr = a.bx * R;  // merged (x, r) rows of the tile
  const int oct = blockIdx.x % 8;
  const int grp = (blockIdx.x / 8) % a.groups;
  int tile = blockIdx.x / (8 * a.groups);
  const int ntx = (h * R + bxr - 1) / bxr, nty = (h + a.by - 1) / a.by;
  const int tx = tile % ntx;
  tile /= ntx;
  const int ty = tile % nty, tz = tile / nty;
  const int xr0 = tx * bxr, y0 = ty * a.by, z0 = tz * a.bz;
  const int cx = oct & 1, cy = (oct >> 1) & 1, cz = (oct >> 2) & 1;
  const int s_beg = grp * kListLen / a.groups, s_end = (grp + 1) * kListLen / a.groups;
  const int* lst = a.slot_lists + oct * kListLen;

  // the source block of an offset; empty when it misses the class grid
  auto source = [&](int slot, int* sc, int* sxr, int* sy, int* sz) {
    const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
    *sc = ((cx + dx) & 1) | (((cy + dy) & 1) << 1) | (((cz + dz) & 1) << 2);
    *sxr = xr0 + ((cx + dx) >> 1) * R;
    *sy = y0 + ((cy + dy) >> 1);
    *sz = z0 + ((cz + dz) >> 1);
    return *sxr < h * R && *sxr + bxr > 0 && *sy < h && *sy + a.by > 0 && *sz < h && *sz + a.bz > 0;
  };

  if (tid == 0) {
    for (int i = 0; i < kMaxStages; ++i) {
      mbar_init(full(i), 1);
      mbar_init(empty(i), 1);
    }
    mbar_init(done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid >= 128 && tid < 160) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"((uint32_t)a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // number of offsets walked (the same count in every thread)
  int nact = 0;
  for (int s = s_beg; s < s_end; ++s) {
    int sc, sxr, sy, sz;
    nact += source(lst[s], &sc, &sxr, &sy, &sz) ? 1 : 0;
  }
  const int nit = nact * nchunk;
  bool ok = true;

  if (tid == 128) {
    // -------------------------------------------------------- producer --
    int it = 0, pst = 0;
    uint32_t pph = 0;  // phase of the current round of the ring
    for (int s = s_beg; s < s_end && ok; ++s) {
      const int slot = lst[s];
      int sc, sxr, sy, sz;
      if (!source(slot, &sc, &sxr, &sy, &sz)) continue;
      for (int c = 0; c < nchunk && ok; ++c, ++it) {
        if (it >= S && !mbar_wait(empty(pst), pph ^ 1u, a.err, 1)) {
          ok = false;
          break;
        }
        const int st = pst;
        if (++pst == S) pst = 0, pph ^= 1u;
        const uint32_t sA = sbase + st * stage;
        mbar_expect_tx(full(st), 2 * a_bytes + 2 * b_bytes);
        tma_load_5d(sA, &tA0, c * E, sxr, sy, sz, sc, full(st));
        tma_load_5d(sA + a_bytes, &tA1, c * E, sxr, sy, sz, sc, full(st));
        const char* src = (const char*)a.kd_img + (((size_t)slot * nchunk + c) * 2) * b_bytes;
        bulk_g2s(sA + 2 * a_bytes, src, 2 * b_bytes, full(st));
      }
    }
    drain_fills(it, S, bars, a.err);
  } else if (tid == 160) {
    // ----------------------------------------------------- MMA issuer --
    const uint32_t id_lo = idesc(TF32 ? 2u : 1u, dp > 256 ? 256u : (uint32_t)dp);
    const uint32_t id_hi = idesc(TF32 ? 2u : 1u, dp > 256 ? (uint32_t)(dp - 256) : 16u);
    // descriptors of the stages' A and B plane 0 (S <= 3), counters instead
    // of divisions in this single-thread loop
    const uint64_t dA0 = sdesc(sbase), dA1 = sdesc(sbase + stage), dA2 = sdesc(sbase + 2 * stage);
    const uint64_t dB0 = dA0 + (2 * a_bytes >> 4), dB1 = dA1 + (2 * a_bytes >> 4), dB2 = dA2 + (2 * a_bytes >> 4);
    int st = 0, c = 0, e = 0, ch = 0;
    uint32_t ph = 0;
    for (int it = 0; it < nit; ++it) {
      if (!mbar_wait(full(st), ph, a.err, 2)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t dacc = tmem + (uint32_t)(ch * dp);
      const bool first = e < a.chains && c == 0;
      const uint64_t da = st == 0 ? dA0 : (st == 1 ? dA1 : dA2);
      const uint64_t db = st == 0 ? dB0 : (st == 1 ? dB1 : dB2);
      issue_chunk<TF32>(dacc, da, db, a_bytes >> 4, b_bytes >> 4, id_lo, id_hi, dp > 256, first);
      mma_commit(empty(st));
      if (++st == S) st = 0, ph ^= 1u;
      if (++c == nchunk) {
        c = 0;
        ++e;
        if (++ch == a.chains) ch = 0;
      }
    }
    if (ok && nit >= 1) mma_commit(done_bar);
  } else if (tid < 128) {
    // --------------------------------------------------------- epilogue --
    const int xr = xr0 + tid % bxr;
    const int yy = y0 + (tid / bxr) % a.by;
    const int zz = z0 + tid / (bxr * a.by);
    const bool valid = xr < h * R && yy < h && zz < h;
    const int x = valid ? xr / R : 0, r = valid ? xr % R : 0;
    const int64_t I = valid ? morton_encode(2 * x + cx, 2 * (valid ? yy : 0) + cy, 2 * (valid ? zz : 0) + cz, a.level) : 0;
    bool have = nit >= 1;
    if (have) have = mbar_wait(done_bar, 0, a.err, 3);
    have = __all_sync(0xffffffffu, have);
    tc_fence_after();
    float* out = a.out + (size_t)grp * a.part_stride + (size_t)(I * R + r) * dp;
    const uint32_t lane_base = (uint32_t)((tid & ~31) << 16);
    const int used = min(a.chains, nact);
    for (int c0 = 0; c0 < dp; c0 += 16) {
      float v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.f;
      if (have)
        for (int ch = 0; ch < used; ++ch) {
          float t[16];
          tmem_ld16(tmem + lane_base + (uint32_t)(ch * dp + c0), t);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] += t[i];
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
  if (tid >= 128 && tid < 160)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)a.tmem_cols));
}

// ---------------------------------------------------------------------------
// Transposed TMA M2L for dp = 128: D^t[m' x row] = K^delta[m' x l] What[row x l]^t
// with M = 128 (m'), N = 256 (target rows), K = l.  One tcgen05.mma then does
// twice the work of an M = 128, N = 128 one at the same issue cost, and the
// shared-memory operand traffic per flop drops by a quarter.
//
// The offsets are walked in segments of kSegOffsets.  A segment accumulates in
// one of two 256-column TMEM buffers (short FP32 accumulation chains) while
// the eight epilogue warps drain the other into FP32 registers; the register
// totals are stored once at the end.  Warp 8 produces (one bulk copy of the
// K^delta image, two 5-D TMA loads of the What planes per stage), warp 9
// issues the MMAs.
// ---------------------------------------------------------------------------
constexpr int kT2Rows = 256;
constexpr int kT2Stages = 2;
constexpr int kSegOffsets = 4;
constexpr int kT2Threads = 320;

// Bounded wait that also gives up when another role has set *abort.
__device__ __forceinline__ bool mbar_wait_ab(uint32_t a, uint32_t parity, int* err, int code,
                                             volatile int* abort) {
  const long long t0 = clock64();
  while (!mbar_try(a, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > kWaitCycles) {
      atomicExch(err, code);
      *abort = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
      "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <bool TF32>
__global__ void __launch_bounds__(kT2Threads, 1)
k_m2l_t256(const __grid_constant__ CUtensorMap tW0, const __grid_constant__ CUtensorMap tW1, M2LTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int esz = TF32 ? 4 : 2;
  const int E = 128 / esz;
  const int dp = a.dp;  // 128
  const int nchunk = dp * esz / 128;
  const uint32_t k_bytes = 128u * 128u;         // one K^delta plane: 128 rows x 128 B
  const uint32_t w_bytes = kT2Rows * 128u;      // one What plane: 256 rows x 128 B
  const uint32_t stage = 2 * k_bytes + 2 * w_bytes;
  uint64_t* bars = (uint64_t*)(smem + kT2Stages * stage);  // full[2] empty[2] sfull[2] sempty[2]
  uint32_t* tslot = (uint32_t*)(bars + 8);
  volatile int* abort = (volatile int*)(tslot + 1);
  int64_t* s_row = (int64_t*)(bars + 9);  // [256] output rows of the tile
  const uint32_t sbase = smem_u32(smem);
  auto full = [&](int st) { return smem_u32(&bars[st]); };
  auto empty = [&](int st) { return smem_u32(&bars[2 + st]); };
  auto sfull = [&](int b) { return smem_u32(&bars[4 + b]); };
  auto sempty = [&](int b) { return smem_u32(&bars[6 + b]); };

  const int h = a.h, R = a.R;
  const int bxr = a.bx * R;
  const int oct = blockIdx.x % 8;
  const int grp = (blockIdx.x / 8) % a.groups;
  int tile = blockIdx.x / (8 * a.groups);
  const int ntx = (h * R + bxr - 1) / bxr, nty = (h + a.by - 1) / a.by;
  const int tx = tile % ntx;
  tile /= ntx;
  const int ty = tile % nty, tz = tile / nty;
  const int xr0 = tx * bxr, y0 = ty * a.by, z0 = tz * a.bz;
  const int cx = oct & 1, cy = (oct >> 1) & 1, cz = (oct >> 2) & 1;
  const int s_beg = grp * kListLen / a.groups, s_end = (grp + 1) * kListLen / a.groups;
  const int* lst = a.slot_lists + oct * kListLen;

  // the source block of an offset; empty when it misses the class grid
  auto source = [&](int slot, int* sc, int* sxr, int* sy, int* sz) {
    const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
    *sc = ((cx + dx) & 1) | (((cy + dy) & 1) << 1) | (((cz + dz) & 1) << 2);
    *sxr = xr0 + ((cx + dx) >> 1) * R;
    *sy = y0 + ((cy + dy) >> 1);
    *sz = z0 + ((cz + dz) >> 1);
    return *sxr < h * R && *sxr + bxr > 0 && *sy < h && *sy + a.by > 0 && *sz < h && *sz + a.bz > 0;
  };

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(full(i), 1);
      mbar_init(empty(i), 1);
      mbar_init(sfull(i), 1);
      mbar_init(sempty(i), 8);  // one arrival per epilogue warp
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(512u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  int nact = 0;
  for (int s = s_beg; s < s_end; ++s) {
    int sc, sxr, sy, sz;
    nact += source(lst[s], &sc, &sxr, &sy, &sz) ? 1 : 0;
  }
  const int nseg = (nact + kSegOffsets - 1) / kSegOffsets;

  if (tid == 256) {
    // -------------------------------------------------------- producer --
    int it = 0, st = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int s = s_beg; s < s_end && ok; ++s) {
      const int slot = lst[s];
      int sc, sxr, sy, sz;
      if (!source(slot, &sc, &sxr, &sy, &sz)) continue;
      for (int c = 0; c < nchunk; ++c, ++it) {
        if (it >= kT2Stages && !mbar_wait_ab(empty(st), ph ^ 1u, a.err, 1, abort)) {
          ok = false;
          break;
        }
        const uint32_t sK = sbase + st * stage;
        const uint32_t sW = sK + 2 * k_bytes;
        mbar_expect_tx(full(st), 2 * k_bytes + 2 * w_bytes);
        bulk_g2s(sK, (const char*)a.kd_img + (((size_t)slot * nchunk + c) * 2) * k_bytes, 2 * k_bytes, full(st));
        tma_load_5d(sW, &tW0, c * E, sxr, sy, sz, sc, full(st));
        tma_load_5d(sW + w_bytes, &tW1, c * E, sxr, sy, sz, sc, full(st));
        if (++st == kT2Stages) st = 0, ph ^= 1u;
      }
    }
    drain_fills(it, kT2Stages, bars, a.err);
  } else if (tid == 288) {
    // ----------------------------------------------------- MMA issuer --
    const uint32_t id = idesc(TF32 ? 2u : 1u, (uint32_t)kT2Rows);
    const uint64_t dK0 = sdesc(sbase), dK1 = sdesc(sbase + stage);
    const uint64_t dW0 = dK0 + (2 * k_bytes >> 4), dW1 = dK1 + (2 * k_bytes >> 4);
    int st = 0, done = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int seg = 0; seg < nseg && ok; ++seg) {
      const int b = seg & 1;
      if (seg >= 2 && !mbar_wait_ab(sempty(b), ((seg >> 1) - 1) & 1, a.err, 4, abort)) break;
      tc_fence_after();
      const uint32_t dacc = tmem + (uint32_t)(b * kT2Rows);
      const int nit = min(kSegOffsets, nact - done) * nchunk;
      for (int i = 0; i < nit; ++i) {
        if (!mbar_wait_ab(full(st), ph, a.err, 2, abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // A = K^delta planes (M), B = What planes (N): hi*hi, hi*lo, lo*hi
        issue_chunk<TF32>(dacc, st == 0 ? dK0 : dK1, st == 0 ? dW0 : dW1, k_bytes >> 4, w_bytes >> 4, id, id,
                          false, i == 0);
        mma_commit(empty(st));
        if (++st == kT2Stages) st = 0, ph ^= 1u;
      }
      done += kSegOffsets;
      if (ok) mma_commit(sfull(b));
    }
  } else if (warp < 8) {
    // ------------------------------------------------------ epilogue --
    // warp w reads TMEM lanes 32 (w % 4) .. (m' rows) and columns
    // 128 (w / 4) .. of the 256 target rows
    const int q = warp & 3, half = warp >> 2;
    float acc[128];
#pragma unroll
    for (int j = 0; j < 128; ++j) acc[j] = 0.f;
    for (int seg = 0; seg < nseg; ++seg) {
      const int b = seg & 1;
      bool have = mbar_wait_ab(sfull(b), (seg >> 1) & 1, a.err, 3, abort);
      have = __all_sync(0xffffffffu, have);
      if (!have) break;
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kT2Rows + 128 * half);
#pragma unroll
      for (int j0 = 0; j0 < 128; j0 += 32) {
        float v[32];
        tmem_ld32(taddr + j0, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[j0 + i] += v[i];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sempty(b)) : "memory");
    }
    // output row of each of the 256 tile rows (x*R + r fastest, then y,
    // then z), -1 outside the grid: one per epilogue thread, then shared
    {
      const int n = tid;
      const int xr = xr0 + n % bxr;
      const int yy = y0 + (n / bxr) % a.by;
      const int zz = z0 + n / (bxr * a.by);
      int64_t row = -1;
      if (xr < h * R && yy < h && zz < h) {
        const int x = xr / R, r = xr % R;
        row = morton_encode(2 * x + cx, 2 * yy + cy, 2 * zz + cz, a.level) * R + r;
      }
      s_row[n] = row;
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");  // the eight epilogue warps
    const int mp = 32 * q + lane;  // m'
    float* outg = a.out + (size_t)grp * a.part_stride + mp;
#pragma unroll
    for (int j = 0; j < 128; ++j) {
      const int64_t row = s_row[128 * half + j];
      if (row >= 0) outg[row * dp] = acc[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 8)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
}

// ---------------------------------------------------------------------------
// Stream-K form of the transposed M2L for one level: exactly one CTA per SM.
// The work is the sequence of (tile, active offset) units over all tiles
// (tile t: parity class t / tpc, tile t % tpc of that class; tu[t] = units
// before tile t); CTA c takes units [c U / N, (c + 1) U / N).  Its pieces
// (the part of one tile inside its range) run through the same producer /
// MMA / segment-drain pipeline as k_m2l_t256, the rings and the TMEM
// buffers continuing from one piece to the next.  A piece that covers its
// whole tile writes g; any other writes a partial tile (256 rows x 128 m') to
// slot 2c (the CTA's first piece) or 2c + 1 (its last), and k_sk_fixup adds
// the partials of each split tile in CTA order.  No CTA waits on another.
// ---------------------------------------------------------------------------
struct SkPlan {
  const int* tu;      // [ntiles + 1] units before each tile
  int ntiles, tpc;    // tiles, tiles per parity class
  int nctas;
  float* part;        // [2 nctas][256][128] partial tiles
};

template <bool TF32>
__global__ void __launch_bounds__(kT2Threads, 1)
k_m2l_t256s(const __grid_constant__ CUtensorMap tW0, const __grid_constant__ CUtensorMap tW1, M2LTcArgs a,
            SkPlan sk) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int esz = TF32 ? 4 : 2;
  const int E = 128 / esz;
  const int dp = a.dp;  // 128
  const int nchunk = dp * esz / 128;
  const uint32_t k_bytes = 128u * 128u;
  const uint32_t w_bytes = kT2Rows * 128u;
  const uint32_t stage = 2 * k_bytes + 2 * w_bytes;
  uint64_t* bars = (uint64_t*)(smem + kT2Stages * stage);  // full[2] empty[2] sfull[2] sempty[2]
  uint32_t* tslot = (uint32_t*)(bars + 8);
  volatile int* abort = (volatile int*)(tslot + 1);
  int64_t* s_row = (int64_t*)(bars + 9);  // [256] output rows of the current tile
  const uint32_t sbase = smem_u32(smem);
  auto full = [&](int st) { return smem_u32(&bars[st]); };
  auto empty = [&](int st) { return smem_u32(&bars[2 + st]); };
  auto sfull = [&](int b) { return smem_u32(&bars[4 + b]); };
  auto sempty = [&](int b) { return smem_u32(&bars[6 + b]); };

  const int h = a.h, R = a.R;
  const int bxr = a.bx * R;
  const int ntx = (h * R + bxr - 1) / bxr, nty = (h + a.by - 1) / a.by;
  const int c = blockIdx.x;
  const int U = sk.tu[sk.ntiles];
  const int u0 = (int)((int64_t)c * U / sk.nctas), u1 = (int)((int64_t)(c + 1) * U / sk.nctas);
  int t_first = 0;  // the tile holding unit u0: the last t with tu[t] <= u0
  {
    int lo = 0, hi = sk.ntiles - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sk.tu[mid] <= u0) lo = mid;
      else hi = mid - 1;
    }
    t_first = lo;
  }
  // geometry of tile t: parity class, first (x r, y, z) of its block
  struct Geo {
    int oct, cx, cy, cz, xr0, y0, z0;
  };
  auto geo = [&](int t) {
    Geo g;
    g.oct = t / sk.tpc;
    int tile = t % sk.tpc;
    const int tx = tile % ntx;
    tile /= ntx;
    const int ty = tile % nty, tz = tile / nty;
    g.xr0 = tx * bxr;
    g.y0 = ty * a.by;
    g.z0 = tz * a.bz;
    g.cx = g.oct & 1;
    g.cy = (g.oct >> 1) & 1;
    g.cz = (g.oct >> 2) & 1;
    return g;
  };
  auto source = [&](const Geo& g, int slot, int* sc, int* sxr, int* sy, int* sz) {
    const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
    *sc = ((g.cx + dx) & 1) | (((g.cy + dy) & 1) << 1) | (((g.cz + dz) & 1) << 2);
    *sxr = g.xr0 + ((g.cx + dx) >> 1) * R;
    *sy = g.y0 + ((g.cy + dy) >> 1);
    *sz = g.z0 + ((g.cz + dz) >> 1);
    return *sxr < h * R && *sxr + bxr > 0 && *sy < h && *sy + a.by > 0 && *sz < h && *sz + a.bz > 0;
  };

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(full(i), 1);
      mbar_init(empty(i), 1);
      mbar_init(sfull(i), 1);
      mbar_init(sempty(i), 8);  // one arrival per epilogue warp
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(512u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (tid == 256) {
    // -------------------------------------------------------- producer --
    int it = 0, st = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int t = t_first; t < sk.ntiles && sk.tu[t] < u1 && ok; ++t) {
      const int lo = max(u0, sk.tu[t]) - sk.tu[t], hi = min(u1, sk.tu[t + 1]) - sk.tu[t];
      const Geo g = geo(t);
      const int* lst = a.slot_lists + g.oct * kListLen;
      int ai = 0;  // index among the tile's active offsets
      for (int s = 0; s < kListLen && ai < hi && ok; ++s) {
        const int slot = lst[s];
        int sc, sxr, sy, sz;
        if (!source(g, slot, &sc, &sxr, &sy, &sz)) continue;
        if (ai++ < lo) continue;
        for (int cc = 0; cc < nchunk; ++cc, ++it) {
          if (it >= kT2Stages && !mbar_wait_ab(empty(st), ph ^ 1u, a.err, 1, abort)) {
            ok = false;
            break;
          }
          const uint32_t sK = sbase + st * stage;
          const uint32_t sW = sK + 2 * k_bytes;
          mbar_expect_tx(full(st), 2 * k_bytes + 2 * w_bytes);
          bulk_g2s(sK, (const char*)a.kd_img + (((size_t)slot * nchunk + cc) * 2) * k_bytes, 2 * k_bytes, full(st));
          tma_load_5d(sW, &tW0, cc * E, sxr, sy, sz, sc, full(st));
          tma_load_5d(sW + w_bytes, &tW1, cc * E, sxr, sy, sz, sc, full(st));
          if (++st == kT2Stages) st = 0, ph ^= 1u;
        }
      }
    }
    drain_fills(it, kT2Stages, bars, a.err);
  } else if (tid == 288) {
    // ----------------------------------------------------- MMA issuer --
    const uint32_t id = idesc(TF32 ? 2u : 1u, (uint32_t)kT2Rows);
    const uint64_t dK0 = sdesc(sbase), dK1 = sdesc(sbase + stage);
    const uint64_t dW0 = dK0 + (2 * k_bytes >> 4), dW1 = dK1 + (2 * k_bytes >> 4);
    int st = 0, seg = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int t = t_first; t < sk.ntiles && sk.tu[t] < u1 && ok; ++t) {
      const int n_here = min(u1, sk.tu[t + 1]) - max(u0, sk.tu[t]);
      for (int done = 0; done < n_here && ok; done += kSegOffsets, ++seg) {
        const int b = seg & 1;
        if (seg >= 2 && !mbar_wait_ab(sempty(b), ((seg >> 1) - 1) & 1, a.err, 4, abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(b * kT2Rows);
        const int nit = min(kSegOffsets, n_here - done) * nchunk;
        for (int i = 0; i < nit; ++i) {
          if (!mbar_wait_ab(full(st), ph, a.err, 2, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          issue_chunk<TF32>(dacc, st == 0 ? dK0 : dK1, st == 0 ? dW0 : dW1, k_bytes >> 4, w_bytes >> 4, id, id,
                            false, i == 0);
          mma_commit(empty(st));
          if (++st == kT2Stages) st = 0, ph ^= 1u;
        }
        if (ok) mma_commit(sfull(b));
      }
    }
  } else if (warp < 8) {
    // ------------------------------------------------------ epilogue --
    const int q = warp & 3, half = warp >> 2;
    const int mp = 32 * q + lane;  // m'
    // every epilogue warp runs through every piece and both named barriers of
    // each, whatever a wait returns, so that the barriers always match
    int seg = 0;
    bool have = true;
    for (int t = t_first; t < sk.ntiles && sk.tu[t] < u1; ++t) {
      const int lo = max(u0, sk.tu[t]) - sk.tu[t], hi = min(u1, sk.tu[t + 1]) - sk.tu[t];
      const int n_here = hi - lo;
      if (n_here <= 0) continue;  // a tile without units: the fix-up writes its zeros
      float acc[128];
#pragma unroll
      for (int j = 0; j < 128; ++j) acc[j] = 0.f;
      for (int done = 0; done < n_here; done += kSegOffsets, ++seg) {
        const int b = seg & 1;
        if (have) have = mbar_wait_ab(sfull(b), (seg >> 1) & 1, a.err, 3, abort);
        have = __all_sync(0xffffffffu, have);
        if (!have) continue;
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kT2Rows + 128 * half);
#pragma unroll
        for (int j0 = 0; j0 < 128; j0 += 32) {
          float v[32];
          tmem_ld32(taddr + j0, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[j0 + i] += v[i];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sempty(b)) : "memory");
      }
      const bool whole = lo == 0 && hi == sk.tu[t + 1] - sk.tu[t];
      asm volatile("bar.sync 1, 256;" ::: "memory");  // the previous tile's rows are read
      {
        const Geo g = geo(t);
        const int n = tid;
        const int xr = g.xr0 + n % bxr;
        const int yy = g.y0 + (n / bxr) % a.by;
        const int zz = g.z0 + n / (bxr * a.by);
        int64_t row = -1;
        if (xr < h * R && yy < h && zz < h) {
          const int x = xr / R, r = xr % R;
          row = morton_encode(2 * x + g.cx, 2 * yy + g.cy, 2 * zz + g.cz, a.level) * R + r;
        }
        s_row[n] = row;
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (!have) continue;
      if (whole) {
        float* outg = a.g + mp;
#pragma unroll
        for (int j = 0; j < 128; ++j) {
          const int64_t row = s_row[128 * half + j];
          if (row >= 0) outg[row * dp] = acc[j];
        }
      } else {
        // slot 2c for the CTA's first piece, 2c + 1 for any later one
        float* slot = sk.part + ((size_t)(2 * c + (t == t_first ? 0 : 1)) * kT2Rows) * 128 + mp;
#pragma unroll
        for (int j = 0; j < 128; ++j) slot[(size_t)(128 * half + j) * 128] = acc[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 8)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
}

// The split tiles of the stream-K M2L: tile fix_t[i] is the sum, in CTA
// order, of the partial slots fix_slot[fix_b[i] .. fix_b[i + 1]) (none: a
// tile without active offsets, g = 0).  Block (i, y) takes rows 32 y .. 32 y
// + 31 of split tile i: warp w rows 32 y + 4 w .. + 3, lane j the 16-byte
// word j of each row, so that every read of a partial row and every write of
// g is one coalesced 512-byte access, with the four rows' reads in flight
// together.
constexpr int kSkFixRowsPerWarp = 4;
__global__ void __launch_bounds__(256)
k_sk_fixup(M2LTcArgs a, SkPlan sk, const int* __restrict__ fix_t, const int* __restrict__ fix_b,
           const int* __restrict__ fix_slot) {
  const int i = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = fix_t[i];
  const int h = a.h, R = a.R, bxr = a.bx * R;
  const int ntx = (h * R + bxr - 1) / bxr, nty = (h + a.by - 1) / a.by;
  const int oct = t / sk.tpc;
  int tile = t % sk.tpc;
  const int tx = tile % ntx;
  tile /= ntx;
  const int ty = tile % nty, tz = tile / nty;
  const int kb = fix_b[i], ke = fix_b[i + 1];
  const int n0 = 32 * (int)blockIdx.y + kSkFixRowsPerWarp * w;
  float4 v[kSkFixRowsPerWarp];
#pragma unroll
  for (int u = 0; u < kSkFixRowsPerWarp; ++u) v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k = kb; k < ke; ++k) {
    const float4* __restrict__ src = reinterpret_cast<const float4*>(sk.part + ((size_t)fix_slot[k] * kT2Rows + n0) * 128);
    float4 p[kSkFixRowsPerWarp];
#pragma unroll
    for (int u = 0; u < kSkFixRowsPerWarp; ++u) p[u] = src[u * 32 + lane];
#pragma unroll
    for (int u = 0; u < kSkFixRowsPerWarp; ++u) {
      v[u].x += p[u].x;
      v[u].y += p[u].y;
      v[u].z += p[u].z;
      v[u].w += p[u].w;
    }
  }
#pragma unroll
  for (int u = 0; u < kSkFixRowsPerWarp; ++u) {
    const int n = n0 + u;
    const int xr = tx * bxr + n % bxr;
    const int yy = ty * a.by + (n / bxr) % a.by;
    const int zz = tz * a.bz + n / (bxr * a.by);
    if (!(xr < h * R && yy < h && zz < h)) continue;
    const int x = xr / R, r = xr % R;
    const int64_t row =
        morton_encode(2 * x + (oct & 1), 2 * yy + ((oct >> 1) & 1), 2 * zz + ((oct >> 2) & 1), a.level) * R + r;
    reinterpret_cast<float4*>(a.g + row * a.dp)[lane] = v[u];
  }
}

// ---------------------------------------------------------------------------
// FP16 M2L with per-offset drains (tier 1): M = 128 target rows, N = DP
// coefficients m', K = l; operands are FP16 hi + lo planes, 3 products.
// FP16 keeps 11 significant bits per plane against BF16's 8, so the split
// operand holds about 22 bits; its narrow exponent range is met by scaling:
// W of a level by a power of two s_W (its largest entry near 2^14) and row
// m' of K^delta Delta by a power of two s_m' (common to all offsets), both
// undone exactly in the epilogue.  The tensor core's FP32 accumulation
// chain is cut after every offset: the 3 x K products of one offset go to
// one of two TMEM accumulators while the eight drain warps read the other
// with tcgen05.ld and add it, in round-to-nearest FP32, to running sums in
// registers.  Warp 8 produces (two 5-D TMA loads of the W planes and one
// bulk copy of the K^delta image per stage), warp 9 issues the MMAs; warp w
// < 8 drains TMEM lanes 32 (w % 4) (tile rows) and columns DP/2 (w / 4).
// ---------------------------------------------------------------------------
constexpr int kH16Threads = 320;
constexpr int kH16Stages = 2;

template <int DP>
__global__ void __launch_bounds__(kH16Threads, 1)
k_m2l_h16(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1, M2LTcArgs a,
          const uint32_t* __restrict__ wmax, const float* __restrict__ kscale) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int E = 64;                 // FP16 elements per 128-byte chunk
  constexpr int NCH = DP / E;           // chunks of l per offset
  constexpr int HALF = DP / 2;          // columns per drain warp
  constexpr uint32_t a_bytes = 16384u;  // 128 rows x 128 B per plane
  constexpr uint32_t b_bytes = DP * 128u;
  constexpr uint32_t stage = 2 * a_bytes + 2 * b_bytes;
  constexpr uint32_t tcols = 2 * DP <= 128 ? 128 : (2 * DP <= 256 ? 256 : 512);
  uint64_t* bars = (uint64_t*)(smem + kH16Stages * stage);  // full[2] empty[2] afull[2] aempty[2]
  uint32_t* tslot = (uint32_t*)(bars + 8);
  volatile int* abort = (volatile int*)(tslot + 1);
  float* s_inv = (float*)(bars + 9);  // [DP] 1 / (s_W s_m')
  const uint32_t sbase = smem_u32(smem);
  auto full = [&](int st) { return smem_u32(&bars[st]); };
  auto empty = [&](int st) { return smem_u32(&bars[2 + st]); };
  auto afull = [&](int b) { return smem_u32(&bars[4 + b]); };
  auto aempty = [&](int b) { return smem_u32(&bars[6 + b]); };

  const int h = a.h, R = a.R;
  const int bxr = a.bx * R;
  const int oct = blockIdx.x % 8;
  const int grp = (blockIdx.x / 8) % a.groups;
  int tile = blockIdx.x / (8 * a.groups);
  const int ntx = (h * R + bxr - 1) / bxr, nty = (h + a.by - 1) / a.by;
  const int tx = tile % ntx;
  tile /= ntx;
  const int ty = tile % nty, tz = tile / nty;
  const int xr0 = tx * bxr, y0 = ty * a.by, z0 = tz * a.bz;
  const int cx = oct & 1, cy = (oct >> 1) & 1, cz = (oct >> 2) & 1;
  const int s_beg = grp * kListLen / a.groups, s_end = (grp + 1) * kListLen / a.groups;
  const int* lst = a.slot_lists + oct * kListLen;

  auto source = [&](int slot, int* sc, int* sxr, int* sy, int* sz) {
    const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
    *sc = ((cx + dx) & 1) | (((cy + dy) & 1) << 1) | (((cz + dz) & 1) << 2);
    *sxr = xr0 + ((cx + dx) >> 1) * R;
    *sy = y0 + ((cy + dy) >> 1);
    *sz = z0 + ((cz + dz) >> 1);
    return *sxr < h * R && *sxr + bxr > 0 && *sy < h && *sy + a.by > 0 && *sz < h && *sz + a.bz > 0;
  };

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(full(i), 1);
      mbar_init(empty(i), 1);
      mbar_init(afull(i), 1);
      mbar_init(aempty(i), 8);  // one arrival per drain warp
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    const float sw = f16_plane_scale(__uint_as_float(wmax[a.level]));
    for (int j = tid; j < DP; j += kH16Threads) s_inv[j] = 1.0f / (sw * kscale[j]);  // powers of two
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  int nact = 0;
  for (int s = s_beg; s < s_end; ++s) {
    int sc, sxr, sy, sz;
    nact += source(lst[s], &sc, &sxr, &sy, &sz) ? 1 : 0;
  }

  if (tid == 256) {
    // -------------------------------------------------------- producer --
    int it = 0, st = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int s = s_beg; s < s_end && ok; ++s) {
      const int slot = lst[s];
      int sc, sxr, sy, sz;
      if (!source(slot, &sc, &sxr, &sy, &sz)) continue;
      for (int c = 0; c < NCH; ++c, ++it) {
        if (it >= kH16Stages && !mbar_wait_ab(empty(st), ph ^ 1u, a.err, 1, abort)) {
          ok = false;
          break;
        }
        const uint32_t sA = sbase + st * stage;
        mbar_expect_tx(full(st), 2 * a_bytes + 2 * b_bytes);
        tma_load_5d(sA, &tA0, c * E, sxr, sy, sz, sc, full(st));
        tma_load_5d(sA + a_bytes, &tA1, c * E, sxr, sy, sz, sc, full(st));
        bulk_g2s(sA + 2 * a_bytes, (const char*)a.kd_img + (((size_t)slot * NCH + c) * 2) * b_bytes,
                 2 * b_bytes, full(st));
        if (++st == kH16Stages) st = 0, ph ^= 1u;
      }
    }
    drain_fills(it, kH16Stages, bars, a.err);
  } else if (tid == 288) {
    // ----------------------------------------------------- MMA issuer --
    const uint32_t id = idesc(0u /* F16 */, (uint32_t)DP);
    const uint64_t dA0 = sdesc(sbase), dA1 = sdesc(sbase + stage);
    const uint64_t dB0 = dA0 + (2 * a_bytes >> 4), dB1 = dA1 + (2 * a_bytes >> 4);
    int st = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int e = 0; e < nact && ok; ++e) {
      const int b = e & 1;
      if (e >= 2 && !mbar_wait_ab(aempty(b), ((e >> 1) - 1) & 1, a.err, 4, abort)) break;
      tc_fence_after();
      const uint32_t dacc = tmem + (uint32_t)(b * DP);
      for (int c = 0; c < NCH; ++c) {
        if (!mbar_wait_ab(full(st), ph, a.err, 2, abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        issue_chunk<false>(dacc, st == 0 ? dA0 : dA1, st == 0 ? dB0 : dB1, a_bytes >> 4, b_bytes >> 4, id, id,
                           false, c == 0);
        mma_commit(empty(st));
        if (++st == kH16Stages) st = 0, ph ^= 1u;
      }
      if (ok) mma_commit(afull(b));
    }
  } else if (warp < 8) {
    // ------------------------------------------------------- drains --
    const int q = warp & 3, hf = warp >> 2;
    float acc[HALF];
#pragma unroll
    for (int j = 0; j < HALF; ++j) acc[j] = 0.f;
    for (int e = 0; e < nact; ++e) {
      const int b = e & 1;
      bool have = mbar_wait_ab(afull(b), (e >> 1) & 1, a.err, 3, abort);
      have = __all_sync(0xffffffffu, have);
      if (!have) break;
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * DP + HALF * hf);
#pragma unroll
      for (int j0 = 0; j0 < HALF; j0 += 32) {
        float v[32];
        tmem_ld32(taddr + j0, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[j0 + i] += v[i];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(aempty(b)) : "memory");
    }
    // tile row 32 q + lane: (x R + r fastest, then y, then z)
    const int t = 32 * q + lane;
    const int xr = xr0 + t % bxr;
    const int yy = y0 + (t / bxr) % a.by;
    const int zz = z0 + t / (bxr * a.by);
    if (xr < h * R && yy < h && zz < h) {
      const int x = xr / R, r = xr % R;
      const int64_t I = morton_encode(2 * x + cx, 2 * yy + cy, 2 * zz + cz, a.level);
      float* out = a.out + (size_t)grp * a.part_stride + (size_t)(I * R + r) * DP + HALF * hf;
      const float* inv = s_inv + HALF * hf;
#pragma unroll
      for (int j = 0; j < HALF; j += 4)
        *reinterpret_cast<float4*>(out + j) =
            make_float4(acc[j] * inv[j], acc[j + 1] * inv[j + 1], acc[j + 2] * inv[j + 2], acc[j + 3] * inv[j + 3]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 8)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

__global__ void k_sum_parts(const float4* __restrict__ parts, int groups, int64_t n4, int64_t stride4,
                            float4* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    // pairwise over the groups (at most 16 partial sums)
    float4 v[16];
    for (int g = 0; g < groups; ++g) v[g] = parts[g * stride4 + i];
    for (int w = 1; w < groups; w <<= 1)
      for (int g = 0; g + w < groups; g += 2 * w) {
        v[g].x += v[g + w].x;
        v[g].y += v[g + w].y;
        v[g].z += v[g + w].z;
        v[g].w += v[g + w].w;
      }
    out[i] = v[0];
  }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that
// nothing completes, with the wait routine of the kernels above and a
// limit of `limit` cycles; it records code 7 and returns.  No copy, MMA or
// tensor memory is involved, so giving up leaves nothing in flight.
__global__ void k_wait_selftest(long long limit, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait_lim(smem_u32(&bar), 0, err, 7, limit);
  }
}

}  // namespace

eifmm_status wait_selftest(long long limit, int* code) {
  int* err = nullptr;
  EIFMM_TRY(dalloc(&err, 1));
  eifmm_status rc = EIFMM_OK;
  int h = 0;
  if (cudaMemset(err, 0, sizeof(int)) != cudaSuccess) rc = EIFMM_ECUDA;
  if (rc == EIFMM_OK) {
    k_wait_selftest<<<1, 32>>>(limit, err);
    count_launch();
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      set_error("eifmm_wait_selftest: launch failed");
      rc = EIFMM_ECUDA;
    }
  }
  dfree(err);
  if (rc != EIFMM_OK) return rc;
  if (code) *code = h;
  if (h != 0) {
    set_error("eifmm_wait_selftest: the bounded wait gave up (code " + std::to_string(h) + ")");
    return EIFMM_ETIMEOUT;
  }
  return EIFMM_OK;
}

int m2l_tc_stages(int dp) {
  const size_t stage = 2 * 16384 + 2 * (size_t)dp * 128;
  return (3 * stage + 4096 <= 227 * 1024) ? 3 : 2;
}

size_t m2l_tc_smem_bytes(int dp, bool tf32) {
  (void)tf32;
  const size_t stage = 2 * 16384 + 2 * (size_t)dp * 128;
  return (size_t)m2l_tc_stages(dp) * stage + 1024 /* align */ + 2048 /* barriers, slot lists */;
}

int m2l_tc_groups(int64_t tiles8, int nsm, int dp) {
  // Split the interaction list over more CTAs (partial sums added in FP64
  // by k_sum_parts): at least two waves of CTAs, and at least 16 FP32
  // accumulation chains per output together with the in-CTA chains.
  const int chains = dp <= 128 ? 4 : (dp <= 256 ? 2 : 1);
  constexpr int gmin = 16;
  int g = 1;
  while (g < 16 && (tiles8 * g < 2 * nsm || chains * g < gmin)) g *= 2;
  return g;
}

// Tile block of the grid layout for R right-hand sides (R a power of two <= 128):
// bx boxes x R rhs along x, by along y, bz along z, 128 rows in all.
// 256-row target tile of the transposed M2L: bx x by x bz boxes x R rows.
bool m2l_t256_block(int R, int* bx, int* by, int* bz) {
  if (R < 1 || R > 256 || (R & (R - 1))) return false;
  *bx = R >= 8 ? 1 : 8 / R;
  const int rem = 256 / (*bx * R);
  *by = rem >= 8 ? 8 : rem;
  *bz = rem / *by;
  return true;
}

// Offset groups of the transposed M2L: the fewest that occupy three quarters
// of the SMs (each extra group costs a pass over its partial sums).
int m2l_t256_groups(int64_t ctas, int nsm) {
  int g = 1;
  while (g < 16 && ctas * g * 4 < (int64_t)nsm * 3) g *= 2;
  return g;
}

bool m2l_tma_block(int R, int* bx, int* by, int* bz) {
  if (R < 1 || R > 128 || (R & (R - 1))) return false;
  *bx = R >= 8 ? 1 : 8 / R;
  const int rem = 128 / (*bx * R);
  *by = rem >= 4 ? 4 : rem;
  *bz = rem / *by;
  return true;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// Tensor map of one What plane in the grid layout of level `level`.
eifmm_status make_plane_map(void* map, void* base, int level, int R, int dp, int fmt, int rows) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return EIFMM_ECUDA;
  }
  int bx, by, bz;
  if (!(rows == 256 ? m2l_t256_block(R, &bx, &by, &bz) : m2l_tma_block(R, &bx, &by, &bz))) {
    set_error("no TMA tile shape for this number of right-hand sides");
    return EIFMM_EUNSUPPORTED;
  }
  const bool tf32 = fmt == kPlaneTF32;
  const int esz = tf32 ? 4 : 2;
  const uint64_t h = (uint64_t)1 << (level - 1);
  cuuint64_t dims[5] = {(cuuint64_t)dp, h * R, h, h, 8};
  cuuint64_t strides[4] = {(cuuint64_t)dp * esz, h * R * dp * esz, h * h * R * dp * esz, h * h * h * R * dp * esz};
  cuuint32_t box[5] = {(cuuint32_t)(128 / esz), (cuuint32_t)(bx * R), (cuuint32_t)by, (cuuint32_t)bz, 1};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : (fmt == kPlaneF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  const CUresult r = fn((CUtensorMap*)map, dt,
                        5, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return EIFMM_ECUDA;
  }
  return EIFMM_OK;
}

// One-time launch setup (the shared-memory limit of a kernel) belongs to one
// device's context, so it is remembered per device.
constexpr int kMaxDevices = 64;
static int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

eifmm_status launch_m2l_tma(const M2LTcArgs& a0, const void* map0, const void* map1, bool tf32,
                            cudaStream_t s) {
  if (tf32) {  // the TF32 planes of an earlier tier are no longer built
    set_error("tensor-core M2L: TF32 operand planes are not built (BF16 and FP16 only)");
    return EIFMM_EUNSUPPORTED;
  }
  M2LTcArgs a = a0;
  a.stages = m2l_tc_stages(a.dp);
  a.chains = a.dp <= 128 ? 4 : (a.dp <= 256 ? 2 : 1);
  a.tmem_cols = 512;
  if (!m2l_tma_block(a.R, &a.bx, &a.by, &a.bz)) {
    set_error("no TMA tile shape for this number of right-hand sides");
    return EIFMM_EUNSUPPORTED;
  }
  a.h = 1 << (a.level - 1);
  const size_t sm = m2l_tc_smem_bytes(a.dp, tf32);
  const int bxr = a.bx * a.R;
  const int64_t tiles = (int64_t)((a.h * a.R + bxr - 1) / bxr) * ((a.h + a.by - 1) / a.by) * ((a.h + a.bz - 1) / a.bz);
  if (a.groups > 1) {
    a.out = a.part;
    a.part_stride = a.rows * (int64_t)a.dp;
  } else {
    a.out = a.g;
    a.part_stride = 0;
  }
  static bool attr[kMaxDevices][2] = {};
  const int dev = current_device();
  if (dev >= kMaxDevices || !attr[dev][tf32]) {
    EIFMM_CUDA(cudaFuncSetAttribute(k_m2l_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    if (dev < kMaxDevices) attr[dev][tf32] = true;
  }
  const unsigned grid = (unsigned)(tiles * 8 * a.groups);
  const CUtensorMap& m0 = *(const CUtensorMap*)map0;
  const CUtensorMap& m1 = *(const CUtensorMap*)map1;
  k_m2l_tma<false><<<grid, 192, sm, s>>>(m0, m1, a);
  EIFMM_CHECK_LAUNCH();
  if (a.groups > 1) {
    const int64_t n4 = a.rows * (int64_t)a.dp / 4;
    k_sum_parts<<<(unsigned)((n4 + 255) / 256 < 4096 ? (n4 + 255) / 256 : 4096), 256, 0, s>>>(
        (const float4*)a.part, a.groups, n4, a.part_stride / 4, (float4*)a.g);
    EIFMM_CHECK_LAUNCH();
  }
  return EIFMM_OK;
}

size_t m2l_t256_smem_bytes() { return (size_t)kT2Stages * (2 * 16384 + 2 * kT2Rows * 128) + 1024 + 128 + 8 * kT2Rows; }

eifmm_status launch_m2l_t256(const M2LTcArgs& a0, const void* map0, const void* map1, bool tf32, cudaStream_t s) {
  if (tf32) {  // the TF32 planes of an earlier tier are no longer built
    set_error("tensor-core M2L: TF32 operand planes are not built (BF16 and FP16 only)");
    return EIFMM_EUNSUPPORTED;
  }
  M2LTcArgs a = a0;
  if (a.dp != 128 || !m2l_t256_block(a.R, &a.bx, &a.by, &a.bz)) {
    set_error("transposed M2L: needs dp = 128 and a tile shape for R");
    return EIFMM_EUNSUPPORTED;
  }
  a.h = 1 << (a.level - 1);
  const int bxr = a.bx * a.R;
  const int64_t tiles =
      (int64_t)((a.h * a.R + bxr - 1) / bxr) * ((a.h + a.by - 1) / a.by) * ((a.h + a.bz - 1) / a.bz);
  if (a.groups > 1) {
    a.out = a.part;
    a.part_stride = a.rows * (int64_t)a.dp;
  } else {
    a.out = a.g;
    a.part_stride = 0;
  }
  const size_t sm = m2l_t256_smem_bytes();
  static bool attr[kMaxDevices][2] = {};
  const int dev = current_device();
  if (dev >= kMaxDevices || !attr[dev][tf32]) {
    EIFMM_CUDA(cudaFuncSetAttribute(k_m2l_t256<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    if (dev < kMaxDevices) attr[dev][tf32] = true;
  }
  const unsigned grid = (unsigned)(tiles * 8 * a.groups);
  const CUtensorMap& m0 = *(const CUtensorMap*)map0;
  const CUtensorMap& m1 = *(const CUtensorMap*)map1;
  k_m2l_t256<false><<<grid, kT2Threads, sm, s>>>(m0, m1, a);
  EIFMM_CHECK_LAUNCH();
  if (a.groups > 1) {
    const int64_t n4 = a.rows * (int64_t)a.dp / 4;
    k_sum_parts<<<(unsigned)((n4 + 255) / 256 < 4096 ? (n4 + 255) / 256 : 4096), 256, 0, s>>>(
        (const float4*)a.part, a.groups, n4, a.part_stride / 4, (float4*)a.g);
    EIFMM_CHECK_LAUNCH();
  }
  return EIFMM_OK;
}

size_t m2l_h16_smem_bytes(int dp) {
  return (size_t)kH16Stages * (2 * 16384 + 2 * (size_t)dp * 128) + 1024 + 128 + 4 * (size_t)dp;
}

int64_t m2l_tma_ctas(int level, int R) {
  int bx, by, bz;
  if (!m2l_tma_block(R, &bx, &by, &bz)) return 0;
  const int h = 1 << (level - 1), bxr = bx * R;
  return (int64_t)((h * R + bxr - 1) / bxr) * ((h + by - 1) / by) * ((h + bz - 1) / bz) * 8;
}

// Offset groups of the FP16 M2L: the fewest that fill one wave of the SMs
// (its per-offset drains need no extra chains for accuracy): with fewer
// tiles than SMs, double the groups until the SMs are covered (at most
// 16).  More groups at a level that already fills the SMs shorten the
// launch alone (256 tiles at the 1M-point leaf level: two waves, 939 us;
// four groups: seven quarter waves, 846 us + 34 us of partial sums) but
// lengthened the evaluate (1.95 -> 2.04 ms): the idle SMs of the second
// wave were running the near field.
int m2l_h16_groups(int64_t ctas, int nsm) {
  int g = 1;
  while (g < 16 && ctas * g < nsm) g *= 2;
  return g;
}

eifmm_status launch_m2l_h16(const M2LTcArgs& a0, const void* map0, const void* map1, const uint32_t* wmax,
                            const float* kscale, cudaStream_t s) {
  M2LTcArgs a = a0;
  if (!(a.dp == 64 || a.dp == 128 || a.dp == 192 || a.dp == 256) || !m2l_tma_block(a.R, &a.bx, &a.by, &a.bz)) {
    set_error("FP16 M2L: needs dp in {64, 128, 192, 256} and a tile shape for R");
    return EIFMM_EUNSUPPORTED;
  }
  a.h = 1 << (a.level - 1);
  const int bxr = a.bx * a.R;
  const int64_t tiles =
      (int64_t)((a.h * a.R + bxr - 1) / bxr) * ((a.h + a.by - 1) / a.by) * ((a.h + a.bz - 1) / a.bz);
  if (a.groups > 1) {
    a.out = a.part;
    a.part_stride = a.rows * (int64_t)a.dp;
  } else {
    a.out = a.g;
    a.part_stride = 0;
  }
  const size_t sm = m2l_h16_smem_bytes(a.dp);
  const int di = a.dp / 64 - 1;
  static bool attr[kMaxDevices][4] = {};
  const int dev = current_device();
  if (dev >= kMaxDevices || !attr[dev][di]) {
    cudaError_t e = cudaSuccess;
    switch (a.dp) {
      case 64: e = cudaFuncSetAttribute(k_m2l_h16<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024); break;
      case 128: e = cudaFuncSetAttribute(k_m2l_h16<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024); break;
      case 192: e = cudaFuncSetAttribute(k_m2l_h16<192>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024); break;
      default: e = cudaFuncSetAttribute(k_m2l_h16<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024); break;
    }
    EIFMM_CUDA(e);
    if (dev < kMaxDevices) attr[dev][di] = true;
  }
  const unsigned grid = (unsigned)(tiles * 8 * a.groups);
  const CUtensorMap& m0 = *(const CUtensorMap*)map0;
  const CUtensorMap& m1 = *(const CUtensorMap*)map1;
  switch (a.dp) {
    case 64: k_m2l_h16<64><<<grid, kH16Threads, sm, s>>>(m0, m1, a, wmax, kscale); break;
    case 128: k_m2l_h16<128><<<grid, kH16Threads, sm, s>>>(m0, m1, a, wmax, kscale); break;
    case 192: k_m2l_h16<192><<<grid, kH16Threads, sm, s>>>(m0, m1, a, wmax, kscale); break;
    default: k_m2l_h16<256><<<grid, kH16Threads, sm, s>>>(m0, m1, a, wmax, kscale); break;
  }
  EIFMM_CHECK_LAUNCH();
  if (a.groups > 1) {
    const int64_t n4 = a.rows * (int64_t)a.dp / 4;
    k_sum_parts<<<(unsigned)((n4 + 255) / 256 < 4096 ? (n4 + 255) / 256 : 4096), 256, 0, s>>>(
        (const float4*)a.part, a.groups, n4, a.part_stride / 4, (float4*)a.g);
    EIFMM_CHECK_LAUNCH();
  }
  return EIFMM_OK;
}

// Host plan of the stream-K M2L at `level` for R right-hand sides on nsm
// CTAs: the units of every tile (its active offsets: the candidate offsets
// of its parity class whose source block meets the class grid, the test the
// kernels make), the CTA ranges, and the split tiles with the slots of their
// partials in CTA order.  Uploaded once into device arrays owned by `p`.
eifmm_status build_sk_plan(int level, int R, int nsm, SkPlanDev* p) {
  int bx, by, bz;
  if (!m2l_t256_block(R, &bx, &by, &bz) || nsm < 1) return EIFMM_EUNSUPPORTED;
  const int h = 1 << (level - 1), bxr = bx * R;
  const int ntx = (h * R + bxr - 1) / bxr, nty = (h + by - 1) / by, ntz = (h + bz - 1) / bz;
  const int tpc = ntx * nty * ntz, ntiles = 8 * tpc;
  std::vector<int> tu(ntiles + 1, 0);
  for (int t = 0; t < ntiles; ++t) {
    const int oct = t / tpc;
    int tile = t % tpc;
    const int tx = tile % ntx;
    tile /= ntx;
    const int ty = tile % nty, tz = tile / nty;
    const int xr0 = tx * bxr, y0 = ty * by, z0 = tz * bz;
    const int cx = oct & 1, cy = (oct >> 1) & 1, cz = (oct >> 2) & 1;
    int n = 0;
    for (int slot = 0; slot < kNumSlots; ++slot) {
      const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
      // the candidate offsets of the class: the parent's neighbours' children
      // that are not neighbours of the box
      if (((cx + dx) >> 1) < -1 || ((cx + dx) >> 1) > 1 || ((cy + dy) >> 1) < -1 || ((cy + dy) >> 1) > 1 ||
          ((cz + dz) >> 1) < -1 || ((cz + dz) >> 1) > 1)
        continue;
      if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) < 2) continue;
      const int sxr = xr0 + ((cx + dx) >> 1) * R, sy = y0 + ((cy + dy) >> 1), sz = z0 + ((cz + dz) >> 1);
      if (sxr < h * R && sxr + bxr > 0 && sy < h && sy + by > 0 && sz < h && sz + bz > 0) ++n;
    }
    tu[t + 1] = tu[t] + n;
  }
  const int U = tu[ntiles];
  const int nctas = std::max(1, std::min(nsm, U));
  // pieces of every CTA; a tile is split unless one CTA covers it whole
  std::vector<std::vector<int>> slots(ntiles);
  std::vector<char> whole(ntiles, 0);
  for (int c = 0; c < nctas; ++c) {
    const int u0 = (int)((int64_t)c * U / nctas), u1 = (int)((int64_t)(c + 1) * U / nctas);
    int t_first = (int)(std::upper_bound(tu.begin(), tu.begin() + ntiles, u0) - tu.begin()) - 1;
    for (int t = t_first; t < ntiles && tu[t] < u1; ++t) {
      const int lo = std::max(u0, tu[t]) - tu[t], hi = std::min(u1, tu[t + 1]) - tu[t];
      if (hi <= lo) continue;
      if (lo == 0 && hi == tu[t + 1] - tu[t]) whole[t] = 1;
      else slots[t].push_back(2 * c + (t == t_first ? 0 : 1));
    }
  }
  std::vector<int> fix_t, fix_b(1, 0), fix_slot;
  for (int t = 0; t < ntiles; ++t) {
    if (whole[t]) continue;  // tiles without units have no pieces: g = 0 from the fix-up
    fix_t.push_back(t);
    for (int sl : slots[t]) fix_slot.push_back(sl);
    fix_b.push_back((int)fix_slot.size());
  }
  p->ntiles = ntiles;
  p->tpc = tpc;
  p->nctas = nctas;
  p->nfix = (int)fix_t.size();
  auto up = [](int** d, const std::vector<int>& v) -> eifmm_status {
    EIFMM_TRY(dalloc(d, v.size() > 0 ? v.size() : 1));
    if (!v.empty()) EIFMM_CUDA(cudaMemcpy(*d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice));
    return EIFMM_OK;
  };
  EIFMM_TRY(up(&p->tu, tu));
  EIFMM_TRY(up(&p->fix_t, fix_t));
  EIFMM_TRY(up(&p->fix_b, fix_b));
  EIFMM_TRY(up(&p->fix_slot, fix_slot));
  EIFMM_TRY(dalloc(&p->part, (size_t)2 * nctas * kT2Rows * 128));
  return EIFMM_OK;
}

void free_sk_plan(SkPlanDev* p) {
  dfree(p->tu);
  dfree(p->fix_t);
  dfree(p->fix_b);
  dfree(p->fix_slot);
  dfree(p->part);
  *p = SkPlanDev();
}

eifmm_status launch_m2l_t256s(const M2LTcArgs& a0, const void* map0, const void* map1, const SkPlanDev& p,
                              cudaStream_t s) {
  M2LTcArgs a = a0;
  if (a.dp != 128 || !m2l_t256_block(a.R, &a.bx, &a.by, &a.bz) || !p.tu) {
    set_error("stream-K M2L: needs dp = 128, a tile shape for R and a plan");
    return EIFMM_EUNSUPPORTED;
  }
  a.h = 1 << (a.level - 1);
  const size_t sm = m2l_t256_smem_bytes();
  static bool attr[kMaxDevices] = {};
  const int dev = current_device();
  if (dev >= kMaxDevices || !attr[dev]) {
    EIFMM_CUDA(cudaFuncSetAttribute(k_m2l_t256s<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    if (dev < kMaxDevices) attr[dev] = true;
  }
  SkPlan sk;
  sk.tu = p.tu;
  sk.ntiles = p.ntiles;
  sk.tpc = p.tpc;
  sk.nctas = p.nctas;
  sk.part = p.part;
  const CUtensorMap& m0 = *(const CUtensorMap*)map0;
  const CUtensorMap& m1 = *(const CUtensorMap*)map1;
  k_m2l_t256s<false><<<(unsigned)p.nctas, kT2Threads, sm, s>>>(m0, m1, a, sk);
  EIFMM_CHECK_LAUNCH();
  if (p.nfix > 0) {
    static_assert(kT2Rows == 32 * 8, "fix-up grid: 8 row groups of 32 rows");
    k_sk_fixup<<<dim3((unsigned)p.nfix, kT2Rows / 32), 256, 0, s>>>(a, sk, p.fix_t, p.fix_b, p.fix_slot);
    EIFMM_CHECK_LAUNCH();
  }
  return EIFMM_OK;
}

int64_t m2l_t256_ctas(int level, int R) {
  int bx, by, bz;
  if (!m2l_t256_block(R, &bx, &by, &bz)) return 0;
  const int h = 1 << (level - 1), bxr = bx * R;
  return (int64_t)((h * R + bxr - 1) / bxr) * ((h + by - 1) / by) * ((h + bz - 1) / bz) * 8;
}

eifmm_status launch_m2l_tc(const M2LTcArgs& a0, bool tf32, cudaStream_t s) {
  if (tf32) {  // the TF32 planes of an earlier tier are no longer built
    set_error("tensor-core M2L: TF32 operand planes are not built (BF16 and FP16 only)");
    return EIFMM_EUNSUPPORTED;
  }
  M2LTcArgs a = a0;
  a.stages = m2l_tc_stages(a.dp);
  a.chains = a.dp <= 128 ? 4 : (a.dp <= 256 ? 2 : 1);
  a.tmem_cols = 512;
  const size_t sm = m2l_tc_smem_bytes(a.dp, tf32);
  static bool attr[kMaxDevices][2] = {};
  const int dev = current_device();
  if (dev >= kMaxDevices || !attr[dev][tf32]) {
    EIFMM_CUDA(cudaFuncSetAttribute(k_m2l_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    if (dev < kMaxDevices) attr[dev][tf32] = true;
  }
  const int64_t tiles = (a.nbox / 8 * a.R + kRows - 1) / kRows;
  if (a.groups > 1) {
    a.out = a.part;
    a.part_stride = a.rows * (int64_t)a.dp;
  } else {
    a.out = a.g;
    a.part_stride = 0;
  }
  const unsigned grid = (unsigned)(tiles * 8 * a.groups);
  k_m2l_tc<false><<<grid, 160, sm, s>>>(a);
  EIFMM_CHECK_LAUNCH();
  if (a.groups > 1) {
    const int64_t n4 = a.rows * (int64_t)a.dp / 4;
    k_sum_parts<<<(unsigned)((n4 + 255) / 256 < 4096 ? (n4 + 255) / 256 : 4096), 256, 0, s>>>(
        (const float4*)a.part, a.groups, n4, a.part_stride / 4, (float4*)a.g);
    EIFMM_CHECK_LAUNCH();
  }
  return EIFMM_OK;
}

}  // namespace eifmm
