// tree.cu -- octree bin/sort of the points (Section 3.3: uniform 2^D-tree
// with kappa + 1 levels; leaves are the 8^kappa boxes of level kappa).
//
// Leaf coordinate floor((x - lo) * (2^kappa / L)) clamped to [0, 2^kappa - 1],
// Morton key with the x bit lowest, then a stable LSD radix sort of the keys
// (8-bit digits; a block ranks its tile warp by warp with __match_any_sync so
// that equal digits keep their input order), leaf offsets from the sorted
// keys and the gather of sorted FP64 coordinates plus FP32 coordinates
// relative to the leaf centre.
#include <mutex>

#include "internal.h"

namespace eifmm {
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 2048 keys per block

__global__ void k_keys(const double* __restrict__ xyz, int64_t n, double lo0,
                       double lo1, double lo2, double hi0, double hi1,
                       double hi2, double scale, int depth,
                       uint32_t* __restrict__ keys, int32_t* __restrict__ idx,
                       int* __restrict__ bad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double lo[3] = {lo0, lo1, lo2};
  const double hi[3] = {hi0, hi1, hi2};
  const int nmax = (1 << depth) - 1;
  int c[3];
  bool out = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double x = xyz[3 * i + a];
    if (!(x >= lo[a] && x <= hi[a])) out = true;
    // (x - lo) * scale: a subtraction then a product, never fused.  The
    // conversion truncates toward zero and clamps to the int range (NaN gives
    // 0); truncation equals floor wherever the clamp to [0, nmax] leaves the
    // value unchanged.
    const int v = __double2int_rz(__dmul_rn(__dsub_rn(x, lo[a]), scale));
    c[a] = min(max(v, 0), nmax);
  }
  if (out) atomicAdd(bad, 1);
  keys[i] = (uint32_t)morton_encode(c[0], c[1], c[2], depth);
  idx[i] = (int32_t)i;
}

__global__ void k_rs_count(const uint32_t* __restrict__ keys, int64_t n,
                           int shift, uint32_t* __restrict__ counts,
                           int nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
    const int64_t p = base + i;
    if (p < n) atomicAdd(&h[(keys[p] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of the digit-major counts (256 x nblocks entries) in two
// launches: per-tile totals, then each tile adds the totals of the tiles
// before it to its own block-wide scan.  A tile is SC_TILE consecutive
// entries, SC_ITEMS per thread.
constexpr int SC_THREADS = 1024;
constexpr int SC_ITEMS = 4;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

inline int64_t scan_tiles(int64_t len) { return (len + SC_TILE - 1) / SC_TILE; }

// Exclusive scan of one value per thread over a block of SC_THREADS threads;
// *total receives the block's sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t ws[SC_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();  // ws may still be read by a previous call
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t u = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, u, o);
      if (lane >= o) u += y;
    }
    ws[lane] = u;
  }
  __syncthreads();
  *total = ws[SC_THREADS / 32 - 1];
  return x - v + (w > 0 ? ws[w - 1] : 0u);
}

__global__ void __launch_bounds__(SC_THREADS)
k_scan_totals(const uint32_t* __restrict__ a, int64_t len, uint32_t* __restrict__ part) {
  const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j)
    if (base + j < len) s += a[base + j];
  uint32_t total;
  block_excl_scan(s, &total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SC_THREADS)
k_scan_apply(uint32_t* __restrict__ a, int64_t len, const uint32_t* __restrict__ part) {
  uint32_t pre = 0;
  for (int j = threadIdx.x; j < (int)blockIdx.x; j += SC_THREADS) pre += part[j];
  uint32_t before;
  block_excl_scan(pre, &before);
  const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
  uint32_t v[SC_ITEMS], s = 0;
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    v[j] = base + j < len ? a[base + j] : 0u;
    s += v[j];
  }
  uint32_t total;
  uint32_t run = before + block_excl_scan(s, &total);
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    if (base + j < len) a[base + j] = run;
    run += v[j];
  }
}

void launch_scan(uint32_t* counts, int64_t len, uint32_t* part, cudaStream_t s) {
  const unsigned nt = (unsigned)scan_tiles(len);
  k_scan_totals<<<nt, SC_THREADS, 0, s>>>(counts, len, part);
  k_scan_apply<<<nt, SC_THREADS, 0, s>>>(counts, len, part);
}

__global__ void __launch_bounds__(RS_THREADS)
k_rs_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
             uint32_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t n,
             int shift, const uint32_t* __restrict__ offsets, int nblocks) {
  __shared__ uint32_t wc[RS_WARPS][257];
  for (int i = threadIdx.x; i < RS_WARPS * 257; i += RS_THREADS) (&wc[0][0])[i] = 0;
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * (32 * RS_ITEMS);
  uint32_t kk[RS_ITEMS];
  int32_t vv[RS_ITEMS];
  uint32_t rank[RS_ITEMS];
  int dig[RS_ITEMS];
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    const int64_t p = wbase + j * 32 + lane;
    const bool valid = p < n;
    kk[j] = valid ? kin[p] : 0u;
    vv[j] = valid ? vin[p] : 0;
    const int d = valid ? (int)((kk[j] >> shift) & 255u) : 256;
    dig[j] = d;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t old = wc[w][d];
    __syncwarp();
    if (lane == __ffs(peers) - 1) wc[w][d] = old + __popc(peers);
    __syncwarp();
    rank[j] = old + __popc(peers & lt);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
    uint32_t run = 0;
    for (int ww = 0; ww < RS_WARPS; ++ww) {
      const uint32_t t = wc[ww][d];
      wc[ww][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    if (dig[j] == 256) continue;
    const uint32_t pos = offsets[(int64_t)dig[j] * nblocks + blockIdx.x] + wc[w][dig[j]] + rank[j];
    kout[pos] = kk[j];
    vout[pos] = vv[j];
  }
}

// off[b] = first sorted position whose key is at least b (b = 0..nleaf;
// off[nleaf] = n): one thread per leaf, a binary search over the sorted
// keys, so runs of empty leaves cost no more than full ones.
__global__ void k_leaf_off(const uint32_t* __restrict__ skeys, int64_t n,
                           int64_t nleaf, int32_t* __restrict__ off) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b > nleaf) return;
  int64_t lo = 0, hi = n;  // the answer lies in [lo, hi]
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)__ldg(skeys + mid) < b) lo = mid + 1;
    else hi = mid;
  }
  off[b] = (int32_t)lo;
}

// Leaf-centre coordinates lo_a + (2 c + 1) l_kappa of the 2^depth cells
// per axis are formed once per block in shared memory ([3][2^depth]).
__global__ void k_gather_points(const double* __restrict__ xyz,
                                const int32_t* __restrict__ perm,
                                const uint32_t* __restrict__ skeys, int64_t n,
                                double lo0, double lo1, double lo2, double lk,
                                int depth, double* __restrict__ x,
                                double* __restrict__ y, double* __restrict__ z,
                                float* __restrict__ lx, float* __restrict__ ly,
                                float* __restrict__ lz) {
  extern __shared__ double s_ctr[];
  const int nc = 1 << depth;
  for (int t = threadIdx.x; t < 3 * nc; t += blockDim.x) {
    const int a = t >> depth, c = t & (nc - 1);
    const double lo = a == 0 ? lo0 : (a == 1 ? lo1 : lo2);
    s_ctr[t] = lo + (2.0 * c + 1.0) * lk;
  }
  __syncthreads();
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int64_t i = perm[p];
  const double px = xyz[3 * i], py = xyz[3 * i + 1], pz = xyz[3 * i + 2];
  int c[3];
  morton_decode(skeys[p], depth, c);
  x[p] = px;
  y[p] = py;
  z[p] = pz;
  lx[p] = (float)(px - s_ctr[c[0]]);
  ly[p] = (float)(py - s_ctr[nc + c[1]]);
  lz[p] = (float)(pz - s_ctr[2 * nc + c[2]]);
}

__global__ void k_nonempty(const int32_t* __restrict__ off, int64_t nleaf,
                           int32_t* __restrict__ list, int32_t* __restrict__ cnt) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nleaf) return;
  if (off[b + 1] > off[b]) list[atomicAdd(cnt, 1)] = (int32_t)b;
}

struct SortScratch {
  std::mutex m;
  unsigned char* p = nullptr;
  size_t cap = 0;
};
SortScratch& sort_scratch(int dev) {
  static SortScratch s[64];
  return s[dev & 63];
}

}  // namespace

eifmm_status build_pointset(const double* xyz, int64_t n, const double lo[3],
                            double L, int depth, cudaStream_t s, PointSet* ps) {
  ps->n = n;
  const int64_t nleaf = (int64_t)1 << (3 * depth);
  const int64_t nn = n > 0 ? n : 1;
  // one slab for the point set, one for the sort's scratch (256-byte aligned parts)
  auto take = [](size_t& off, size_t bytes) { const size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
  size_t off = 0;
  const size_t o_perm = take(off, nn * 4), o_keys = take(off, nn * 4), o_loff = take(off, (nleaf + 1) * 4),
               o_ne = take(off, nleaf * 4), o_x = take(off, nn * 8), o_y = take(off, nn * 8),
               o_z = take(off, nn * 8), o_lx = take(off, nn * 4), o_ly = take(off, nn * 4),
               o_lz = take(off, nn * 4);
  unsigned char* slab = nullptr;
  EIFMM_TRY(dalloc(&slab, off));
  ps->slab = slab;
  ps->perm = (int32_t*)(slab + o_perm);
  ps->keys = (uint32_t*)(slab + o_keys);
  ps->leaf_off = (int32_t*)(slab + o_loff);
  ps->nonempty = (int32_t*)(slab + o_ne);
  ps->x = (double*)(slab + o_x);
  ps->y = (double*)(slab + o_y);
  ps->z = (double*)(slab + o_z);
  ps->lx = (float*)(slab + o_lx);
  ps->ly = (float*)(slab + o_ly);
  ps->lz = (float*)(slab + o_lz);

  const int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
  const int nb1 = nblocks > 0 ? nblocks : 1;
  size_t soff = 0;
  const size_t o_k2 = take(soff, nn * 4), o_v2 = take(soff, nn * 4), o_cnt = take(soff, (size_t)256 * nb1 * 4),
               o_part = take(soff, scan_tiles((int64_t)256 * nb1) * 4), o_bad = take(soff, 2 * sizeof(int));
  // The sort's scratch is kept per device between builds (grown on demand,
  // held until the process exits); builds on one device take turns on it.
  int dev = 0;
  EIFMM_CUDA(cudaGetDevice(&dev));
  SortScratch& sc = sort_scratch(dev);
  std::unique_lock<std::mutex> hold(sc.m);
  if (sc.cap < soff) {
    dfree(sc.p);
    sc.p = nullptr;
    sc.cap = 0;
    EIFMM_TRY(dalloc(&sc.p, soff));
    sc.cap = soff;
  }
  unsigned char* scratch = sc.p;
  uint32_t* k2 = (uint32_t*)(scratch + o_k2);
  int32_t* v2 = (int32_t*)(scratch + o_v2);
  uint32_t* counts = (uint32_t*)(scratch + o_cnt);
  uint32_t* parts = (uint32_t*)(scratch + o_part);
  int* dbad = (int*)(scratch + o_bad);
  EIFMM_CUDA(cudaMemsetAsync(dbad, 0, 2 * sizeof(int), s));

  const double scale = ldexp(1.0, depth) / L;
  if (n > 0) {
    k_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        xyz, n, lo[0], lo[1], lo[2], lo[0] + L, lo[1] + L, lo[2] + L, scale,
        depth, ps->keys, ps->perm, dbad);
    EIFMM_CHECK_LAUNCH();
    uint32_t* kin = ps->keys;
    int32_t* vin = ps->perm;
    uint32_t* kout = k2;
    int32_t* vout = v2;
    const int bits = 3 * depth;
    for (int shift = 0; shift < bits; shift += 8) {
      k_rs_count<<<nblocks, RS_THREADS, 0, s>>>(kin, n, shift, counts, nblocks);
      EIFMM_CHECK_LAUNCH();
      launch_scan(counts, (int64_t)256 * nblocks, parts, s);
      EIFMM_CHECK_LAUNCH();
      k_rs_scatter<<<nblocks, RS_THREADS, 0, s>>>(kin, vin, kout, vout, n, shift,
                                                   counts, nblocks);
      EIFMM_CHECK_LAUNCH();
      uint32_t* tk = kin; kin = kout; kout = tk;
      int32_t* tv = vin; vin = vout; vout = tv;
    }
    if (kin != ps->keys) {
      EIFMM_CUDA(cudaMemcpyAsync(ps->keys, kin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
      EIFMM_CUDA(cudaMemcpyAsync(ps->perm, vin, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
  }
  k_leaf_off<<<(unsigned)((nleaf + 1 + 255) / 256), 256, 0, s>>>(ps->keys, n, nleaf, ps->leaf_off);
  EIFMM_CHECK_LAUNCH();
  if (n > 0) {
    const double lk = L * ldexp(1.0, -(depth + 1));
    k_gather_points<<<(unsigned)((n + 255) / 256), 256, (size_t)3 * sizeof(double) << depth, s>>>(
        xyz, ps->perm, ps->keys, n, lo[0], lo[1], lo[2], lk, depth, ps->x, ps->y,
        ps->z, ps->lx, ps->ly, ps->lz);
    EIFMM_CHECK_LAUNCH();
  }
  k_nonempty<<<(unsigned)((nleaf + 255) / 256), 256, 0, s>>>(ps->leaf_off, nleaf, ps->nonempty, dbad + 1);
  EIFMM_CHECK_LAUNCH();
  int hb[2] = {0, 0};
  EIFMM_CUDA(cudaMemcpyAsync(hb, dbad, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  EIFMM_CUDA(cudaStreamSynchronize(s));
  ps->n_nonempty = hb[1];
  if (hb[0] != 0) {
    set_error("eifmm_tree_build: " + std::to_string(hb[0]) +
              " coordinates lie outside the cube [lo, lo + L]^3");
    return EIFMM_EINVAL;
  }
  return EIFMM_OK;
}

void free_pointset(PointSet* ps) {
  dfree(ps->slab);
  *ps = PointSet();
}

}  // namespace eifmm

// ---------------------------------------------------------------------------
// Allocation-free variant of the bin/sort (eifmm_tree_sort_static).  Its
// radix-sort scratch lives in a file-scope device array: keys and indices of
// the other half of the ping-pong (4 + 4 bytes per point), the per-block
// digit counts (256 x 4 bytes per 2048 points) and an error counter.
// ---------------------------------------------------------------------------
namespace eifmm {
namespace {
constexpr int64_t kStaticMax = EIFMM_STATIC_SORT_MAX_POINTS;
constexpr int64_t kStaticBlocks = (kStaticMax + RS_TILE - 1) / RS_TILE;
constexpr size_t kOffKeys = 0;
constexpr size_t kOffVals = kOffKeys + (size_t)kStaticMax * 4;
constexpr size_t kOffCounts = kOffVals + (size_t)kStaticMax * 4;
constexpr size_t kOffParts = kOffCounts + (size_t)256 * kStaticBlocks * 4;
constexpr size_t kOffBad = kOffParts + (((size_t)256 * kStaticBlocks + SC_TILE - 1) / SC_TILE) * 4 + 16;
constexpr size_t kStaticBytes = kOffBad + 256;
static_assert(kStaticBytes == EIFMM_STATIC_SORT_SCRATCH_BYTES, "scratch size of the header");

__device__ __align__(256) unsigned char g_sort_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch on the current device, looked up once per
// device (the host-side symbol is only a stand-in, never a device address).
eifmm_status static_scratch(unsigned char** out) {
  int dev = 0;
  EIFMM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("eifmm_tree_sort_static: device ordinal out of range");
    return EIFMM_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error(std::string("eifmm_tree_sort_static: cudaGetSymbolAddress failed: ") +
                cudaGetErrorString(e));
      return EIFMM_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return EIFMM_OK;
}
}  // namespace
}  // namespace eifmm

using namespace eifmm;

extern "C" eifmm_status eifmm_tree_sort_static(const double* xyz, int64_t n, const double lo[3],
                                               double L, int depth, uint32_t* keys_out,
                                               int32_t* perm_out, int32_t* leaf_off_out,
                                               eifmm_stream stream) {
  if (!lo || !leaf_off_out || n < 0 || (n > 0 && (!xyz || !keys_out || !perm_out)) || depth < 2 ||
      depth > kMaxLevel || !(L > 0.0)) {
    set_error("eifmm_tree_sort_static: invalid argument");
    return EIFMM_EINVAL;
  }
  if (n > kStaticMax) {
    set_error("eifmm_tree_sort_static: n = " + std::to_string(n) + " exceeds the static scratch limit of " +
              std::to_string(kStaticMax) + " points (EIFMM_STATIC_SORT_MAX_POINTS)");
    return EIFMM_EINVAL;
  }
  unsigned char* base = nullptr;
  EIFMM_TRY(static_scratch(&base));
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* k2 = (uint32_t*)(base + kOffKeys);
  int32_t* v2 = (int32_t*)(base + kOffVals);
  uint32_t* counts = (uint32_t*)(base + kOffCounts);
  uint32_t* parts = (uint32_t*)(base + kOffParts);
  int* bad = (int*)(base + kOffBad);
  // the error counter must start at zero on every call
  EIFMM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  const int64_t nleaf = (int64_t)1 << (3 * depth);
  const int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
  if (n > 0) {
    k_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xyz, n, lo[0], lo[1], lo[2], lo[0] + L, lo[1] + L,
                                                        lo[2] + L, ldexp(1.0, depth) / L, depth, keys_out,
                                                        perm_out, bad);
    EIFMM_CHECK_LAUNCH();
    uint32_t* kin = keys_out;
    int32_t* vin = perm_out;
    uint32_t* kout = k2;
    int32_t* vout = v2;
    for (int shift = 0; shift < 3 * depth; shift += 8) {
      k_rs_count<<<nblocks, RS_THREADS, 0, s>>>(kin, n, shift, counts, nblocks);
      EIFMM_CHECK_LAUNCH();
      launch_scan(counts, (int64_t)256 * nblocks, parts, s);
      EIFMM_CHECK_LAUNCH();
      k_rs_scatter<<<nblocks, RS_THREADS, 0, s>>>(kin, vin, kout, vout, n, shift, counts, nblocks);
      EIFMM_CHECK_LAUNCH();
      uint32_t* tk = kin; kin = kout; kout = tk;
      int32_t* tv = vin; vin = vout; vout = tv;
    }
    if (kin != keys_out) {
      EIFMM_CUDA(cudaMemcpyAsync(keys_out, kin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
      EIFMM_CUDA(cudaMemcpyAsync(perm_out, vin, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
  }
  k_leaf_off<<<(unsigned)((nleaf + 1 + 255) / 256), 256, 0, s>>>(keys_out, n, nleaf, leaf_off_out);
  EIFMM_CHECK_LAUNCH();
  int hbad = 0;
  EIFMM_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  EIFMM_CUDA(cudaStreamSynchronize(s));
  if (hbad != 0) {
    set_error("eifmm_tree_sort_static: " + std::to_string(hbad) +
              " coordinates lie outside the cube [lo, lo + L]^3");
    return EIFMM_EINVAL;
  }
  return EIFMM_OK;
}
