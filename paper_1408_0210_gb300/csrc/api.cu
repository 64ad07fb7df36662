// api.cu -- the C ABI (include/eifmm.h): handles, validation, workspaces and
// the dispatch of the evaluation paths.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <mutex>
#include <set>
#include <vector>

#include "internal.h"
#include "solve.cuh"

namespace eifmm {

static std::atomic<uint64_t> g_launches{0};
static std::atomic<uint64_t> g_ops_uid{0};
// ids of the operator sets not yet destroyed
static std::mutex g_live_mu;
static std::set<uint64_t> g_live_ops;
static bool ops_alive(uint64_t uid) {
  std::lock_guard<std::mutex> lock(g_live_mu);
  return g_live_ops.count(uid) != 0;
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static thread_local std::string g_err;
static bool g_timing = false;

void set_error(const std::string& msg) { g_err = msg; }
bool timing_enabled() { return g_timing; }

eifmm_status dmalloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    set_error("device allocation of " + std::to_string(bytes) + " bytes failed: " +
              cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? EIFMM_ENOMEM : EIFMM_ECUDA;
  }
  return EIFMM_OK;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

void free_workspace(Workspace* ws) {
  for (int k = 0; k <= kMaxLevel; ++k) {
    dfree(ws->W[k]); dfree(ws->Wh[k]); dfree(ws->g[k]);
    if (k != 2) dfree(ws->l[k]);
    ws->l[k] = nullptr;
    dfree(ws->W32[k]); dfree(ws->Wh32[k]); dfree(ws->g32[k]); dfree(ws->wa[k]);
    if (k != 2) dfree(ws->l32[k]);
    ws->W[k] = ws->Wh[k] = ws->g[k] = nullptr;
    ws->W32[k] = ws->Wh32[k] = ws->g32[k] = ws->l32[k] = nullptr;
    ws->wa[k] = nullptr;
  }
  dfree(ws->lh); dfree(ws->lh32); dfree(ws->sig); dfree(ws->sig32); dfree(ws->m2l_part);
  ws->m2l_part = nullptr;
  ws->m2l_part_cap = 0;
  dfree(ws->m2l_part_leaf);
  ws->m2l_part_leaf = nullptr;
  ws->m2l_part_leaf_cap = 0;
  dfree(ws->part64);
  ws->part64 = nullptr;
  ws->part64_cap = 0;
  dfree(ws->blas_ws);
  ws->blas_ws = nullptr;
  for (int k = 0; k <= kMaxLevel; ++k) ws->m2l_kind[k] = ws->m2l_gshift[k] = 0;
  ws->p2p_sym = 0;
  free_sk_plan(&ws->sk);
  dfree(ws->fnear); dfree(ws->ffar); dfree(ws->tmp); dfree(ws->gsym); dfree(ws->wmax);
  ws->gsym = nullptr;
  ws->wmax = nullptr;
  ws->tmp = nullptr;
  ws->lh = nullptr; ws->lh32 = nullptr; ws->sig = nullptr; ws->sig32 = nullptr;
  ws->fnear = nullptr; ws->ffar = nullptr;
  ws->ops_id = nullptr;
  ws->ops_uid = 0;
  ws->nrhs = 0;
  ws->prec = -1;
  ws->tier = -1;
  ws->evaluated = false;
}

static void free_streams(Workspace* ws) {
  if (ws->side) cudaStreamDestroy(ws->side);
  if (ws->ev_fork) cudaEventDestroy(ws->ev_fork);
  if (ws->ev_join) cudaEventDestroy(ws->ev_join);
  if (ws->side2) cudaStreamDestroy(ws->side2);
  if (ws->hi) cudaStreamDestroy(ws->hi);
  if (ws->ev_hi) cudaEventDestroy(ws->ev_hi);
  ws->hi = nullptr;
  ws->ev_hi = nullptr;
  if (ws->ev_fork2) cudaEventDestroy(ws->ev_fork2);
  if (ws->ev_join2) cudaEventDestroy(ws->ev_join2);
  for (auto& e : ws->ev_m2le)
    if (e) cudaEventDestroy(e);
  for (auto& e : ws->ev_t)
    if (e) cudaEventDestroy(e);
  for (auto& e : ws->ev_nf)
    if (e) cudaEventDestroy(e);
  for (auto& e : ws->ev_m2l)
    if (e) cudaEventDestroy(e);
  ws->side = nullptr;
  ws->ev_fork = ws->ev_join = nullptr;
  ws->side2 = nullptr;
  ws->ev_fork2 = ws->ev_join2 = nullptr;
  for (auto& e : ws->ev_m2le) e = nullptr;
  for (auto& e : ws->ev_t) e = nullptr;
  for (auto& e : ws->ev_m2l) e = nullptr;
  for (auto& e : ws->ev_nf) e = nullptr;
  dfree(ws->host_sig);
  dfree(ws->host_f);
  ws->host_sig = ws->host_f = nullptr;
  ws->host_cap = 0;
  dfree(ws->err);
  if (ws->err_host) cudaFreeHost(ws->err_host);
  ws->err = nullptr;
  ws->err_host = nullptr;
}

eifmm_status alloc_mixed_workspace(Tree* t, const Ops* ops, int R);  // fmm32.cu

eifmm_status ensure_workspace(Tree* t, const Ops* ops, int R, int prec) {
  Workspace& ws = t->ws;
  if (!ws.side) {
    EIFMM_CUDA(cudaStreamCreateWithFlags(&ws.side, cudaStreamNonBlocking));
    EIFMM_CUDA(cudaEventCreateWithFlags(&ws.ev_fork, cudaEventDisableTiming));
    EIFMM_CUDA(cudaEventCreateWithFlags(&ws.ev_join, cudaEventDisableTiming));
    int prio_lo = 0, prio_hi = 0;
    EIFMM_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    EIFMM_CUDA(cudaStreamCreateWithPriority(&ws.side2, cudaStreamNonBlocking, prio_hi));
    EIFMM_CUDA(cudaStreamCreateWithPriority(&ws.hi, cudaStreamNonBlocking, prio_hi));
    EIFMM_CUDA(cudaEventCreateWithFlags(&ws.ev_hi, cudaEventDisableTiming));
    EIFMM_CUDA(cudaEventCreateWithFlags(&ws.ev_fork2, cudaEventDisableTiming));
    EIFMM_CUDA(cudaEventCreateWithFlags(&ws.ev_join2, cudaEventDisableTiming));
    for (auto& e : ws.ev_m2le) EIFMM_CUDA(cudaEventCreate(&e));
    for (auto& e : ws.ev_t) EIFMM_CUDA(cudaEventCreate(&e));
    for (auto& e : ws.ev_m2l) EIFMM_CUDA(cudaEventCreate(&e));
    for (auto& e : ws.ev_nf) EIFMM_CUDA(cudaEventCreate(&e));
  }
  const int tier = (prec == EIFMM_PREC_MIXED) ? ops->tier : -1;
  if (ws.ops_id == (const void*)ops && ws.ops_uid == ops->uid && ws.nrhs == R &&
      ws.prec == prec && ws.tier == tier)
    return EIFMM_OK;
  free_workspace(&ws);
  const int kap = t->depth;
  const bool fp64_far = (prec == EIFMM_PREC_FP64) || tier >= 3;
  if (fp64_far) {
    for (int k = 2; k <= kap; ++k) {
      const size_t n = ((size_t)1 << (3 * k)) * R * ops->lv[k].d;
      EIFMM_TRY(dalloc(&ws.W[k], n));
      EIFMM_TRY(dalloc(&ws.Wh[k], n));
      EIFMM_TRY(dalloc(&ws.g[k], n));
      if (k == 2) ws.l[k] = ws.g[k];
      else EIFMM_TRY(dalloc(&ws.l[k], n));
    }
    EIFMM_TRY(dalloc(&ws.lh, ((size_t)1 << (3 * kap)) * R * ops->lv[kap].d));
    // partial sums of the offset groups of the coarse levels' M2L
    int dev = 0;
    EIFMM_CUDA(cudaGetDevice(&dev));
    EIFMM_CUDA(cudaDeviceGetAttribute(&ws.nsm, cudaDevAttrMultiProcessorCount, dev));
    size_t need = 0;
    for (int k = 2; k <= kap; ++k) {
      const int d = ops->lv[k].d;
      const int G = std::max(m2l64_groups(m2l64_blocks(k, R), ws.nsm), m2l64_groups(m2l_df_blocks(k, d, R), ws.nsm));
      if (G > 1) need = std::max(need, (size_t)G * ((size_t)1 << (3 * k)) * R * d);
    }
    if (need) EIFMM_TRY(dalloc(&ws.part64, need));
    ws.part64_cap = need;
  } else {
    EIFMM_TRY(alloc_mixed_workspace(t, ops, R));
  }
  {
    int dpmax = 0;
    for (int k = 2; k <= kap; ++k) dpmax = ops->lv[k].dp > dpmax ? ops->lv[k].dp : dpmax;
    EIFMM_TRY(dmalloc(&ws.tmp, ((size_t)1 << (3 * kap)) * R * dpmax * sizeof(double)));
  }
  EIFMM_TRY(dalloc(&ws.sig, (size_t)(t->src.n > 0 ? t->src.n : 1) * R));
  EIFMM_TRY(dalloc(&ws.sig32, (size_t)(t->src.n > 0 ? t->src.n : 1) * R));
  EIFMM_TRY(dalloc(&ws.fnear, (size_t)(t->tgt.n > 0 ? t->tgt.n : 1) * R));
  EIFMM_TRY(dalloc(&ws.ffar, (size_t)(t->tgt.n > 0 ? t->tgt.n : 1) * R));
  ws.ops_id = ops;
  ws.ops_uid = ops->uid;
  ws.nrhs = R;
  ws.prec = prec;
  ws.tier = tier;
  return EIFMM_OK;
}

}  // namespace eifmm

using namespace eifmm;

struct eifmm_ops {
  Ops o;
};
struct eifmm_tree {
  Tree t;
};

extern "C" const char* eifmm_last_error(void) { return g_err.c_str(); }
extern "C" const char* eifmm_version(void) { return "eifmm-gb300 0.1 (sm_103a)"; }
extern "C" void eifmm_set_timing(int on) { g_timing = on != 0; }
extern "C" uint64_t eifmm_kernel_launches(void) { return g_launches.load(); }

namespace eifmm {
eifmm_status launch_direct_sum(int kern, const double* tgt, const double* src, int64_t n_src,
                               const double* sigma, int64_t ld, int R, int exclude_self,
                               const int64_t* idx, int64_t n_eval, double* f, cudaStream_t s);
}

extern "C" eifmm_status eifmm_direct_sum(eifmm_kernel kern, const double* tgt_xyz, int64_t n_tgt,
                                         const double* src_xyz, int64_t n_src, const double* sigma,
                                         int64_t ld_sigma, int n_rhs, int exclude_self,
                                         const int64_t* tgt_idx, int64_t n_eval, double* f,
                                         eifmm_stream stream) {
  if (!tgt_xyz || !src_xyz || !sigma || !f || n_tgt < 1 || n_src < 1 || n_eval < 1 ||
      n_rhs < 1 || n_rhs > kMaxRhs || ld_sigma < n_src || (int)kern < 0 || (int)kern > 6 ||
      (!tgt_idx && n_eval > n_tgt)) {
    set_error("eifmm_direct_sum: invalid argument");
    return EIFMM_EINVAL;
  }
  return launch_direct_sum((int)kern, tgt_xyz, src_xyz, n_src, sigma, ld_sigma, n_rhs,
                           exclude_self, tgt_idx, n_eval, f, (cudaStream_t)stream);
}

// Arithmetic tier of the mixed path from the EIM tolerance: the requested
// tolerance when the operators were built here, otherwise the largest
// built-in estimate of the levels (which the greedy keeps just below the
// tolerance, hence the factor 1/3 in the thresholds).
static int tier_for_eps(double eps, bool requested) {
  const double f = requested ? 1.0 - 1e-9 : 1.0 / 3.0;
  if (eps >= 1e-5 * f) return 0;
  if (eps >= 1e-6 * f) return 1;
  return 3;
}

extern "C" eifmm_status eifmm_ops_load(eifmm_kernel kern, double L, int depth,
                                       const eifmm_level_data* levels, eifmm_ops** out) {
  if (!out || !levels || depth < 2 || depth > kMaxLevel || !(L > 0.0) || (int)kern < 0 ||
      (int)kern > 6) {
    set_error("eifmm_ops_load: invalid kernel, L, depth or null pointer");
    return EIFMM_EINVAL;
  }
  *out = nullptr;
  for (int k = 2; k <= depth; ++k) {
    const eifmm_level_data& e = levels[k];
    if (e.d < 1 || e.d > kMaxD || !e.X || !e.Y || !e.Gamma || !e.B) {
      set_error("eifmm_ops_load: level " + std::to_string(k) + " has d outside [1, 512] or null arrays");
      return EIFMM_EINVAL;
    }
    for (int i = 0; i < e.d; ++i)
      if (e.Gamma[(int64_t)i * e.d + i] == 0.0) {
        set_error("eifmm_ops_load: level " + std::to_string(k) + " has a zero pivot in Gamma");
        return EIFMM_EINVAL;
      }
  }
  eifmm_ops* h = new eifmm_ops();
  Ops& o = h->o;
  o.kern = kern;
  o.L = L;
  o.depth = depth;
  o.uid = g_ops_uid.fetch_add(1, std::memory_order_relaxed) + 1;
  double eps_max = 0.0;
  cudaStream_t s = nullptr;
  eifmm_status rc = EIFMM_OK;
  for (int k = 2; k <= depth && rc == EIFMM_OK; ++k) {
    const eifmm_level_data& e = levels[k];
    LevelOps& v = o.lv[k];
    v.d = e.d;
    v.dp = (e.d + 63) / 64 * 64;
    v.eps_est = e.eps_est;
    if (e.eps_est > eps_max) eps_max = e.eps_est;
    if ((rc = dalloc(&v.X, 3 * e.d)) != EIFMM_OK) break;
    if ((rc = dalloc(&v.Y, 3 * e.d)) != EIFMM_OK) break;
    if ((rc = dalloc(&v.G_rm, (size_t)e.d * e.d)) != EIFMM_OK) break;
    if ((rc = dalloc(&v.B_rm, (size_t)e.d * e.d)) != EIFMM_OK) break;
    const size_t dd = (size_t)e.d * e.d * sizeof(double);
    if (cudaMemcpy(v.X, e.X, 3 * e.d * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(v.Y, e.Y, 3 * e.d * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(v.G_rm, e.Gamma, dd, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(v.B_rm, e.B, dd, cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("eifmm_ops_load: upload failed");
      rc = EIFMM_ECUDA;
    }
  }
  if (rc == EIFMM_OK) rc = assemble_ops(&o, s);
  if (rc != EIFMM_OK) {
    free_ops(&o);
    delete h;
    return rc;
  }
  o.tier = tier_for_eps(eps_max > 0.0 ? eps_max : 1e-16, false);
  if (o.tier <= 1) rc = build_kd_image(&o, o.tier == 1 ? kPlaneF16 : kPlaneBF16, s);
  else if (o.tier == 2) rc = build_kd32(&o, s);
  if (rc != EIFMM_OK) {
    free_ops(&o);
    delete h;
    return rc;
  }
  {
    std::lock_guard<std::mutex> lock(g_live_mu);
    g_live_ops.insert(o.uid);
  }
  *out = h;
  return EIFMM_OK;
}

extern "C" eifmm_status eifmm_ops_build(eifmm_kernel kern, double L, int depth, double eps,
                                        int d_max, eifmm_stream stream, eifmm_ops** out) {
  if (!out || depth < 2 || depth > kMaxLevel || !(L > 0.0) || !(eps > 0.0) || d_max < 1 ||
      d_max > kMaxD) {
    set_error("eifmm_ops_build: invalid argument");
    return EIFMM_EINVAL;
  }
  std::vector<eifmm_level_data> lv(depth + 1);
  std::vector<std::vector<double>> keep;
  for (int k = 2; k <= depth; ++k) {
    int64_t nx = 0, ny = 0;
    EIFMM_TRY(eifmm_training_sets(k, L, 9, nullptr, &nx, nullptr, &ny));
    std::vector<double> X(3 * nx), Y(3 * ny);
    EIFMM_TRY(eifmm_training_sets(k, L, 9, X.data(), &nx, Y.data(), &ny));
    std::vector<int64_t> ia(d_max), ib(d_max);
    std::vector<double> G((size_t)d_max * d_max), B((size_t)d_max * d_max), piv(d_max + 1);
    int d = 0;
    double est = 0;
    EIFMM_TRY(eifmm_eim_build(kern, X.data(), nx, Y.data(), ny, eps, d_max, &d, ia.data(),
                              ib.data(), G.data(), B.data(), piv.data(), &est, stream));
    if (d < 1) {
      set_error("eifmm_ops_build: the EIM selected no point at level " + std::to_string(k));
      return EIFMM_EINVAL;
    }
    std::vector<double> px(3 * d), py(3 * d), pg((size_t)d * d), pb((size_t)d * d);
    for (int m = 0; m < d; ++m)
      for (int a = 0; a < 3; ++a) {
        px[3 * m + a] = X[3 * ia[m] + a];
        py[3 * m + a] = Y[3 * ib[m] + a];
      }
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        pg[(size_t)i * d + j] = G[(size_t)i * d_max + j];
        pb[(size_t)i * d + j] = B[(size_t)i * d_max + j];
      }
    keep.push_back(std::move(px));
    keep.push_back(std::move(py));
    keep.push_back(std::move(pg));
    keep.push_back(std::move(pb));
    const size_t b0 = keep.size() - 4;
    lv[k] = eifmm_level_data{d, keep[b0].data(), keep[b0 + 1].data(), keep[b0 + 2].data(),
                             keep[b0 + 3].data(), est};
  }
  EIFMM_TRY(eifmm_ops_load(kern, L, depth, lv.data(), out));
  eifmm_status rc = eifmm_ops_calibrate(*out, eps, stream, nullptr);
  if (rc != EIFMM_OK) {
    eifmm_ops_destroy(*out);
    *out = nullptr;
  }
  return rc;
}

extern "C" eifmm_status eifmm_ops_error_estimate(const eifmm_ops* ops, int level, double* eps_k,
                                                 int* d_k) {
  if (!ops || level < 2 || level > ops->o.depth) {
    set_error("eifmm_ops_error_estimate: invalid handle or level");
    return EIFMM_EINVAL;
  }
  if (eps_k) *eps_k = ops->o.lv[level].eps_est;
  if (d_k) *d_k = ops->o.lv[level].d;
  return EIFMM_OK;
}

extern "C" eifmm_status eifmm_ops_plan(eifmm_ops* ops, int tier_override, int* tier) {
  if (!ops || tier_override > 4) {
    set_error("eifmm_ops_plan: invalid handle or tier");
    return EIFMM_EINVAL;
  }
  if (tier_override >= 0) {
    ops->o.tier = tier_override;
    if (tier_override <= 1) EIFMM_TRY(build_kd_image(&ops->o, tier_override == 1 ? kPlaneF16 : kPlaneBF16, nullptr));
    else if (tier_override == 2) EIFMM_TRY(build_kd32(&ops->o, nullptr));
  }
  if (tier) *tier = ops->o.tier;
  return EIFMM_OK;
}

static void invalidate_batch(const void* h);

extern "C" void eifmm_ops_destroy(eifmm_ops* ops) {
  if (!ops) return;
  {
    std::lock_guard<std::mutex> lock(g_live_mu);
    g_live_ops.erase(ops->o.uid);
  }
  invalidate_batch(ops);
  free_ops(&ops->o);
  delete ops;
}

extern "C" eifmm_status eifmm_tree_build(const double* src_xyz, int64_t n_src,
                                         const double* tgt_xyz, int64_t n_tgt, const double lo[3],
                                         double L, int depth, int exclude_self,
                                         eifmm_stream stream, eifmm_tree** out) {
  if (!out || !lo || n_src < 0 || n_tgt < 0 || (n_src > 0 && !src_xyz) ||
      (n_tgt > 0 && !tgt_xyz) || depth < 2 || depth > kMaxLevel || !(L > 0.0) ||
      n_src >= ((int64_t)1 << 31) || n_tgt >= ((int64_t)1 << 31)) {
    set_error("eifmm_tree_build: invalid argument");
    return EIFMM_EINVAL;
  }
  const bool same = (src_xyz == tgt_xyz && n_src == n_tgt);
  if (exclude_self && !same) {
    set_error("eifmm_tree_build: exclude_self needs the target array to be the source array");
    return EIFMM_EINVAL;
  }
  *out = nullptr;
  eifmm_tree* h = new eifmm_tree();
  Tree& t = h->t;
  t.depth = depth;
  t.L = L;
  for (int a = 0; a < 3; ++a) t.lo[a] = lo[a];
  t.exclude_self = exclude_self ? 1 : 0;
  t.same = same;
  cudaStream_t s = (cudaStream_t)stream;
  eifmm_status rc = build_pointset(src_xyz, n_src, lo, L, depth, s, &t.src);
  if (rc == EIFMM_OK) {
    if (same) t.tgt = t.src;
    else rc = build_pointset(tgt_xyz, n_tgt, lo, L, depth, s, &t.tgt);
  }
  if (rc != EIFMM_OK) {
    free_pointset(&t.src);
    if (!same) free_pointset(&t.tgt);
    delete h;
    return rc;
  }
  *out = h;
  return EIFMM_OK;
}

extern "C" eifmm_status eifmm_tree_export(const eifmm_tree* tree, int which, uint32_t* keys,
                                          int32_t* perm, int64_t* leaf_off) {
  if (!tree || (which != 0 && which != 1)) {
    set_error("eifmm_tree_export: invalid handle or `which`");
    return EIFMM_EINVAL;
  }
  const PointSet& p = which == 0 ? tree->t.src : tree->t.tgt;
  if (keys && p.n) EIFMM_CUDA(cudaMemcpy(keys, p.keys, p.n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (perm && p.n) EIFMM_CUDA(cudaMemcpy(perm, p.perm, p.n * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (leaf_off) {
    const int64_t nl = ((int64_t)1 << (3 * tree->t.depth)) + 1;
    std::vector<int32_t> tmp(nl);
    EIFMM_CUDA(cudaMemcpy(tmp.data(), p.leaf_off, nl * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < nl; ++i) leaf_off[i] = tmp[i];
  }
  return EIFMM_OK;
}

extern "C" void eifmm_tree_destroy(eifmm_tree* tree) {
  if (!tree) return;
  invalidate_batch(tree);
  // the library's own streams of this tree finish first; work on the
  // caller's streams is the caller's to finish (see the header)
  Workspace& ws = tree->t.ws;
  for (cudaStream_t st : {ws.side, ws.side2, ws.hi})
    if (st) cudaStreamSynchronize(st);
  free_workspace(&tree->t.ws);
  free_streams(&tree->t.ws);
  free_pointset(&tree->t.src);
  if (!tree->t.same) free_pointset(&tree->t.tgt);
  delete tree;
}

extern "C" eifmm_status eifmm_tree_set_option(eifmm_tree* tree, eifmm_option opt, int value) {
  if (!tree || (int)opt < 0 || (int)opt >= kNumOptions || (value != 0 && value != 1)) {
    set_error("eifmm_tree_set_option: null tree, unknown option or value other than 0 or 1");
    return EIFMM_EINVAL;
  }
  tree->t.opt[(int)opt] = value;
  return EIFMM_OK;
}

static eifmm_status check_eval(const eifmm_tree* tree, const eifmm_ops* ops, int n_rhs,
                               int64_t ld_sigma, int64_t ld_f, int prec) {
  if (!tree || !ops || n_rhs < 1 || n_rhs > kMaxRhs || (prec != 0 && prec != 1)) {
    set_error("eifmm_evaluate: invalid handle, n_rhs or precision");
    return EIFMM_EINVAL;
  }
  const Tree& t = tree->t;
  if (ops->o.depth < t.depth || ops->o.L != t.L) {
    set_error("eifmm_evaluate: operator depth below the tree depth, or another L");
    return EIFMM_EINVAL;
  }
  if (ld_sigma < t.src.n || ld_f < t.tgt.n) {
    set_error("eifmm_evaluate: leading dimension smaller than the number of points");
    return EIFMM_EINVAL;
  }
  return EIFMM_OK;
}

static eifmm_status evaluate_impl(eifmm_tree* tree, const eifmm_ops* ops, const double* sigma,
                                  int64_t ld_sigma, int n_rhs, double* f, int64_t ld_f,
                                  int prec, cudaStream_t s) {
  Tree& t = tree->t;
  EIFMM_TRY(ensure_workspace(&t, &ops->o, n_rhs, prec));
  eifmm_status rc;
  if (prec == EIFMM_PREC_FP64)
    rc = eval_fp64(&t, &ops->o, sigma, ld_sigma, n_rhs, f, ld_f, s);
  else if (ops->o.tier >= 4)  // FP64 everywhere, the M2L in FP32 pairs
    rc = eval_fp64(&t, &ops->o, sigma, ld_sigma, n_rhs, f, ld_f, s, false, true);
  else
    rc = eval_mixed(&t, &ops->o, sigma, ld_sigma, n_rhs, f, ld_f, s);
  if (rc != EIFMM_OK) return rc;
  t.ws.evaluated = true;
  if (g_timing) {
    EIFMM_CUDA(cudaEventSynchronize(t.ws.ev_t[8]));
    for (int i = 0; i < 8; ++i) cudaEventElapsedTime(&t.ws.step_ms[i], t.ws.ev_t[i], t.ws.ev_t[i + 1]);
    cudaEventElapsedTime(&t.ws.step_ms[8], t.ws.ev_nf[0], t.ws.ev_nf[1]);
    for (int k = 2; k <= t.depth; ++k)
      cudaEventElapsedTime(&t.ws.step_ms[9 + k], t.ws.ev_m2l[k], t.ws.ev_m2le[k]);
  }
  return EIFMM_OK;
}


// ---------------------------------------------------------------------------
// Measured choice of the mixed-precision tier.  A uniform problem of 32 points
// per leaf (the near field carries its usual share of the result) is
// evaluated at depth min(depth, 4) with the operators' own kernel in FP64
// and in every mixed tier; the cheapest tier whose relative L2
// difference to FP64 stays below eps/4 is kept (else tier 4: FP64
// throughout, the M2L in FP32 pairs).
// ---------------------------------------------------------------------------
extern "C" eifmm_status eifmm_ops_calibrate(eifmm_ops* ops, double eps, eifmm_stream stream,
                                            int* tier_out) {
  if (!ops || !(eps > 0.0)) {
    set_error("eifmm_ops_calibrate: invalid handle or eps");
    return EIFMM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int depth = ops->o.depth < 4 ? ops->o.depth : 4;
  const int64_t n = (int64_t)32 << (3 * depth);
  const double L = ops->o.L;
  std::vector<double> hx(3 * n), hs(n);
  uint64_t st = 0x9E3779B97F4A7C15ull;
  auto next = [&]() {  // splitmix64
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (double)((z ^ (z >> 31)) >> 11) * 0x1.0p-53;
  };
  for (int64_t i = 0; i < 3 * n; ++i) hx[i] = L * next();
  for (int64_t i = 0; i < n; ++i) hs[i] = 2.0 * next() - 1.0;
  double *dx = nullptr, *ds = nullptr, *fr = nullptr, *fm = nullptr;
  eifmm_tree* tree = nullptr;
  eifmm_status rc = EIFMM_OK;
  int best = 4;
  for (double& e : ops->o.calib_err) e = -1.0;
  ops->o.calib_tier = -1;
  do {
    if ((rc = dalloc(&dx, 3 * n)) != EIFMM_OK) break;
    if ((rc = dalloc(&ds, n)) != EIFMM_OK) break;
    if ((rc = dalloc(&fr, n)) != EIFMM_OK) break;
    if ((rc = dalloc(&fm, n)) != EIFMM_OK) break;
    if (cudaMemcpy(dx, hx.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ds, hs.data(), n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = EIFMM_ECUDA;
      set_error("eifmm_ops_calibrate: upload failed");
      break;
    }
    const double lo[3] = {0.0, 0.0, 0.0};
    if ((rc = eifmm_tree_build(dx, n, dx, n, lo, L, depth, 1, stream, &tree)) != EIFMM_OK) break;
    // a view of the operators restricted to the calibration depth
    eifmm_ops view;
    view.o = ops->o;
    view.o.depth = depth;
    if ((rc = evaluate_impl(tree, &view, ds, n, 1, fr, n, EIFMM_PREC_FP64, s)) != EIFMM_OK) break;
    std::vector<double> href(n), hm(n);
    if (cudaMemcpyAsync(href.data(), fr, n * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = EIFMM_ECUDA;
      set_error("eifmm_ops_calibrate: copy failed");
      break;
    }
    double nref = 0.0;
    for (double v : href) nref += v * v;
    for (int t = 0; t <= 3 && rc == EIFMM_OK; ++t) {
      if (t <= 1 && (rc = build_kd_image(&ops->o, t == 1 ? kPlaneF16 : kPlaneBF16, s)) != EIFMM_OK) break;
      if (t == 2 && (rc = build_kd32(&ops->o, s)) != EIFMM_OK) break;
      // tier 0 needs its M2L operand image at every level (d too large: the
      // tier is skipped); tier 1 runs the SIMT M2L where it has none
      bool have_img = true;
      for (int k = 2; k <= depth; ++k)
        if (t == 0 && ops->o.lv[k].kd_img == nullptr) have_img = false;
      if (!have_img) continue;
      view.o = ops->o;
      view.o.depth = depth;
      view.o.tier = t;
      rc = evaluate_impl(tree, &view, ds, n, 1, fm, n, EIFMM_PREC_MIXED, s);
      if (rc == EIFMM_EUNSUPPORTED) {  // this tier cannot run these operators
        rc = EIFMM_OK;
        continue;
      }
      if (rc != EIFMM_OK) break;
      cudaMemcpyAsync(hm.data(), fm, n * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) {
        rc = EIFMM_ECUDA;
        set_error("eifmm_ops_calibrate: evaluation failed");
        break;
      }
      double ne = 0.0;
      for (int64_t i = 0; i < n; ++i) ne += (hm[i] - href[i]) * (hm[i] - href[i]);
      const double err = sqrt(ne / (nref > 0 ? nref : 1.0));
      ops->o.calib_err[t] = err;
      if (err <= 0.25 * eps) {
        best = t;
        break;
      }
    }
  } while (false);
  if (tree) eifmm_tree_destroy(tree);
  dfree(dx);
  dfree(ds);
  dfree(fr);
  dfree(fm);
  if (rc != EIFMM_OK) return rc;
  EIFMM_TRY(eifmm_ops_plan(ops, best, nullptr));
  ops->o.calib_tier = best;
  if (tier_out) *tier_out = best;
  return EIFMM_OK;
}

extern "C" eifmm_status eifmm_wait_selftest(int64_t limit_cycles, int* code) {
  if (limit_cycles < 0) {
    set_error("eifmm_wait_selftest: negative limit");
    return EIFMM_EINVAL;
  }
  return wait_selftest((long long)limit_cycles, code);
}

extern "C" eifmm_status eifmm_ops_compress(eifmm_ops* ops, double eps, eifmm_stream stream, int* ranks) {
  if (!ops || !(eps >= 0.0) || eps >= 1.0) {
    set_error("eifmm_ops_compress: null handle or eps outside [0, 1)");
    return EIFMM_EINVAL;
  }
  EIFMM_TRY(compress_ops(&ops->o, eps, (cudaStream_t)stream));
  if (ranks)
    for (int k = 0; k <= kMaxLevel; ++k) ranks[k] = (k >= 2 && k <= ops->o.depth) ? ops->o.lv[k].r : 0;
  return EIFMM_OK;
}

extern "C" eifmm_status eifmm_ops_basis(const eifmm_ops* ops, int level, double* U, int* d, int* r,
                                        double* info) {
  if (!ops || level < 2 || level > ops->o.depth) {
    set_error("eifmm_ops_basis: null handle or level outside [2, depth]");
    return EIFMM_EINVAL;
  }
  const LevelOps& v = ops->o.lv[level];
  if (d) *d = v.d;
  if (r) *r = v.r;
  if (info) {
    info[0] = v.r_i;
    info[1] = v.r_ii;
    info[2] = v.s_kept;
    info[3] = v.s_next;
  }
  if (U && v.r > 0) EIFMM_CUDA(cudaMemcpy(U, v.U, (size_t)v.d * v.r * sizeof(double), cudaMemcpyDeviceToHost));
  return EIFMM_OK;
}

extern "C" eifmm_status eifmm_ops_calibration(const eifmm_ops* ops, double* err4, int* tier) {
  if (!ops) {
    set_error("eifmm_ops_calibration: null handle");
    return EIFMM_EINVAL;
  }
  if (err4)
    for (int t = 0; t < 4; ++t) err4[t] = ops->o.calib_err[t];
  if (tier) *tier = ops->o.calib_tier;
  return EIFMM_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the tensor-core M2L (no counterpart in the paper): per level,
// every applicable variant and offset-group count is timed on this tree with
// CUDA events and the fastest is kept in the tree's workspace.
// ---------------------------------------------------------------------------
extern "C" eifmm_status eifmm_autotune(eifmm_tree* tree, const eifmm_ops* ops, int n_rhs,
                                       eifmm_precision prec, eifmm_stream stream, int* choice) {
  if (!tree || !ops) {
    set_error("eifmm_autotune: null handle");
    return EIFMM_EINVAL;
  }
  Tree& t = tree->t;
  EIFMM_TRY(check_eval(tree, ops, n_rhs, t.src.n, t.tgt.n, (int)prec));
  if (choice)
    for (int k = 0; k <= kMaxLevel; ++k) choice[2 * k] = choice[2 * k + 1] = 0;
  if (prec != EIFMM_PREC_MIXED || ops->o.tier >= 2) return EIFMM_OK;  // no tensor-core M2L
  cudaStream_t s = (cudaStream_t)stream;
  const int R = n_rhs, kap = t.depth;
  const int64_t ns = t.src.n > 0 ? t.src.n : 1, nt = t.tgt.n > 0 ? t.tgt.n : 1;
  double *sg = nullptr, *fo = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  eifmm_status rc = EIFMM_OK;
  do {
    // one evaluation (sigma = 0) sets up the workspace and the operand planes
    if ((rc = dalloc(&sg, (size_t)ns * R)) != EIFMM_OK) break;
    if ((rc = dalloc(&fo, (size_t)nt * R)) != EIFMM_OK) break;
    cudaMemsetAsync(sg, 0, (size_t)ns * R * sizeof(double), s);
    if ((rc = evaluate_impl(tree, ops, sg, ns, R, fo, nt, (int)prec, s)) != EIFMM_OK) break;
    Workspace& ws = t.ws;
    for (int k = 0; k <= kMaxLevel; ++k) ws.m2l_kind[k] = ws.m2l_gshift[k] = 0;
    ws.p2p_sym = 0;
    // room for the partial sums of larger group counts, within 1 GiB per
    // buffer (the leaf level has its own: it runs concurrently)
    size_t want = ws.m2l_part_cap, want_leaf = ws.m2l_part_leaf_cap;
    for (int k = 2; k <= kap; ++k) {
      const size_t per = ((size_t)1 << (3 * k)) * R * ops->o.lv[k].dp;
      size_t& w = k == kap ? want_leaf : want;
      for (int g = 2; g <= 16; g *= 2)
        if (g * per <= ((size_t)1 << 28) && g * per > w) w = g * per;
    }
    if (want > ws.m2l_part_cap) {
      dfree(ws.m2l_part);
      ws.m2l_part = nullptr;
      ws.m2l_part_cap = 0;
      if ((rc = dalloc(&ws.m2l_part, want)) != EIFMM_OK) break;
      ws.m2l_part_cap = want;
    }
    if (want_leaf > ws.m2l_part_leaf_cap) {
      dfree(ws.m2l_part_leaf);
      ws.m2l_part_leaf = nullptr;
      ws.m2l_part_leaf_cap = 0;
      if ((rc = dalloc(&ws.m2l_part_leaf, want_leaf)) != EIFMM_OK) break;
      ws.m2l_part_leaf_cap = want_leaf;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = EIFMM_ECUDA;
      set_error("eifmm_autotune: event creation failed");
      break;
    }
    for (int k = 2; k <= kap && rc == EIFMM_OK; ++k) {
      float best = 1e30f;
      int bk = 0, bg = 0;
      for (int kind = 0; kind <= 3 && rc == EIFMM_OK; ++kind)
        for (int gs = -1; gs <= 1; ++gs) {
          if (kind == 0 && gs != 0) continue;  // the built-in rule as it stands
          eifmm_status r = launch_m2l_level(&t, &ops->o, k, R, kind, gs, s);  // warm-up
          if (r == EIFMM_EUNSUPPORTED) continue;
          if (r != EIFMM_OK) {
            rc = r;
            break;
          }
          float ms[3];
          for (int rep = 0; rep < 3 && rc == EIFMM_OK; ++rep) {
            cudaEventRecord(e0, s);
            rc = launch_m2l_level(&t, &ops->o, k, R, kind, gs, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms[rep], e0, e1);
          }
          if (rc != EIFMM_OK) break;
          const float med = ms[0] < ms[1] ? (ms[1] < ms[2] ? ms[1] : (ms[0] < ms[2] ? ms[2] : ms[0]))
                                          : (ms[0] < ms[2] ? ms[0] : (ms[1] < ms[2] ? ms[2] : ms[1]));
          if (med < best * 0.98f) {  // a variant must win by 2% to replace the rule
            best = med;
            bk = kind;
            bg = gs;
          }
        }
      ws.m2l_kind[k] = bk;
      ws.m2l_gshift[k] = bg;
      if (choice) {
        choice[2 * k] = bk;
        choice[2 * k + 1] = bg;
      }
    }
    // the near field of tier 0 with one right-hand side and targets =
    // sources: the per-target kernel against the pair-symmetric one
    if (rc == EIFMM_OK && ops->o.tier == 0 && R == 1 && t.same && t.exclude_self && ws.gsym) {
      float tn[2] = {1e30f, 1e30f};
      for (int v = 0; v < 2 && rc == EIFMM_OK; ++v) {
        ws.p2p_sym = v;
        float ms[3];
        for (int rep = 0; rep < 4 && rc == EIFMM_OK; ++rep) {  // the first is a warm-up
          cudaEventRecord(e0, s);
          rc = launch_p2p32(&t, (int)ops->o.kern, ws.sig32, R, ws.fnear, s, false, ws.gsym);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          if (rep > 0) cudaEventElapsedTime(&ms[rep - 1], e0, e1);
        }
        // the median of the three
        tn[v] = ms[0] + ms[1] + ms[2] - std::min(ms[0], std::min(ms[1], ms[2])) -
                std::max(ms[0], std::max(ms[1], ms[2]));
      }
      ws.p2p_sym = tn[1] < tn[0] * 0.98f ? 1 : 0;  // the pair-symmetric kernel must win by 2%
      if (choice) choice[0] = ws.p2p_sym;
    }
    if (rc == EIFMM_OK && cudaStreamSynchronize(s) != cudaSuccess) {
      rc = EIFMM_ECUDA;
      set_error("eifmm_autotune: a timed launch failed");
    }
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dfree(sg);
  dfree(fo);
  return rc;
}

extern "C" eifmm_status eifmm_evaluate(eifmm_tree* tree, const eifmm_ops* ops, const double* sigma,
                                       int64_t ld_sigma, int n_rhs, double* f, int64_t ld_f,
                                       eifmm_precision prec, eifmm_stream stream) {
  EIFMM_TRY(check_eval(tree, ops, n_rhs, ld_sigma, ld_f, (int)prec));
  if ((tree->t.src.n > 0 && !sigma) || (tree->t.tgt.n > 0 && !f)) {
    set_error("eifmm_evaluate: null sigma or f");
    return EIFMM_EINVAL;
  }
  if (tree->t.tgt.n == 0) return EIFMM_OK;
  return evaluate_impl(tree, ops, sigma, ld_sigma, n_rhs, f, ld_f, (int)prec, (cudaStream_t)stream);
}

extern "C" eifmm_status eifmm_evaluate_host(eifmm_tree* tree, const eifmm_ops* ops,
                                            const double* sigma_host, int64_t ld_sigma, int n_rhs,
                                            double* f_host, int64_t ld_f, eifmm_precision prec,
                                            eifmm_stream stream) {
  EIFMM_TRY(check_eval(tree, ops, n_rhs, ld_sigma, ld_f, (int)prec));
  Tree& t = tree->t;
  if ((t.src.n > 0 && !sigma_host) || (t.tgt.n > 0 && !f_host)) {
    set_error("eifmm_evaluate_host: null sigma or f");
    return EIFMM_EINVAL;
  }
  if (t.tgt.n == 0) return EIFMM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace& ws = t.ws;
  const size_t need = (size_t)(t.src.n > t.tgt.n ? t.src.n : t.tgt.n) * n_rhs;
  if (ws.host_cap < need) {
    dfree(ws.host_sig);
    dfree(ws.host_f);
    ws.host_sig = ws.host_f = nullptr;
    ws.host_cap = 0;
    EIFMM_TRY(dalloc(&ws.host_sig, need));
    EIFMM_TRY(dalloc(&ws.host_f, need));
    ws.host_cap = need;
  }
  for (int r = 0; r < n_rhs; ++r)
    EIFMM_CUDA(cudaMemcpyAsync(ws.host_sig + (size_t)r * t.src.n, sigma_host + (size_t)r * ld_sigma,
                               t.src.n * sizeof(double), cudaMemcpyHostToDevice, s));
  EIFMM_TRY(evaluate_impl(tree, ops, ws.host_sig, t.src.n, n_rhs, ws.host_f, t.tgt.n, (int)prec, s));
  for (int r = 0; r < n_rhs; ++r)
    EIFMM_CUDA(cudaMemcpyAsync(f_host + (size_t)r * ld_f, ws.host_f + (size_t)r * t.tgt.n,
                               t.tgt.n * sizeof(double), cudaMemcpyDeviceToHost, s));
  EIFMM_CUDA(cudaStreamSynchronize(s));
  return EIFMM_OK;
}

// The batch is recorded once into a CUDA graph (after one direct pass that
// sizes every workspace) and replayed by a single cudaGraphLaunch while the
// same trees, operators, precision and array pointers are passed again.  The
// problems run on kBranches parallel branches (balanced by an estimated
// cost, below), each tree on its own workspace and streams and the
// operators only read, so the many small launches of uneven problems
// overlap instead of following one another.
constexpr int kBranches = 8;
namespace {
struct BatchGraph {
  std::vector<const void*> key;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  int dev = -1;  // device of the branch streams
  cudaStream_t br[kBranches] = {};
  cudaEvent_t fork = nullptr, join[kBranches] = {};
};
BatchGraph g_batch;
std::mutex g_batch_mu;  // guards g_batch
}  // namespace

// A graph refers to the workspaces of its trees and operators: drop it when
// one of them is destroyed.
static void invalidate_batch(const void* h) {
  std::lock_guard<std::mutex> lock(g_batch_mu);
  if (!g_batch.exec) return;
  for (const void* k : g_batch.key)
    if (k == h) {
      cudaGraphExecDestroy(g_batch.exec);
      g_batch.exec = nullptr;
      g_batch.key.clear();
      return;
    }
}

extern "C" eifmm_status eifmm_evaluate_batched(eifmm_tree* const* trees, const double* const* sigma,
                                               double* const* f, int n_problems,
                                               const eifmm_ops* ops, eifmm_precision prec,
                                               eifmm_stream stream) {
  if (!trees || !sigma || !f || n_problems < 0 || !ops || (prec != 0 && prec != 1)) {
    set_error("eifmm_evaluate_batched: invalid argument");
    return EIFMM_EINVAL;
  }
  for (int p = 0; p < n_problems; ++p) {
    if (!trees[p]) {
      set_error("eifmm_evaluate_batched: null tree");
      return EIFMM_EINVAL;
    }
    EIFMM_TRY(check_eval(trees[p], ops, 1, trees[p]->t.src.n, trees[p]->t.tgt.n, (int)prec));
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_batch_mu);
  std::vector<const void*> key;
  key.push_back(ops);
  key.push_back((const void*)(intptr_t)prec);
  key.push_back((const void*)(intptr_t)ops->o.tier);
  key.push_back((const void*)s);
  for (int p = 0; p < n_problems; ++p) {
    key.push_back(trees[p]);
    key.push_back(sigma[p]);
    key.push_back(f[p]);
  }
  if (g_batch.exec && g_batch.key == key && !g_timing) {
    EIFMM_CUDA(cudaGraphLaunch(g_batch.exec, s));
    for (int p = 0; p < n_problems; ++p) trees[p]->t.ws.evaluated = true;
    return EIFMM_OK;
  }
  // the branch streams of this device
  int dev = 0;
  EIFMM_CUDA(cudaGetDevice(&dev));
  if (g_batch.dev != dev) {
    for (int b = 0; b < kBranches; ++b) {
      if (g_batch.br[b]) cudaStreamDestroy(g_batch.br[b]);
      if (g_batch.join[b]) cudaEventDestroy(g_batch.join[b]);
      g_batch.br[b] = nullptr;
      g_batch.join[b] = nullptr;
    }
    if (g_batch.fork) cudaEventDestroy(g_batch.fork);
    g_batch.fork = nullptr;
    g_batch.dev = -1;
    EIFMM_CUDA(cudaEventCreateWithFlags(&g_batch.fork, cudaEventDisableTiming));
    for (int b = 0; b < kBranches; ++b) {
      EIFMM_CUDA(cudaStreamCreateWithFlags(&g_batch.br[b], cudaStreamNonBlocking));
      EIFMM_CUDA(cudaEventCreateWithFlags(&g_batch.join[b], cudaEventDisableTiming));
    }
    g_batch.dev = dev;
  }
  // every problem on a branch: largest estimated cost first, each to the
  // branch with the least cost so far (longest-processing-time order), so
  // that the few deep problems of an uneven batch do not share a branch.
  // Cost: the leaf-level M2L (boxes x d^2) plus the near field (points x
  // 27 leaves' points).
  const int K = n_problems < kBranches ? (n_problems > 0 ? n_problems : 1) : kBranches;
  std::vector<int> order(n_problems), branch(n_problems, 0);
  {
    std::vector<double> cost(n_problems);
    for (int p = 0; p < n_problems; ++p) {
      const Tree& t = trees[p]->t;
      const double boxes = std::ldexp(1.0, 3 * t.depth);
      const double dl = t.depth <= ops->o.depth ? ops->o.lv[t.depth].d : 1.0;
      const double per_leaf = (double)t.src.n / boxes;
      cost[p] = boxes * dl * dl + (double)t.tgt.n * 27.0 * per_leaf;
      order[p] = p;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    double load[kBranches] = {};
    for (int p : order) {
      int b = 0;
      for (int c = 1; c < K; ++c)
        if (load[c] < load[b]) b = c;
      branch[p] = b;
      load[b] += cost[p];
    }
  }
  // the branches fork from and join into s
  auto run_all = [&]() -> eifmm_status {
    EIFMM_CUDA(cudaEventRecord(g_batch.fork, s));
    for (int b = 0; b < K; ++b) EIFMM_CUDA(cudaStreamWaitEvent(g_batch.br[b], g_batch.fork, 0));
    eifmm_status rc = EIFMM_OK;
    for (int i = 0; i < n_problems && rc == EIFMM_OK; ++i) {
      const int p = order[i];
      if (trees[p]->t.tgt.n == 0) continue;
      rc = evaluate_impl(trees[p], ops, sigma[p], trees[p]->t.src.n, 1, f[p], trees[p]->t.tgt.n, (int)prec,
                         g_batch.br[branch[p]]);
    }
    for (int b = 0; b < K; ++b) {  // joined also after a failure
      cudaEventRecord(g_batch.join[b], g_batch.br[b]);
      cudaStreamWaitEvent(s, g_batch.join[b], 0);
    }
    return rc;
  };
  // direct pass (sizes the workspaces; also the result of this call)
  EIFMM_TRY(run_all());
  if (g_timing || s == nullptr) return EIFMM_OK;  // the legacy stream cannot be captured
  if (g_batch.exec) {
    cudaGraphExecDestroy(g_batch.exec);
    g_batch.exec = nullptr;
    g_batch.key.clear();
  }
  EIFMM_CUDA(cudaStreamSynchronize(s));
  cudaGraph_t graph = nullptr;
  EIFMM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  eifmm_status rc = run_all();
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (rc != EIFMM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) {
    set_error(std::string("eifmm_evaluate_batched: stream capture failed: ") + cudaGetErrorString(e));
    return EIFMM_ECUDA;
  }
  e = cudaGraphInstantiate(&g_batch.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g_batch.exec = nullptr;
    set_error(std::string("eifmm_evaluate_batched: graph instantiation failed: ") + cudaGetErrorString(e));
    return EIFMM_ECUDA;
  }
  g_batch.key = key;
  g_batch.stream = s;
  return EIFMM_OK;
}

namespace eifmm {
eifmm_status export_mixed(const Tree& t, const Ops& o, int what, int level, double* out, int64_t n);
}

extern "C" eifmm_status eifmm_debug_export(const eifmm_tree* tree, int what, int level,
                                           double* out, int64_t n) {
  if (!tree || !out || !tree->t.ws.evaluated) {
    set_error("eifmm_debug_export: nothing evaluated on this tree");
    return EIFMM_EINVAL;
  }
  const Tree& t = tree->t;
  const Workspace& ws = t.ws;
  const int R = ws.nrhs;
  EIFMM_CUDA(cudaDeviceSynchronize());
  if (what == 5 || what == 6) {
    if (n < t.tgt.n * R) {
      set_error("eifmm_debug_export: output too small");
      return EIFMM_EINVAL;
    }
    const double* src = what == 5 ? ws.ffar : ws.fnear;
    std::vector<double> tmp((size_t)t.tgt.n * R);
    std::vector<int32_t> perm(t.tgt.n);
    EIFMM_CUDA(cudaMemcpy(tmp.data(), src, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost));
    EIFMM_CUDA(cudaMemcpy(perm.data(), t.tgt.perm, t.tgt.n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int r = 0; r < R; ++r)
      for (int64_t p = 0; p < t.tgt.n; ++p) out[perm[p] + r * t.tgt.n] = tmp[p + r * t.tgt.n];
    return EIFMM_OK;
  }
  if (level < 2 || level > t.depth || what < 0 || what > 4 || (what == 4 && level != t.depth)) {
    set_error("eifmm_debug_export: invalid `what` or level");
    return EIFMM_EINVAL;
  }
  if (!ops_alive(ws.ops_uid)) {
    set_error("eifmm_debug_export: the operators of the last evaluation were destroyed");
    return EIFMM_EINVAL;
  }
  const Ops& o = reinterpret_cast<const eifmm_ops*>(ws.ops_id)->o;
  const int d = o.lv[level].d;
  const int64_t cnt = ((int64_t)1 << (3 * level)) * R * d;
  if (n < cnt) {
    set_error("eifmm_debug_export: output too small");
    return EIFMM_EINVAL;
  }
  if (ws.W[level] == nullptr && ws.lh == nullptr) return export_mixed(t, o, what, level, out, n);
  if (what == 1) {
    // What = Delta W (the evaluation applies K^delta Delta to W instead)
    DeltaBatch b;
    b.nlev = 1;
    b.lv[0] = delta_level(d, delta_ops64(o.lv[level]), false, ws.W[level], d, ws.Wh[level], d, nullptr,
                          ((int64_t)1 << (3 * level)) * R);
    EIFMM_TRY((launch_delta_batch<double, double, double, 0>(b, false, 0)));
    EIFMM_CUDA(cudaDeviceSynchronize());
  }
  const double* src = what == 0 ? ws.W[level] : what == 1 ? ws.Wh[level] : what == 2 ? ws.g[level]
                     : what == 3 ? ws.l[level] : ws.lh;
  EIFMM_CUDA(cudaMemcpy(out, src, cnt * sizeof(double), cudaMemcpyDeviceToHost));
  return EIFMM_OK;
}

extern "C" eifmm_status eifmm_last_step_times(const eifmm_tree* tree, float* ms20) {
  if (!tree || !ms20) {
    set_error("eifmm_last_step_times: null argument");
    return EIFMM_EINVAL;
  }
  for (int i = 0; i < 20; ++i) ms20[i] = tree->t.ws.step_ms[i];
  return EIFMM_OK;
}
