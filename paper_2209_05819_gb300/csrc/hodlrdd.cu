// C ABI of libhodlrdd: argument checks, handle lifecycle, build orchestration
// (Algorithm 1 on the device), matvec dispatch (Algorithm 2), statistics and
// read-only introspection of the integer structure.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>

#include "internal.cuh"

namespace hd {

namespace {
thread_local std::string g_last_error = "";
std::atomic<int64_t> g_fail_after{-1};
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  std::snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  g_last_error = buf;
  if (e == cudaErrorMemoryAllocation) return HODLRDD_ERR_OOM;
  return HODLRDD_ERR_CUDA;
}

void debug_fail_alloc_after(int64_t k) { g_fail_after.store(k); }

namespace {
std::atomic<int64_t> g_aca_pool_cap{-1};
}  // namespace
int64_t debug_aca_pool_bytes() { return g_aca_pool_cap.load(); }

int dev_alloc(void** p, size_t bytes) {
  int64_t f = g_fail_after.load();
  if (f >= 0) {
    if (f == 0) {
      g_fail_after.store(-1);
      set_error("device allocation failed (injected)");
      return HODLRDD_ERR_OOM;
    }
    g_fail_after.store(f - 1);
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[160];
    std::snprintf(buf, sizeof buf, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    set_error(buf);
    return HODLRDD_ERR_OOM;
  }
  return HODLRDD_OK;
}

namespace {

// 0 host, 1 device (of any device), -1 error.
int pointer_kind(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? 1 : 0;
}

bool kernel_ok(int id, const double* prm) {
  if (id < HODLRDD_K_LOG || id > HODLRDD_K_INV_SQRT1P) return false;
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(prm[i])) return false;
  if ((id == HODLRDD_K_MATERN32 || id == HODLRDD_K_GAUSS || id == HODLRDD_K_EXP) && !(prm[2] > 0.0)) return false;
  return true;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void fill_stats(hodlrdd_s* h) {
  hodlrdd_stats& s = h->stats;
  s.d = h->d;
  s.kappa = h->kappa;
  s.precision = h->opt.precision;
  s.N = h->N;
  s.n_blocks = h->nblk;
  s.n_lowrank = 0;
  s.n_dense = 0;
  s.max_rank = 0;
  for (int l = 0; l < HODLRDD_MAX_LEVELS; ++l) {
    s.boxes_per_level[l] = 0;
    s.blocks_per_level[l] = 0;
    s.max_rank_per_level[l] = 0;
    s.mean_rank_per_level[l] = 0.0;
  }
  std::vector<int64_t> rsum(h->kappa + 1, 0), rcnt(h->kappa + 1, 0);
  for (int64_t b = 0; b < h->nblk; ++b) {
    const int l = h->h_blevel[b];
    if (l < HODLRDD_MAX_LEVELS) s.blocks_per_level[l]++;
    if (h->h_dense[b]) {
      s.n_dense++;
    } else {
      s.n_lowrank++;
      s.max_rank = std::max(s.max_rank, h->h_rank[b]);
      if (l < HODLRDD_MAX_LEVELS) s.max_rank_per_level[l] = std::max(s.max_rank_per_level[l], h->h_rank[b]);
      rsum[l] += h->h_rank[b];
      rcnt[l]++;
    }
  }
  for (int l = 0; l <= h->kappa && l < HODLRDD_MAX_LEVELS; ++l) {
    s.boxes_per_level[l] = h->lv[l].nb;
    s.mean_rank_per_level[l] = rcnt[l] ? (double)rsum[l] / rcnt[l] : 0.0;
  }
  s.n_rank_capped = h->n_rank_capped;
  s.n_near = (int64_t)h->h_nearidx.size();
  s.factor_elems = h->factor_elems;
  s.factor_bytes = h->factor_bytes;
  s.dense_pairs = h->dense_pairs;
  const Plan& P = h->plan;
  int64_t bytes = (int64_t)(h->perm.bytes() + h->skey.bytes() + h->pts64.bytes() + h->pts32.bytes() +
                            h->nearoff.bytes() + h->nearidx.bytes() + h->bI0.bytes() + h->bm.bytes() +
                            h->bJ0.bytes() + h->bn.bytes() + h->rank.bytes() + h->dense.bytes() + h->toff.bytes() +
                            h->piv_sigma.bytes() + h->piv_tau.bytes() + h->su.bytes() + h->sv.bytes() +
                            h->xt.bytes() + h->tbuf.bytes() + h->ylev.bytes() + h->xstage.bytes() +
                            h->ystage.bytes() + P.vs.data.bytes() + P.us.data.bytes() + P.vs.panels.bytes() +
                            P.us.panels.bytes() + P.vs.stages.bytes() + P.us.stages.bytes() + P.vs.splits.bytes() +
                            P.us.splits.bytes() + P.vmap.bytes() + P.vs2.data.bytes() + P.us2.data.bytes() +
                            P.vs2.panels.bytes() + P.us2.panels.bytes() + P.vs2.stages.bytes() +
                            P.us2.stages.bytes() + P.vs2.splits.bytes() + P.us2.splits.bytes() + P.vmap2.bytes() +
                            h->pbuf.bytes() + h->ynear.bytes() + h->nctr.bytes() + h->err.bytes() + P.tasks.bytes() +
                            P.srcs.bytes() + P.soff.bytes() + P.tasks4.bytes() + P.srcs4.bytes() +
                            P.soff4.bytes() + P.tbox4.bytes() + P.brow4.bytes() + P.boff4.bytes() +
                            P.emask4.bytes());
  bytes += (int64_t)(P.sk_lu.bytes() + P.sk_luoff.bytes() + P.sk_blist.bytes() + P.sk_rtask.bytes() +
                     P.sk_rsum.bytes() + P.sk_rows.bytes() + P.sk_ctask.bytes() + P.sk_cols.bytes() +
                     P.sk_boff.bytes() + P.sk_part.bytes() + P.sk_hi.bytes() + P.sk_lo.bytes());
  for (auto& a : P.hi4) bytes += (int64_t)a.bytes();
  for (auto& a : P.lo4) bytes += (int64_t)a.bytes();
  for (auto& a : P.hq4) bytes += (int64_t)a.bytes();
  for (auto& a : P.lq4) bytes += (int64_t)a.bytes();
  for (auto& r : P.rel) bytes += (int64_t)r.bytes();
  bytes += tc_device_bytes(h);
  for (auto& L : h->lv)
    bytes += (int64_t)(L.bstart.bytes() + L.bkey.bytes() + L.cfirst.bytes() + L.iloff.bytes() + L.ilidx.bytes());
  s.device_bytes = bytes;
  const int64_t es = (int64_t)elem_size(h->opt.precision);
  s.factor_bytes_u = P.us.elems * es + P.us2.elems * 2 + P.tcu.rows * 128;
  s.factor_bytes_v = P.vs.elems * es + P.vs2.elems * 2 + P.tcv.rows * 128;
  s.tail_cols = P.tail_cols;
  s.total_rank = h->total_rank;
  s.lowrank_form = h->opt.lowrank_form;
  s.skeleton_bytes = P.sk_bytes;
  s.skeleton_pairs = P.sk_pairs;
  s.skeleton_terms = P.sk_terms;
  s.near_sms = h->opt.near_sms;
}

int validate_build(const double* points, int d, int64_t N, int kernel_id, const double* prm, int leaf, double tol,
                   const hodlrdd_options& o, hodlrdd_handle* out) {
  if (!out) { set_error("hodlrdd_build: out is NULL"); return HODLRDD_ERR_INVALID; }
  if (!points) { set_error("hodlrdd_build: points is NULL"); return HODLRDD_ERR_INVALID; }
  if (d < 1 || d > kMaxDim) { set_error("hodlrdd_build: d must be in 1..8"); return HODLRDD_ERR_INVALID; }
  if (N < 1 || N >= ((int64_t)1 << 31)) { set_error("hodlrdd_build: N must be in 1..2^31-1"); return HODLRDD_ERR_INVALID; }
  if (leaf < 1) { set_error("hodlrdd_build: leaf_size must be >= 1"); return HODLRDD_ERR_INVALID; }
  if (!(tol > 0.0) || !std::isfinite(tol)) { set_error("hodlrdd_build: tol must be > 0"); return HODLRDD_ERR_INVALID; }
  if (!kernel_ok(kernel_id, prm)) { set_error("hodlrdd_build: unknown kernel or invalid kernel parameters"); return HODLRDD_ERR_INVALID; }
  if (o.precision < HODLRDD_PREC_FP64 || o.precision > HODLRDD_PREC_FP16X2) { set_error("hodlrdd_build: unknown precision"); return HODLRDD_ERR_INVALID; }
  if (o.precision == HODLRDD_PREC_FP16X2 && (o.lowrank_form != 0 || d > 4)) {
    set_error("hodlrdd_build: the tensor-core form (FP16X2) needs lowrank_form 0 and d <= 4");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  if (o.max_nrhs < 1 || o.aca_max_rank < 1) { set_error("hodlrdd_build: max_nrhs and aca_max_rank must be >= 1"); return HODLRDD_ERR_INVALID; }
  if (o.dense_if_cheaper < 0 || o.dense_if_cheaper > 2) { set_error("hodlrdd_build: dense_if_cheaper must be 0, 1 or 2"); return HODLRDD_ERR_INVALID; }
  if (o.near_mode < 0 || o.near_mode > 2) { set_error("hodlrdd_build: near_mode must be 0, 1 or 2"); return HODLRDD_ERR_INVALID; }
  if (o.near_coords < 0 || o.near_coords > 1) {
    set_error("hodlrdd_build: near_coords must be 0 or 1");
    return HODLRDD_ERR_INVALID;
  }
  if (o.near_sms < -1 || o.near_sms > 4096) {
    set_error("hodlrdd_build: near_sms must be -1 or 0 .. SMs - 1");
    return HODLRDD_ERR_INVALID;
  }
  if (o.fp64_near < 0 || o.fp64_near > 1) {
    set_error("hodlrdd_build: fp64_near must be 0 or 1");
    return HODLRDD_ERR_INVALID;
  }
  if (o.fp64_near == 1 && o.precision == HODLRDD_PREC_FP64 && (d > 4 || kernel_id == HODLRDD_K_SIN)) {
    set_error("hodlrdd_build: the float-float FP64 near field (fp64_near 1) needs d <= 4 and a kernel other than sin r");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  if (o.admissible_face_dim < -1 || o.admissible_face_dim > d - 1) {
    set_error("hodlrdd_build: admissible_face_dim must be in -1 .. d - 1");
    return HODLRDD_ERR_INVALID;
  }
  if (o.lowrank_form < 0 || o.lowrank_form > 1) { set_error("hodlrdd_build: lowrank_form must be 0 or 1"); return HODLRDD_ERR_INVALID; }
  if (o.lowrank_form == 1) {
    if (o.precision != HODLRDD_PREC_FP64 && o.precision != HODLRDD_PREC_FP32) {
      set_error("hodlrdd_build: the skeleton form needs precision FP64 or FP32");
      return HODLRDD_ERR_UNSUPPORTED;
    }
    if (d > 4) { set_error("hodlrdd_build: the skeleton form needs d <= 4"); return HODLRDD_ERR_UNSUPPORTED; }
    if (o.aca_max_rank > 1024) {
      set_error("hodlrdd_build: the skeleton form needs aca_max_rank <= 1024");
      return HODLRDD_ERR_UNSUPPORTED;
    }
  }
  return HODLRDD_OK;
}

int do_build(hodlrdd_s* h, const double* points) {
  auto t0 = std::chrono::steady_clock::now();
  HD_CUDA(cudaGetDevice(&h->device));
  {
    int sms = 0;
    HD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    if (h->opt.near_sms >= sms) {
      set_error("hodlrdd_build: near_sms must be -1 or 0 .. SMs - 1");
      return HODLRDD_ERR_INVALID;
    }
  }
  HD_CUDA(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
  HD_CUDA(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
  HD_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  HD_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  // the caller's points, as a device array (copied if they live on the host)
  DevBuf<double> staged;
  const double* dpts = points;
  if (pointer_kind(points) == 0) {
    for (int64_t i = 0; i < h->N * h->d; ++i)
      if (!std::isfinite(points[i])) {
        set_error("hodlrdd_build: points contain NaN or Inf");
        return HODLRDD_ERR_INVALID;
      }
    HD_TRY(staged.alloc((size_t)h->N * h->d));
    HD_CUDA(cudaMemcpyAsync(staged.p, points, staged.bytes(), cudaMemcpyHostToDevice, h->st));
    dpts = staged.p;
  }
  auto t = std::chrono::steady_clock::now();
  HD_TRY(build_tree(h, dpts));
  staged.release();
  h->stats.t_tree_ms = ms_since(t);
  t = std::chrono::steady_clock::now();
  HD_TRY(build_lists(h));
  HD_TRY(build_blocks(h));
  h->stats.t_classify_ms = ms_since(t);
  t = std::chrono::steady_clock::now();
  DevBuf<double> U64, V64;
  std::vector<int64_t> uoff64, voff64;
  HD_TRY(run_aca(h, U64, V64, uoff64, voff64));
  h->stats.t_aca_ms = ms_since(t);
  t = std::chrono::steady_clock::now();
  if (h->opt.lowrank_form == 1) HD_TRY(build_skeleton(h, U64, V64, uoff64, voff64));
  else HD_TRY(pack_factors(h, U64, V64, uoff64, voff64));
  U64.release();
  V64.release();
  HD_TRY(build_plan(h));
  if (h->opt.lowrank_form == 1) HD_TRY(build_skeleton_plan(h));
  HD_TRY(alloc_workspace(h));
  if (h->opt.near_sms < 0) HD_TRY(tune_near_sms(h));
  HD_CUDA(cudaStreamSynchronize(h->st));
  h->stats.t_pack_ms = ms_since(t);
  h->stats.t_build_ms = ms_since(t0);
  fill_stats(h);
  return HODLRDD_OK;
}

void destroy(hodlrdd_s* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  if (h->aux) cudaStreamSynchronize(h->aux);
  cudaStream_t st = h->st, aux = h->aux;
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (auto& v : h->ev_pending)
    for (cudaEvent_t e : v) {
      cudaEventSynchronize(e);
      cudaEventDestroy(e);
    }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
  if (st) cudaStreamDestroy(st);
  if (aux) cudaStreamDestroy(aux);
}

}  // namespace

// The handle's kernels, workspace and streams live on the device it was built
// on; a call made while another device is current is rejected.
int check_device(const hodlrdd_s* h, const char* who) {
  int dev = 0;
  HD_CUDA(cudaGetDevice(&dev));
  if (dev != h->device) {
    char buf[200];
    std::snprintf(buf, sizeof buf, "%s: the current device (%d) is not the handle's device (%d)", who, dev,
                  h->device);
    set_error(buf);
    return HODLRDD_ERR_INVALID;
  }
  return HODLRDD_OK;
}

}  // namespace hd

using namespace hd;

extern "C" {

int hodlrdd_options_default(hodlrdd_options* opt) {
  if (!opt) return HODLRDD_ERR_INVALID;
  std::memset(opt, 0, sizeof *opt);
  opt->precision = HODLRDD_PREC_FP64;
  opt->dense_if_cheaper = 1;
  opt->max_nrhs = 8;
  opt->aca_max_rank = 1024;
  return HODLRDD_OK;
}

int hodlrdd_build_ex(const double* points, int d, int64_t N, int kernel_id, const double* kernel_params,
                     int leaf_size, double tol, const hodlrdd_options* opt, hodlrdd_handle* out) {
  hodlrdd_options o;
  hodlrdd_options_default(&o);
  if (opt) o = *opt;
  double prm[4] = {1.0, 0.0, 0.0, 0.0};
  if (kernel_params) std::memcpy(prm, kernel_params, sizeof prm);
  int s = validate_build(points, d, N, kernel_id, prm, leaf_size, tol, o, out);
  if (s != HODLRDD_OK) return s;
  *out = nullptr;
  hodlrdd_s* h = new (std::nothrow) hodlrdd_s();
  if (!h) {
    set_error("hodlrdd_build: host allocation failed");
    return HODLRDD_ERR_OOM;
  }
  h->d = d;
  h->N = N;
  h->K = KernelSpec{kernel_id, prm[0], prm[1], prm[2], prm[3]};
  h->leaf = leaf_size;
  h->tol = tol;
  h->opt = o;
  try {
    s = do_build(h, points);
  } catch (const std::bad_alloc&) {
    set_error("hodlrdd_build: host allocation failed");
    s = HODLRDD_ERR_OOM;
  }
  if (s != HODLRDD_OK) {
    destroy(h);
    return s;
  }
  *out = h;
  return HODLRDD_OK;
}

int hodlrdd_build(const double* points, int d, int64_t N, int kernel_id, const double* kernel_params, int leaf_size,
                  double tol, hodlrdd_handle* out) {
  return hodlrdd_build_ex(points, d, N, kernel_id, kernel_params, leaf_size, tol, nullptr, out);
}

int hodlrdd_matvec(hodlrdd_handle h, const void* x, void* y, int nrhs, void* stream) {
  if (!h || !x || !y || nrhs < 1) {
    set_error("hodlrdd_matvec: NULL handle / pointer or nrhs < 1");
    return HODLRDD_ERR_INVALID;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t io = h->opt.precision == HODLRDD_PREC_FP64 ? 8 : 4;
  const size_t bytes = (size_t)h->N * nrhs * io;
  const char* xa = static_cast<const char*>(x);
  char* ya = static_cast<char*>(y);
  if (xa < ya + bytes && ya < xa + bytes) {
    set_error("hodlrdd_matvec: x and y overlap");
    return HODLRDD_ERR_INVALID;
  }
  HD_TRY(check_device(h, "hodlrdd_matvec"));
  const bool xdev = pointer_kind(x) == 1, ydev = pointer_kind(y) == 1;
  if (xdev && ydev) return launch_matvec(h, x, y, nrhs, st);
  // host buffers: stage through handle-owned device memory, then wait
  if (h->xstage.bytes() < bytes) HD_TRY(h->xstage.alloc(bytes));
  if (h->ystage.bytes() < bytes) HD_TRY(h->ystage.alloc(bytes));
  const void* dx = x;
  void* dy = y;
  if (!xdev) {
    HD_CUDA(cudaMemcpyAsync(h->xstage.p, x, bytes, cudaMemcpyHostToDevice, st));
    dx = h->xstage.p;
  }
  if (!ydev) dy = h->ystage.p;
  int rc = launch_matvec(h, dx, dy, nrhs, st);
  if (rc == HODLRDD_OK && !ydev) {
    const cudaError_t e = cudaMemcpyAsync(y, h->ystage.p, bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(y)", __FILE__, __LINE__);
  }
  // also on failure: the copy from the caller's host x may still be in flight
  const cudaError_t e = cudaStreamSynchronize(st);
  if (rc == HODLRDD_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
  return rc;
}

int hodlrdd_direct(hodlrdd_handle h, const void* x, void* y, void* stream) {
  if (!h || !x || !y) {
    set_error("hodlrdd_direct: NULL handle or pointer");
    return HODLRDD_ERR_INVALID;
  }
  const size_t bytes = (size_t)h->N * sizeof(float);
  const char* xa = static_cast<const char*>(x);
  char* ya = static_cast<char*>(y);
  if (xa < ya + bytes && ya < xa + bytes) {
    set_error("hodlrdd_direct: x and y overlap");
    return HODLRDD_ERR_INVALID;
  }
  if (pointer_kind(x) != 1 || pointer_kind(y) != 1) {
    set_error("hodlrdd_direct: x and y must be device memory");
    return HODLRDD_ERR_INVALID;
  }
  HD_TRY(check_device(h, "hodlrdd_direct"));
  return launch_direct(h, static_cast<const float*>(x), static_cast<float*>(y), static_cast<cudaStream_t>(stream));
}

int hodlrdd_destroy(hodlrdd_handle h) {
  destroy(h);
  return HODLRDD_OK;
}

int hodlrdd_get_stats(hodlrdd_handle h, hodlrdd_stats* s) {
  if (!h || !s) return HODLRDD_ERR_INVALID;
  fill_stats(h);
  *s = h->stats;
  return HODLRDD_OK;
}

const char* hodlrdd_error_string(int status) {
  switch (status) {
    case HODLRDD_OK: return "success";
    case HODLRDD_ERR_INVALID: return "invalid argument";
    case HODLRDD_ERR_OOM: return "out of memory";
    case HODLRDD_ERR_CUDA: return "CUDA error";
    case HODLRDD_ERR_UNSUPPORTED: return "unsupported";
    case HODLRDD_ERR_TIMEOUT: return "device-side wait timed out";
    case HODLRDD_ERR_NUMERIC: return "non-finite values";
  }
  return "unknown status";
}

const char* hodlrdd_last_error(void) { return g_last_error.c_str(); }

int hodlrdd_get_tree(hodlrdd_handle h, int64_t* perm, uint64_t* keys) {
  if (!h) return HODLRDD_ERR_INVALID;
  for (int64_t i = 0; i < h->N; ++i) {
    if (perm) perm[i] = h->h_perm[i];
    if (keys) keys[i] = h->h_skey[i];
  }
  return HODLRDD_OK;
}

int hodlrdd_get_cube(hodlrdd_handle h, double* lo, double* side_inv) {
  if (!h || !lo || !side_inv) return HODLRDD_ERR_INVALID;
  for (int k = 0; k < h->d; ++k) lo[k] = h->lo[k];
  side_inv[0] = h->side;
  side_inv[1] = h->inv;
  return HODLRDD_OK;
}

int hodlrdd_get_level(hodlrdd_handle h, int l, int64_t* nboxes, int64_t* bstart, uint64_t* bkey) {
  if (!h || !nboxes || l < 0 || l > h->kappa) return HODLRDD_ERR_INVALID;
  const Level& L = h->lv[l];
  *nboxes = L.nb;
  if (bstart)
    for (int64_t b = 0; b <= L.nb; ++b) bstart[b] = L.h_bstart[b];
  if (bkey)
    for (int64_t b = 0; b < L.nb; ++b) bkey[b] = L.h_bkey[b];
  return HODLRDD_OK;
}

int hodlrdd_get_il(hodlrdd_handle h, int l, int64_t* nnz, int64_t* off, int64_t* idx) {
  if (!h || !nnz || l < 1 || l > h->kappa) return HODLRDD_ERR_INVALID;
  const Level& L = h->lv[l];
  *nnz = (int64_t)L.h_ilidx.size();
  if (off)
    for (size_t i = 0; i < L.h_iloff.size(); ++i) off[i] = L.h_iloff[i];
  if (idx)
    for (size_t i = 0; i < L.h_ilidx.size(); ++i) idx[i] = L.h_ilidx[i];
  return HODLRDD_OK;
}

int hodlrdd_get_near(hodlrdd_handle h, int64_t* nnz, int64_t* off, int64_t* idx) {
  if (!h || !nnz) return HODLRDD_ERR_INVALID;
  *nnz = (int64_t)h->h_nearidx.size();
  if (off)
    for (size_t i = 0; i < h->h_nearoff.size(); ++i) off[i] = h->h_nearoff[i];
  if (idx)
    for (size_t i = 0; i < h->h_nearidx.size(); ++i) idx[i] = h->h_nearidx[i];
  return HODLRDD_OK;
}

int hodlrdd_get_blocks(hodlrdd_handle h, int64_t* rec) {
  if (!h || !rec) return HODLRDD_ERR_INVALID;
  for (int64_t b = 0; b < h->nblk; ++b) {
    int64_t* r = rec + b * 9;
    r[0] = h->h_blevel[b]; r[1] = h->h_bti[b]; r[2] = h->h_bsj[b]; r[3] = h->h_bI0[b]; r[4] = h->h_bm[b];
    r[5] = h->h_bJ0[b]; r[6] = h->h_bn[b]; r[7] = h->h_rank[b]; r[8] = h->h_dense[b];
  }
  return HODLRDD_OK;
}

int hodlrdd_get_pivots(hodlrdd_handle h, int64_t b, int64_t* sigma, int64_t* tau) {
  if (!h || b < 0 || b >= h->nblk || !sigma || !tau) return HODLRDD_ERR_INVALID;
  const int p = h->h_rank[b];
  if (p == 0) return HODLRDD_OK;
  int64_t to = 0;
  HD_CUDA(cudaMemcpy(&to, h->toff.p + b, sizeof to, cudaMemcpyDeviceToHost));
  std::vector<int32_t> s(p), t(p);
  HD_CUDA(cudaMemcpy(s.data(), h->piv_sigma.p + to, p * sizeof(int32_t), cudaMemcpyDeviceToHost));
  HD_CUDA(cudaMemcpy(t.data(), h->piv_tau.p + to, p * sizeof(int32_t), cudaMemcpyDeviceToHost));
  for (int q = 0; q < p; ++q) {
    sigma[q] = s[q];
    tau[q] = t[q];
  }
  return HODLRDD_OK;
}

int hodlrdd_get_factors(hodlrdd_handle h, int64_t b, double* U, double* V) {
  if (!h || b < 0 || b >= h->nblk) return HODLRDD_ERR_INVALID;
  if (h->opt.lowrank_form != 0) {
    set_error("hodlrdd_get_factors: the handle is in the skeleton form (no factors kept)");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  if (h->opt.precision == HODLRDD_PREC_FP32_FP16 || h->opt.precision == HODLRDD_PREC_FP16X2) {
    set_error("hodlrdd_get_factors: not available for the mixed FP32 / FP16 and FP16X2 storage");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  return unpack_block(h, b, U, V);
}

int hodlrdd_import_factors(hodlrdd_handle h, const int32_t* rank, const int32_t* dense, const double* U_all,
                           const double* V_all) {
  if (!h || (!rank && h->nblk) || (!dense && h->nblk)) return HODLRDD_ERR_INVALID;
  if (h->opt.lowrank_form != 0) {
    set_error("hodlrdd_import_factors: the handle is in the skeleton form");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  const int64_t nblk = h->nblk;
  std::vector<int64_t> uoff64(nblk + 1, 0), voff64(nblk + 1, 0), toff(nblk + 1, 0);
  for (int64_t b = 0; b < nblk; ++b) {
    if (rank[b] < 0 || rank[b] > std::min(h->h_bm[b], h->h_bn[b]) || (dense[b] && rank[b] != 0)) {
      set_error("hodlrdd_import_factors: invalid rank / dense flag");
      return HODLRDD_ERR_INVALID;
    }
    uoff64[b + 1] = uoff64[b] + (int64_t)rank[b] * h->h_bm[b];
    voff64[b + 1] = voff64[b] + (int64_t)rank[b] * h->h_bn[b];
    toff[b + 1] = toff[b] + rank[b];
  }
  if ((uoff64[nblk] && !U_all) || (voff64[nblk] && !V_all)) return HODLRDD_ERR_INVALID;
  HD_CUDA(cudaStreamSynchronize(h->st));
  h->h_rank.assign(rank, rank + nblk);
  h->h_dense.assign(dense, dense + nblk);
  h->total_rank = toff[nblk];
  HD_TRY(upload(h->rank, h->h_rank, h->st));
  HD_TRY(upload(h->dense, h->h_dense, h->st));
  HD_TRY(upload(h->toff, toff, h->st));
  DevBuf<double> U64, V64;
  HD_TRY(U64.alloc(std::max<int64_t>(uoff64[nblk], 1)));
  HD_TRY(V64.alloc(std::max<int64_t>(voff64[nblk], 1)));
  if (uoff64[nblk]) HD_CUDA(cudaMemcpyAsync(U64.p, U_all, uoff64[nblk] * 8, cudaMemcpyHostToDevice, h->st));
  if (voff64[nblk]) HD_CUDA(cudaMemcpyAsync(V64.p, V_all, voff64[nblk] * 8, cudaMemcpyHostToDevice, h->st));
  HD_TRY(h->piv_sigma.alloc(std::max<int64_t>(h->total_rank, 1)));
  HD_TRY(h->piv_tau.alloc(std::max<int64_t>(h->total_rank, 1)));
  HD_CUDA(cudaMemsetAsync(h->piv_sigma.p, 0xff, std::max<int64_t>(h->total_rank, 1) * 4, h->st));
  HD_CUDA(cudaMemsetAsync(h->piv_tau.p, 0xff, std::max<int64_t>(h->total_rank, 1) * 4, h->st));
  HD_TRY(pack_factors(h, U64, V64, uoff64, voff64));
  HD_TRY(build_plan(h));
  HD_TRY(alloc_workspace(h));
  HD_CUDA(cudaStreamSynchronize(h->st));
  fill_stats(h);
  return HODLRDD_OK;
}

int hodlrdd_sync(hodlrdd_handle h) {
  if (!h) return HODLRDD_ERR_INVALID;
  int32_t code = 0;
  HD_TRY(read_error_word(h, &code));
  if (code != 0) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "a bounded device-side wait expired (code %d); the matvec output is invalid",
                  code);
    set_error(buf);
    HD_CUDA(cudaMemset(h->err.p, 0, sizeof(int32_t)));
    return HODLRDD_ERR_TIMEOUT;
  }
  return HODLRDD_OK;
}

int hodlrdd_set_profiling(hodlrdd_handle h, int on) {
  if (!h) return HODLRDD_ERR_INVALID;
  for (auto& v : h->ev_pending)
    for (cudaEvent_t e : v) {
      cudaEventSynchronize(e);
      h->ev_pool.push_back(e);
    }
  h->ev_pending.clear();
  for (double& m : h->prof_ms) m = 0.0;
  h->prof_chunks = 0;
  h->profiling = on != 0;
  return HODLRDD_OK;
}

int hodlrdd_get_profile(hodlrdd_handle h, double* ms, int64_t* chunks, int64_t* launches) {
  if (!h) return HODLRDD_ERR_INVALID;
  for (auto& v : h->ev_pending) {
    HD_CUDA(cudaEventSynchronize(v[4]));
    for (int i = 0; i < 4; ++i) {
      float t = 0.f;
      // with 7 events the near field ran on the aux stream between events 5 and 6
      if (i == 3 && v.size() == 7) HD_CUDA(cudaEventElapsedTime(&t, v[5], v[6]));
      else HD_CUDA(cudaEventElapsedTime(&t, v[i], v[i + 1]));
      h->prof_ms[i] += t;
    }
    h->prof_chunks += 1;
    for (cudaEvent_t e : v) h->ev_pool.push_back(e);
  }
  h->ev_pending.clear();
  if (ms)
    for (int i = 0; i < 4; ++i) ms[i] = h->prof_ms[i];
  if (chunks) *chunks = h->prof_chunks;
  if (launches) *launches = h->launches;
  return HODLRDD_OK;
}

// Test hook: caps the ACA's one-pass factor pool (bytes; -1 default).
int hodlrdd_debug_aca_pool_bytes(int64_t bytes) {
  g_aca_pool_cap.store(bytes < 0 ? -1 : bytes);
  return HODLRDD_OK;
}

// Test hook: make the k-th device allocation from now fail with
// HODLRDD_ERR_OOM; k < 0 disarms.
int hodlrdd_debug_fail_alloc_after(int64_t k) {
  debug_fail_alloc_after(k);
  return HODLRDD_OK;
}

}  // extern "C"
