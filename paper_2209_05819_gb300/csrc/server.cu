// A request loop over HODLRdD models kept resident under a device-memory
// budget: the serving side of the batched-trees use (many instances, uneven
// sizes, products and second-kind solves arriving over time).
//
// A model is a point set with its kernel and build options. It is built on its
// first request and stays resident; when the handles' device bytes exceed the
// budget, the least recently used idle models are destroyed (and rebuilt if
// asked for again). A solve request also keeps an FP64 twin of the model as the
// refinement operator. Worker threads (each with a high-priority CUDA stream
// for products and a low-priority one for solves) take queued
// products first (they are short) and solves otherwise, with at most
// workers - 1 solves at a time so that one worker stays free for products;
// each kind in arrival order. Products of different models run side by side,
// requests for one model run one at a time (its workspace). Every result
// equals the one the model's handle gives alone (the same kernels on the same
// data).
#include <chrono>
#include <condition_variable>
#include <deque>
#include <string>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace hd {
namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Model {
  std::vector<double> points;  // host copy, N x d row-major
  int d = 0;
  int64_t N = 0;
  int kid = 0;
  double prm[4] = {1.0, 0.0, 0.0, 0.0};
  int leaf = 0;
  double tol = 0.0;
  hodlrdd_options opt{};
  hodlrdd_s* h = nullptr;    // built on first use
  hodlrdd_s* h64 = nullptr;  // FP64 twin, built on the first solve (unless opt is FP64)
  int64_t bytes = 0;         // device bytes of h and h64
  int64_t last_bytes = 0;    // size when last resident (0: never built)
  uint64_t last_use = 0;
  int running = 0;           // requests past residency, running on it (never evicted meanwhile)
  std::mutex run;            // one request at a time on its workspace
};

struct Request {
  int64_t model = 0;
  int kind = 0;
  const void* x = nullptr;
  void* y = nullptr;
  int nrhs = 1;
  int status = HODLRDD_OK;
  std::string msg;  // the worker's error detail
  bool done = false;
  double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
};

int64_t handle_bytes(hodlrdd_s* h) {
  if (!h) return 0;
  hodlrdd_stats s;
  return hodlrdd_get_stats(h, &s) == HODLRDD_OK ? s.device_bytes : 0;
}

}  // namespace
}  // namespace hd

struct hodlrdd_server_s {
  int device = 0;
  int64_t budget = 0;
  std::vector<std::unique_ptr<hd::Model>> models;
  std::deque<int64_t> queue_mv, queue_sv;  // products, solves
  std::unordered_map<int64_t, hd::Request> reqs;
  std::mutex mu;  // models' residency fields, queue, requests, counters
  std::condition_variable cv_work, cv_done;
  std::mutex build_mu;  // one build at a time
  std::vector<std::thread> workers;
  bool stop = false;
  int64_t resident = 0, builds = 0, evictions = 0, next_id = 1;
  int64_t batches = 0, batched = 0;  // products run together: batches of two or more, their requests
  uint64_t tick = 0;
  int nworkers = 1, solves_running = 0;
  int batch_cols = 64;  // columns of one batched product (<= 1: no batching)
};

namespace hd {
namespace {

// Destroys least recently used models that no request is running on (other
// than keep) until the resident bytes fit the budget. Called with s->mu held,
// by the holder of s->build_mu only.
void evict_locked(hodlrdd_server_s* s, const Model* keep) {
  while (s->resident > s->budget) {
    Model* victim = nullptr;
    for (auto& m : s->models)
      if (m.get() != keep && (m->h || m->h64) && m->running == 0 && (!victim || m->last_use < victim->last_use))
        victim = m.get();
    if (!victim) return;
    if (victim->h) hodlrdd_destroy(victim->h);
    if (victim->h64) hodlrdd_destroy(victim->h64);
    victim->h = victim->h64 = nullptr;
    s->resident -= victim->bytes;
    victim->bytes = 0;
    s->evictions++;
  }
}

// Makes m resident (and its FP64 twin for a solve) and, on success, counts
// the caller as running on it (so that no build evicts it until it is done).
// Builds are serialised; a build that leaves the budget exceeded waits for
// running requests to finish and evicts their models, and fails with
// HODLRDD_ERR_OOM only when nothing else is left to evict.
int ensure(hodlrdd_server_s* s, Model& m, bool twin) {
  auto needs_locked = [&](bool& need_h, bool& need_64) {
    need_h = m.h == nullptr;
    need_64 = twin && m.opt.precision != HODLRDD_PREC_FP64 && m.h64 == nullptr;
    return need_h || need_64;
  };
  bool need_h = false, need_64 = false;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!needs_locked(need_h, need_64)) {  // resident: no wait on builds
      m.running++;
      return HODLRDD_OK;
    }
  }
  std::lock_guard<std::mutex> build(s->build_mu);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!needs_locked(need_h, need_64)) {
      m.running++;
      return HODLRDD_OK;
    }
    // room first, from the model's last known size when it was resident before
    const int64_t want = s->resident + (need_h ? m.last_bytes : 0);
    if (want > s->budget) {
      const int64_t saved = s->resident;
      s->resident = want;
      evict_locked(s, &m);
      s->resident -= want - saved;
    }
  }
  // each new handle is counted as soon as it exists, so that a failed build of
  // the twin leaves the model's first handle resident and accounted
  auto account_locked = [&] {
    const int64_t b = handle_bytes(m.h) + handle_bytes(m.h64);
    s->resident += b - m.bytes;
    m.bytes = m.last_bytes = b;
  };
  if (need_h) {
    hodlrdd_s* h = nullptr;
    HD_TRY(hodlrdd_build_ex(m.points.data(), m.d, m.N, m.kid, m.prm, m.leaf, m.tol, &m.opt, &h));
    std::lock_guard<std::mutex> lk(s->mu);
    m.h = h;
    s->builds++;
    account_locked();
  }
  if (need_64) {
    hodlrdd_options o64 = m.opt;
    o64.precision = HODLRDD_PREC_FP64;
    o64.lowrank_form = 0;
    // the refinement operator: float-float near field where it exists
    o64.fp64_near = m.d <= 4 && m.kid != HODLRDD_K_SIN ? 1 : 0;
    hodlrdd_s* h = nullptr;
    HD_TRY(hodlrdd_build_ex(m.points.data(), m.d, m.N, m.kid, m.prm, m.leaf, m.tol, &o64, &h));
    std::lock_guard<std::mutex> lk(s->mu);
    m.h64 = h;
    s->builds++;
    account_locked();
  }
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    evict_locked(s, &m);
    if (s->resident <= s->budget) {
      m.running++;
      return HODLRDD_OK;
    }
    // wait while any request runs, on another model (it becomes evictable when
    // done) or on this one (its handles cannot be destroyed under its kernels)
    bool busy = false;
    for (auto& o : s->models) busy |= o->running > 0;
    if (!busy) break;
    s->cv_done.wait(lk);
  }
  // the model alone does not fit, and nothing runs on it: do not keep it
  if (m.h) hodlrdd_destroy(m.h);
  if (m.h64) hodlrdd_destroy(m.h64);
  m.h = m.h64 = nullptr;
  s->resident -= m.bytes;
  m.bytes = 0;
  set_error("hodlrdd_server: the model does not fit the device-memory budget");
  return HODLRDD_ERR_OOM;
}

// Device staging of one worker for solves and batched products (grown on demand).
struct Staging {
  DevBuf<double> b, x;
  DevBuf<float> xc, yc;  // batched products: N x columns, row-major
  int grow(int64_t n) {
    if ((int64_t)b.n < n) HD_TRY(b.alloc(n));
    if ((int64_t)x.n < n) HD_TRY(x.alloc(n));
    return HODLRDD_OK;
  }
  int grow_batch(int64_t n) {
    if ((int64_t)xc.n < n) HD_TRY(xc.alloc(n));
    if ((int64_t)yc.n < n) HD_TRY(yc.alloc(n));
    return HODLRDD_OK;
  }
};



// The handle's bounded-wait error word after a product on st (already
// synchronised), read and cleared on st: hodlrdd_sync would synchronise the
// whole device, i.e. wait for every other worker's requests.
int check_waits(hodlrdd_s* h, cudaStream_t st) {
  int32_t code = 0;
  HD_TRY(take_error_word(h, st, &code));
  if (code == 0) return HODLRDD_OK;
  set_error("a bounded device-side wait expired; the product is invalid");
  return HODLRDD_ERR_TIMEOUT;
}

// Products of one model that were queued together, as one product over their
// columns side by side: x_i into columns [c_i, c_i + nrhs_i) of one N x C
// array, one hodlrdd_matvec, the columns back into y_i (2-D copies, host or
// device buffers). FP32-I/O forms only (their results stay within the FP32
// chunk bound of the single products; FP64 models run their products alone).
int run_batch(Model& m, const std::vector<Request>& rs, cudaStream_t st, Staging& sg) {
  std::lock_guard<std::mutex> one(m.run);
  int64_t C = 0;
  for (const Request& r : rs) C += r.nrhs;
  HD_TRY(sg.grow_batch(m.N * C));
  const size_t es = sizeof(float);
  int64_t c0 = 0;
  for (const Request& r : rs) {
    HD_CUDA(cudaMemcpy2DAsync(sg.xc.p + c0, C * es, r.x, r.nrhs * es, r.nrhs * es, m.N, cudaMemcpyDefault, st));
    c0 += r.nrhs;
  }
  HD_TRY(hodlrdd_matvec(m.h, sg.xc.p, sg.yc.p, (int)C, st));
  c0 = 0;
  for (const Request& r : rs) {
    HD_CUDA(cudaMemcpy2DAsync(r.y, r.nrhs * es, sg.yc.p + c0, C * es, r.nrhs * es, m.N, cudaMemcpyDefault, st));
    c0 += r.nrhs;
  }
  HD_CUDA(cudaStreamSynchronize(st));
  return check_waits(m.h, st);
}

int run_request(Model& m, const Request& r, cudaStream_t st, Staging& sg) {
  std::lock_guard<std::mutex> one(m.run);
  if (r.kind == HODLRDD_REQ_MATVEC) {
    HD_TRY(hodlrdd_matvec(m.h, r.x, r.y, r.nrhs, st));
    HD_CUDA(cudaStreamSynchronize(st));
    return check_waits(m.h, st);
  }
  // solve, one right-hand side per column, FP64 b and x on the host
  hodlrdd_s* outer = m.opt.precision == HODLRDD_PREC_FP64 ? m.h : m.h64;
  HD_TRY(sg.grow(m.N));
  const double* b = static_cast<const double*>(r.x);
  double* x = static_cast<double*>(r.y);
  std::vector<double> col(m.N);
  for (int c = 0; c < r.nrhs; ++c) {
    for (int64_t i = 0; i < m.N; ++i) col[i] = b[i * r.nrhs + c];
    HD_CUDA(cudaMemcpyAsync(sg.b.p, col.data(), m.N * sizeof(double), cudaMemcpyHostToDevice, st));
    HD_TRY(hodlrdd_solve(m.h, outer, sg.b.p, sg.x.p, nullptr, nullptr, st));
    HD_CUDA(cudaMemcpyAsync(col.data(), sg.x.p, m.N * sizeof(double), cudaMemcpyDeviceToHost, st));
    HD_CUDA(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < m.N; ++i) x[i * r.nrhs + c] = col[i];
  }
  return HODLRDD_OK;
}

void worker(hodlrdd_server_s* s) {
  cudaSetDevice(s->device);
  // products on a high-priority stream, so that their CTAs are placed ahead of
  // the long solves' as SMs free up; solves on a low-priority one
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  cudaStream_t st_mv = nullptr, st_sv = nullptr;
  const bool have_stream = cudaStreamCreateWithPriority(&st_mv, cudaStreamNonBlocking, hi) == cudaSuccess &&
                           cudaStreamCreateWithPriority(&st_sv, cudaStreamNonBlocking, lo) == cudaSuccess;
  Staging sg;
  for (;;) {
    int64_t id = 0;
    Model* m = nullptr;
    Request r;
    std::vector<int64_t> batch;  // further products of the same model, run with r
    std::vector<Request> rs;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      const int max_solves = s->nworkers > 1 ? s->nworkers - 1 : 1;
      auto ready = [&] { return !s->queue_mv.empty() || (!s->queue_sv.empty() && s->solves_running < max_solves); };
      s->cv_work.wait(lk, [&] { return ready() || (s->stop && s->queue_mv.empty() && s->queue_sv.empty()); });
      if (!ready()) break;  // stopping, nothing left
      if (!s->queue_mv.empty()) {
        id = s->queue_mv.front();
        s->queue_mv.pop_front();
      } else {
        id = s->queue_sv.front();
        s->queue_sv.pop_front();
        s->solves_running++;
      }
      Request& q = s->reqs[id];
      q.t_start = now_ms();
      r = q;
      m = s->models[(size_t)r.model].get();
      m->last_use = ++s->tick;
      // continuous batching: products of the same model queued meanwhile join
      // this one, up to batch_cols columns (FP32-I/O forms with stored factors)
      if (r.kind == HODLRDD_REQ_MATVEC && s->batch_cols > 1 && m->opt.precision != HODLRDD_PREC_FP64 &&
          m->opt.lowrank_form == 0) {
        int64_t cols = r.nrhs;
        for (auto it = s->queue_mv.begin(); it != s->queue_mv.end();) {
          Request& q2 = s->reqs[*it];
          if (q2.model == r.model && cols + q2.nrhs <= s->batch_cols) {
            cols += q2.nrhs;
            q2.t_start = q.t_start;
            batch.push_back(*it);
            it = s->queue_mv.erase(it);
          } else {
            ++it;
          }
        }
        if (!batch.empty()) {
          rs.push_back(r);
          for (int64_t b : batch) rs.push_back(s->reqs[b]);
          s->batches += 1;
          s->batched += (int64_t)rs.size();
        }
      }
    }
    int rc = have_stream ? ensure(s, *m, r.kind == HODLRDD_REQ_SOLVE) : HODLRDD_ERR_CUDA;
    const bool ran = rc == HODLRDD_OK;
    if (ran) {
      if (!rs.empty()) rc = run_batch(*m, rs, st_mv, sg);
      else rc = run_request(*m, r, r.kind == HODLRDD_REQ_SOLVE ? st_sv : st_mv, sg);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (ran) m->running--;
      m->last_use = ++s->tick;
      const std::string msg = rc != HODLRDD_OK ? std::string(hodlrdd_last_error()) : std::string();
      batch.push_back(id);
      const double t_done = now_ms();
      for (int64_t b : batch) {
        Request& q = s->reqs[b];
        q.status = rc;
        if (rc != HODLRDD_OK) q.msg = msg;
        q.done = true;
        q.t_done = t_done;
      }
      if (r.kind == HODLRDD_REQ_SOLVE) s->solves_running--;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();  // a solve slot may have opened
  }
  if (st_mv) cudaStreamDestroy(st_mv);
  if (st_sv) cudaStreamDestroy(st_sv);
}

}  // namespace
}  // namespace hd

using namespace hd;

extern "C" int hodlrdd_server_create(int64_t budget_bytes, int workers, hodlrdd_server* out) {
  if (!out || budget_bytes <= 0 || workers < 1 || workers > 64) {
    set_error("hodlrdd_server_create: NULL out, budget <= 0 or workers outside 1..64");
    return HODLRDD_ERR_INVALID;
  }
  hodlrdd_server_s* s = new (std::nothrow) hodlrdd_server_s();
  if (!s) return HODLRDD_ERR_OOM;
  HD_CUDA(cudaGetDevice(&s->device));
  s->budget = budget_bytes;
  s->nworkers = workers;
  for (int i = 0; i < workers; ++i) s->workers.emplace_back(worker, s);
  *out = s;
  return HODLRDD_OK;
}

extern "C" int hodlrdd_server_add(hodlrdd_server s, const double* points, int d, int64_t N, int kernel_id,
                                  const double* kernel_params, int leaf_size, double tol,
                                  const hodlrdd_options* opt, int64_t* model_id) {
  if (!s || !points || !model_id || d < 1 || d > kMaxDim || N < 1 || leaf_size < 1 || !(tol > 0.0)) {
    set_error("hodlrdd_server_add: invalid argument");
    return HODLRDD_ERR_INVALID;
  }
  std::unique_ptr<Model> m(new (std::nothrow) Model());
  if (!m) return HODLRDD_ERR_OOM;
  m->points.assign(points, points + N * d);
  m->d = d;
  m->N = N;
  m->kid = kernel_id;
  if (kernel_params)
    for (int k = 0; k < 4; ++k) m->prm[k] = kernel_params[k];
  m->leaf = leaf_size;
  m->tol = tol;
  hodlrdd_options_default(&m->opt);
  if (opt) m->opt = *opt;
  std::lock_guard<std::mutex> lk(s->mu);
  *model_id = (int64_t)s->models.size();
  s->models.push_back(std::move(m));
  return HODLRDD_OK;
}

extern "C" int hodlrdd_server_submit(hodlrdd_server s, int64_t model_id, int kind, const void* x, void* y, int nrhs,
                                     int64_t* request_id) {
  if (!s || !x || !y || !request_id || nrhs < 1 || (kind != HODLRDD_REQ_MATVEC && kind != HODLRDD_REQ_SOLVE)) {
    set_error("hodlrdd_server_submit: invalid argument");
    return HODLRDD_ERR_INVALID;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (model_id < 0 || model_id >= (int64_t)s->models.size()) {
      set_error("hodlrdd_server_submit: unknown model");
      return HODLRDD_ERR_INVALID;
    }
    const int64_t id = s->next_id++;
    Request& r = s->reqs[id];
    r.model = model_id;
    r.kind = kind;
    r.x = x;
    r.y = y;
    r.nrhs = nrhs;
    r.t_submit = now_ms();
    (kind == HODLRDD_REQ_SOLVE ? s->queue_sv : s->queue_mv).push_back(id);
    *request_id = id;
  }
  s->cv_work.notify_all();
  return HODLRDD_OK;
}

extern "C" int hodlrdd_server_wait(hodlrdd_server s, int64_t request_id, double* latency_ms) {
  if (!s) return HODLRDD_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) {
    set_error("hodlrdd_server_wait: unknown request");
    return HODLRDD_ERR_INVALID;
  }
  s->cv_done.wait(lk, [&] { return it->second.done; });
  const int rc = it->second.status;
  if (rc != HODLRDD_OK) set_error(it->second.msg);  // the detail, on the caller's thread
  if (latency_ms) {
    latency_ms[0] = it->second.t_done - it->second.t_submit;
    latency_ms[1] = it->second.t_done - it->second.t_start;
  }
  s->reqs.erase(it);
  return rc;
}

extern "C" int hodlrdd_server_stats(hodlrdd_server s, int64_t* out) {
  if (!s || !out) return HODLRDD_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  int64_t res_models = 0;
  for (auto& m : s->models) res_models += (m->h || m->h64) ? 1 : 0;
  out[0] = s->resident;
  out[1] = res_models;
  out[2] = s->builds;
  out[3] = s->evictions;
  out[4] = (int64_t)(s->queue_mv.size() + s->queue_sv.size());
  return HODLRDD_OK;
}

extern "C" int hodlrdd_server_set_batching(hodlrdd_server s, int max_cols) {
  if (!s || max_cols < 0) {
    set_error("hodlrdd_server_set_batching: NULL server or max_cols < 0");
    return HODLRDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->batch_cols = max_cols;
  return HODLRDD_OK;
}

extern "C" int hodlrdd_server_batch_stats(hodlrdd_server s, int64_t* out) {
  if (!s || !out) return HODLRDD_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  out[0] = s->batches;
  out[1] = s->batched;
  return HODLRDD_OK;
}

extern "C" int hodlrdd_server_destroy(hodlrdd_server s) {
  if (!s) return HODLRDD_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& m : s->models) {
    if (m->h) hodlrdd_destroy(m->h);
    if (m->h64) hodlrdd_destroy(m->h64);
  }
  delete s;
  return HODLRDD_OK;
}
