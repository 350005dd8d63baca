// Batched products over many resident HODLRdD handles (uneven trees): a fixed
// set of requests is captured once into a CUDA graph, the requests spread over
// several streams inside it so that small trees run side by side, and each run
// replays the graph with one launch. Inputs and outputs pass through buffers the
// batch owns, so the graph's pointers stay fixed.
#include <algorithm>
#include <new>
#include <vector>

#include "internal.cuh"

struct hodlrdd_batch_s {
  std::vector<hodlrdd_s*> h;
  std::vector<int> nrhs;
  std::vector<size_t> bytes;          // per request: N * nrhs * element size
  std::vector<hd::DevBuf<char>> xin, yout;
  std::vector<cudaStream_t> lanes;    // capture-time streams
  std::vector<cudaEvent_t> ev;        // fork / join events of the capture
  cudaStream_t st = nullptr;          // capture origin
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace hd {
namespace {

constexpr int kBatchLanes = 8;

void batch_free(hodlrdd_batch_s* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  for (cudaStream_t s : b->lanes) cudaStreamDestroy(s);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

bool is_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int capture(hodlrdd_batch_s* b) {
  const int n = (int)b->h.size();
  const int lanes = std::min(kBatchLanes, n);
  // every handle applies once outside the capture first (kernel attributes,
  // lazily loaded device code), and must not be profiling
  for (int i = 0; i < n; ++i) {
    if (b->h[i]->profiling) {
      set_error("hodlrdd_batch_create: a handle has profiling on");
      return HODLRDD_ERR_INVALID;
    }
    HD_TRY(launch_matvec(b->h[i], b->xin[i].p, b->yout[i].p, b->nrhs[i], b->st));
  }
  HD_CUDA(cudaStreamSynchronize(b->st));
  for (int k = 0; k < lanes; ++k) {
    cudaStream_t s;
    HD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    b->lanes.push_back(s);
  }
  b->ev.resize(lanes + 1);
  for (cudaEvent_t& e : b->ev) HD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  HD_CUDA(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
  int rc = HODLRDD_OK;
  cudaError_t e = cudaEventRecord(b->ev[lanes], b->st);
  for (int k = 0; k < lanes && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->lanes[k], b->ev[lanes], 0);
  // larger trees first, round-robin over the lanes
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->bytes[a] > b->bytes[c]; });
  for (int r = 0; r < n && e == cudaSuccess && rc == HODLRDD_OK; ++r) {
    const int i = order[r];
    rc = launch_matvec(b->h[i], b->xin[i].p, b->yout[i].p, b->nrhs[i], b->lanes[r % lanes]);
  }
  for (int k = 0; k < lanes && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->ev[k], b->lanes[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->ev[k], 0);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(b->st, &g);
  b->graph = g;
  if (e != cudaSuccess) return cuda_fail(e, "batch capture", __FILE__, __LINE__);
  if (rc != HODLRDD_OK) return rc;
  if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture", __FILE__, __LINE__);
  HD_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return HODLRDD_OK;
}

}  // namespace
}  // namespace hd

using namespace hd;

extern "C" int hodlrdd_batch_create(const hodlrdd_handle* handles, const int* nrhs, int count,
                                    hodlrdd_batch* out) {
  if (!handles || !nrhs || count < 1 || !out) {
    set_error("hodlrdd_batch_create: NULL argument or count < 1");
    return HODLRDD_ERR_INVALID;
  }
  for (int i = 0; i < count; ++i) {
    if (!handles[i] || nrhs[i] < 1) {
      set_error("hodlrdd_batch_create: NULL handle or nrhs < 1");
      return HODLRDD_ERR_INVALID;
    }
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) {
        set_error("hodlrdd_batch_create: a handle appears twice (its workspace would be shared)");
        return HODLRDD_ERR_INVALID;
      }
  }
  hodlrdd_batch_s* b = new (std::nothrow) hodlrdd_batch_s();
  if (!b) return HODLRDD_ERR_OOM;
  int rc = HODLRDD_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
  if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamCreateWithFlags", __FILE__, __LINE__);
  b->xin.resize(count);
  b->yout.resize(count);
  for (int i = 0; i < count && rc == HODLRDD_OK; ++i) {
    hodlrdd_s* h = handles[i];
    b->h.push_back(h);
    b->nrhs.push_back(nrhs[i]);
    const size_t es = h->opt.precision == HODLRDD_PREC_FP64 ? 8 : 4;
    b->bytes.push_back((size_t)h->N * nrhs[i] * es);
    rc = b->xin[i].alloc(b->bytes.back());
    if (rc == HODLRDD_OK) rc = b->yout[i].alloc(b->bytes.back());
    if (rc == HODLRDD_OK && cudaMemset(b->xin[i].p, 0, b->bytes.back()) != cudaSuccess)
      rc = cuda_fail(cudaGetLastError(), "cudaMemset", __FILE__, __LINE__);
  }
  if (rc == HODLRDD_OK) rc = capture(b);
  if (rc != HODLRDD_OK) {
    batch_free(b);
    return rc;
  }
  *out = b;
  return HODLRDD_OK;
}

extern "C" int hodlrdd_batch_run(hodlrdd_batch b, const void* const* x, void* const* y, void* stream) {
  if (!b || !x || !y) {
    set_error("hodlrdd_batch_run: NULL argument");
    return HODLRDD_ERR_INVALID;
  }
  const int n = (int)b->h.size();
  for (int i = 0; i < n; ++i)
    if (!x[i] || !y[i]) {
      set_error("hodlrdd_batch_run: NULL x or y");
      return HODLRDD_ERR_INVALID;
    }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool host = false;
  for (int i = 0; i < n; ++i) {
    const bool xd = is_device(x[i]);
    host |= !xd;
    HD_CUDA(cudaMemcpyAsync(b->xin[i].p, x[i], b->bytes[i], xd ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            st));
  }
  HD_CUDA(cudaGraphLaunch(b->exec, st));
  for (int i = 0; i < n; ++i) {
    const bool yd = is_device(y[i]);
    host |= !yd;
    HD_CUDA(cudaMemcpyAsync(y[i], b->yout[i].p, b->bytes[i], yd ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            st));
  }
  if (host) HD_CUDA(cudaStreamSynchronize(st));
  return HODLRDD_OK;
}

extern "C" int hodlrdd_batch_destroy(hodlrdd_batch b) {
  if (b && b->st) cudaStreamSynchronize(b->st);
  batch_free(b);
  return HODLRDD_OK;
}
