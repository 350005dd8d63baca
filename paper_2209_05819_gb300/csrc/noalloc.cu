// y = K x for callers that must not allocate device memory.
//
// hodlrdd_matvec stages host right-hand sides and results through device
// buffers the handle grows on demand, so its first host call (and any call with
// more right-hand sides than before) runs cudaMalloc. Some callers cannot accept
// that: a serving loop whose device memory is reserved up front by another
// allocator (a later cudaMalloc fails or fragments the pool), or a latency-bound
// loop that cannot take the device-wide synchronisation cudaMalloc/cudaFree may
// imply. This entry point stages through a fixed scratch array in the library's
// static device memory instead; the matvec kernels themselves are the ones
// hodlrdd_matvec launches, on the handle's workspace, which the build allocated.
#include <mutex>

#include "internal.cuh"

namespace hd {
namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr size_t kScratchAlign = 256;
constexpr int kMaxDevices = 64;

// Staging area: x in [0, round_up(bytes_x)), y after it. Nothing in it needs to
// start at zero: the host-to-device copy writes every x element the kernels
// read, and the last near-field kernel writes every y element before the
// device-to-host copy reads it.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_scratch_mu;
char* g_scratch_ptr[kMaxDevices] = {};

// Set-up, once per device: the device address of g_scratch. The first lookup
// also makes the driver load this file's device module.
int scratch_on(int dev, char** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("hodlrdd_matvec_noalloc: device ordinal out of range");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
    }
    g_scratch_ptr[dev] = static_cast<char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return HODLRDD_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace
}  // namespace hd

using namespace hd;

extern "C" int hodlrdd_matvec_noalloc(hodlrdd_handle h, const void* x, void* y, int nrhs, void* stream) {
  if (!h || !x || !y || nrhs < 1) {
    set_error("hodlrdd_matvec_noalloc: NULL handle / pointer or nrhs < 1");
    return HODLRDD_ERR_INVALID;
  }
  if (h->profiling) {
    set_error("hodlrdd_matvec_noalloc: profiling creates events; turn it off for this call");
    return HODLRDD_ERR_INVALID;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t io = h->opt.precision == HODLRDD_PREC_FP64 ? 8 : 4;
  const size_t bytes = (size_t)h->N * nrhs * io;
  const char* xa = static_cast<const char*>(x);
  char* ya = static_cast<char*>(y);
  if (xa < ya + bytes && ya < xa + bytes) {
    set_error("hodlrdd_matvec_noalloc: x and y overlap");
    return HODLRDD_ERR_INVALID;
  }
  const bool xdev = on_device(x), ydev = on_device(y);
  const size_t need = (xdev ? 0 : round_up(bytes, kScratchAlign)) + (ydev ? 0 : bytes);
  if (need > kScratchBytes) {
    char buf[256];
    std::snprintf(buf, sizeof buf,
                  "hodlrdd_matvec_noalloc: staging needs %zu bytes (N=%lld, nrhs=%d, %zu-byte values, host x: %d, "
                  "host y: %d) but the static scratch holds %zu",
                  need, (long long)h->N, nrhs, io, (int)!xdev, (int)!ydev, kScratchBytes);
    set_error(buf);
    return HODLRDD_ERR_INVALID;
  }
  // the handle's kernels and workspace, and the scratch the staging uses, are
  // those of the device the handle was built on
  HD_TRY(check_device(h, "hodlrdd_matvec_noalloc"));
  if (xdev && ydev) return launch_matvec(h, x, y, nrhs, st);
  char* scratch = nullptr;
  HD_TRY(scratch_on(h->device, &scratch));
  const void* dx = x;
  void* dy = y;
  if (!xdev) {
    HD_CUDA(cudaMemcpyAsync(scratch, x, bytes, cudaMemcpyHostToDevice, st));
    dx = scratch;
  }
  if (!ydev) dy = scratch + (xdev ? 0 : round_up(bytes, kScratchAlign));
  int rc = launch_matvec(h, dx, dy, nrhs, st);
  if (rc == HODLRDD_OK && !ydev) {
    const cudaError_t e = cudaMemcpyAsync(y, dy, bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(y)", __FILE__, __LINE__);
  }
  // also when a launch failed: the copy from the caller's host x may still be
  // in flight, and the caller may free x as soon as this call returns
  const cudaError_t e = cudaStreamSynchronize(st);
  if (rc == HODLRDD_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
  return rc;
}
