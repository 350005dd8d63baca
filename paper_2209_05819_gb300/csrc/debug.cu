// Test entry for the bounded device-side waits: a kernel that waits on an
// mbarrier phase nothing completes, with the same bounded-wait pattern the
// panel kernels use (try_wait until a cycle limit, then record an error code
// in the handle's error word and return). hodlrdd_sync then reports
// HODLRDD_ERR_TIMEOUT and the context stays usable. It faults nothing: the
// wait ends by itself, and no copy or tensor-memory allocation is pending.
#include "internal.cuh"

namespace hd {
namespace {

__device__ __forceinline__ uint32_t smem32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__global__ void k_expire_wait(long long limit, int32_t* err, int code) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem32(&bar)), "r"(1) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem32(&bar)), "r"(0)
        : "memory");
    if (ok) return;  // not reached: nothing arrives on the barrier
    if (clock64() - t0 > limit) {
      atomicCAS(err, 0, code);
      return;
    }
  }
}

}  // namespace
}  // namespace hd

using namespace hd;

extern "C" int hodlrdd_debug_expire_wait(hodlrdd_handle h, long long cycles) {
  if (!h || !h->err.p || cycles < 0 || cycles > 8000000000LL) {
    set_error("hodlrdd_debug_expire_wait: NULL handle or cycles outside 0..8e9");
    return HODLRDD_ERR_INVALID;
  }
  k_expire_wait<<<1, 32, 0, h->st>>>(cycles, h->err.p, 99);
  HD_CUDA(cudaGetLastError());
  HD_CUDA(cudaStreamSynchronize(h->st));
  return HODLRDD_OK;
}
