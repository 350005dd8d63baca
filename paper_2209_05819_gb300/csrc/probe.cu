// Throughput probes of the arithmetic pipes the near field and the FP64 form
// are bound by: FP32 FMA, FP64 FMA, and the multi-function unit (MUFU) for
// rsqrt.approx and ex2.approx, timed with CUDA events on the caller's stream.
// They change no device setting; they only run enough independent dependency
// chains on every SM to keep each pipe busy, at whatever clock the GPU runs.
#include <algorithm>

#include "internal.cuh"

namespace hd {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;  // independent dependency chains per thread

// sink: written only when a chain ends at an impossible value, which keeps the
// arithmetic alive without a store per thread
__global__ void __launch_bounds__(kProbeThreads) k_probe_f32(int iters, float b, float c, float* sink) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.2345f) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_f64(int iters, double b, double c, double* sink) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (double)(threadIdx.x + i) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.2345) sink[0] = s;
}

__device__ __forceinline__ float mufu_rsqrt(float x) {
  float r;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float mufu_ex2(float x) {
  float r;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// x -> rsqrt(x) oscillates around 1; x -> 2^-x stays in (1/2, 1): no value
// leaves the normal range, so every step is one MUFU operation (plus, for ex2,
// the negation, which the FP32 pipe takes)
template <bool EX2>
__global__ void __launch_bounds__(kProbeThreads) k_probe_mufu(int iters, float* sink) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 0.5f + (float)(threadIdx.x + i) * 1e-4f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = EX2 ? mufu_ex2(-a[i]) : mufu_rsqrt(a[i]);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.2345f) sink[0] = s;
}

// Best of `reps` event-timed launches of f on st, in milliseconds.
template <class F>
int best_ms(cudaStream_t st, int reps, F&& f, float* out) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HD_CUDA(cudaEventCreate(&e0));
  const cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce, "cudaEventCreate", __FILE__, __LINE__);
  }
  float best = 1e30f;
  int rc = HODLRDD_OK;
  f();  // warm-up (module load, clocks)
  for (int r = 0; r < reps && rc == HODLRDD_OK; ++r) {
    cudaEventRecord(e0, st);
    f();
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "probe launch", __FILE__, __LINE__);
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *out = best;
  return rc;
}

}  // namespace
}  // namespace hd

using namespace hd;

extern "C" int hodlrdd_probe_peaks(double* out, int n, void* stream) {
  if (!out || n < 1) {
    set_error("hodlrdd_probe_peaks: NULL out or n < 1");
    return HODLRDD_ERR_INVALID;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  HD_CUDA(cudaGetDevice(&dev));
  HD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // eight CTAs of 256 threads per SM: 64 warps, the SM's full complement
  const int grid = sms * 8;
  const double threads = (double)grid * kProbeThreads;
  DevBuf<double> sink;
  HD_TRY(sink.alloc(2));
  float* fs = reinterpret_cast<float*>(sink.p);
  double vals[4] = {0, 0, 0, 0};
  float ms = 0.f;
  const int it32 = 16384, it64 = 512, itmu = 4096;
  HD_TRY(best_ms(st, 3, [&] { k_probe_f32<<<grid, kProbeThreads, 0, st>>>(it32, 0.999f, 1e-3f, fs); }, &ms));
  vals[0] = 2.0 * kChains * it32 * threads / (ms * 1e-3) / 1e12;
  HD_TRY(best_ms(st, 3, [&] { k_probe_f64<<<grid, kProbeThreads, 0, st>>>(it64, 0.999, 1e-3, sink.p); }, &ms));
  vals[1] = 2.0 * kChains * it64 * threads / (ms * 1e-3) / 1e12;
  HD_TRY(best_ms(st, 3, [&] { k_probe_mufu<false><<<grid, kProbeThreads, 0, st>>>(itmu, fs); }, &ms));
  vals[2] = (double)kChains * itmu * threads / (ms * 1e-3) / 1e9;
  HD_TRY(best_ms(st, 3, [&] { k_probe_mufu<true><<<grid, kProbeThreads, 0, st>>>(itmu, fs); }, &ms));
  vals[3] = (double)kChains * itmu * threads / (ms * 1e-3) / 1e9;
  for (int i = 0; i < std::min(n, 4); ++i) out[i] = vals[i];
  return HODLRDD_OK;
}
