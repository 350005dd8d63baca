// Solve K x = b with GMRES on a fast (FP32 / 16-bit) HODLRdD operator inside
// iterative refinement with the FP64 operator: the integral-equation use of the
// hierarchical product (the second-kind system (I + K/N) u = b of the paper's
// numerical experiments). Vector work runs in the kernels below; the small
// Hessenberg least-squares problem (at most `restart` columns) is solved on the
// host between them.
//
// Reading taken where the paper is silent: x0 = 0, relative residual
// ||b - K x||_2 / ||b||_2 of the FP64 operator as the stopping test, GMRES(m)
// with m = 50 by default, classical Gram-Schmidt applied twice.
#include <algorithm>
#include <cmath>
#include <vector>

#include <memory>
#include <new>

#include "internal.cuh"

namespace hd {
namespace {

constexpr int kDotThreads = 256;
constexpr int kDotBlocks = 256;  // fixed, so the reduction order does not depend on the device

// part[blk * nc + j] = sum over rows of this block's grid-stride range of V[:, j] . w
// (V column-major with leading dimension ld); FP64 accumulation.
template <class T>
__global__ void __launch_bounds__(kDotThreads) k_dots(const T* __restrict__ V, int64_t ld, int nc,
                                                     const T* __restrict__ w, int64_t N, double* __restrict__ part) {
  __shared__ double red[kDotThreads];
  for (int j = 0; j < nc; ++j) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kDotThreads + threadIdx.x; i < N; i += (int64_t)kDotBlocks * kDotThreads)
      s += (double)V[(int64_t)j * ld + i] * (double)w[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kDotThreads / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * nc + j] = red[0];
    __syncthreads();
  }
}

// out[j] = sum over blocks of part[blk * nc + j], in block order.
__global__ void k_dots_sum(const double* __restrict__ part, int nc, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nc) return;
  double s = 0.0;
  for (int b = 0; b < kDotBlocks; ++b) s += part[(int64_t)b * nc + j];
  out[j] = s;
}

// w[i] -= sum_j V[i, j] c[j]
template <class T>
__global__ void k_sub_combination(const T* __restrict__ V, int64_t ld, int nc, const double* __restrict__ c,
                                  T* __restrict__ w, int64_t N) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < nc; ++j) s += (double)V[(int64_t)j * ld + i] * c[j];
    w[i] = (T)((double)w[i] - s);
  }
}

// out[i] = a * p[i] + b * q[i] (out may alias p or q), converting types.
template <class TO, class TP, class TQ>
__global__ void k_axpby(int64_t N, double a, const TP* __restrict__ p, double b, const TQ* __restrict__ q,
                        TO* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)(a * (double)p[i] + (q ? b * (double)q[i] : 0.0));
}

int grid_for(int64_t N) { return (int)std::min<int64_t>((N + 255) / 256, 4096); }

// Device scratch of one solve.
template <class T>
struct Work {
  DevBuf<T> V;         // Krylov basis, N x (m + 1)
  DevBuf<T> w;         // N
  DevBuf<double> part; // kDotBlocks x (m + 1)
  DevBuf<double> c;    // m + 1
};

// dots[j] = V[:, j] . w for j < nc (copied to the host).
template <class T>
int dots(Work<T>& W, int64_t ld, int nc, const T* w, int64_t N, std::vector<double>& out, cudaStream_t st) {
  k_dots<T><<<kDotBlocks, kDotThreads, 0, st>>>(W.V.p, ld, nc, w, N, W.part.p);
  k_dots_sum<<<(nc + 127) / 128, 128, 0, st>>>(W.part.p, nc, W.c.p);
  HD_CUDA(cudaGetLastError());
  out.resize(nc);
  HD_CUDA(cudaMemcpyAsync(out.data(), W.c.p, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
  HD_CUDA(cudaStreamSynchronize(st));
  return HODLRDD_OK;
}

// ||v||_2 of a device vector through the dot kernels (v as a one-column basis).
template <class T>
int norm2(const T* v, int64_t N, DevBuf<double>& part, DevBuf<double>& c, double* out, cudaStream_t st) {
  k_dots<T><<<kDotBlocks, kDotThreads, 0, st>>>(v, N, 1, v, N, part.p);
  k_dots_sum<<<1, 128, 0, st>>>(part.p, 1, c.p);
  HD_CUDA(cudaGetLastError());
  double s = 0.0;
  HD_CUDA(cudaMemcpyAsync(&s, c.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  HD_CUDA(cudaStreamSynchronize(st));
  *out = std::sqrt(std::max(s, 0.0));
  return HODLRDD_OK;
}

// Inner GMRES(m) on the fast operator: d ~ A^{-1} r in precision T (FP32 for
// 16-bit and FP32 handles, FP64 for FP64 handles), to a relative residual
// reduction of tol_in or max_it matvecs. d is overwritten.
template <class T>
int gmres(hodlrdd_s* A, const T* r, T* d, int64_t N, int m, double tol_in, int max_it, Work<T>& W,
          int* iters, cudaStream_t st) {
  const int64_t ld = N;
  const int grid = grid_for(N);
  HD_CUDA(cudaMemsetAsync(d, 0, N * sizeof(T), st));
  double beta0 = 0.0;
  HD_TRY(norm2<T>(r, N, W.part, W.c, &beta0, st));
  if (beta0 == 0.0) return HODLRDD_OK;
  int it = 0;
  // residual of the current d: starts as r
  HD_CUDA(cudaMemcpyAsync(W.w.p, r, N * sizeof(T), cudaMemcpyDeviceToDevice, st));
  double beta = beta0;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), h1, h2;
  while (it < max_it) {
    // v_0 = residual / beta
    k_axpby<T, T, T><<<grid, 256, 0, st>>>(N, 1.0 / beta, W.w.p, 0.0, (const T*)nullptr, W.V.p);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    bool done = false;
    for (; k < m && it < max_it; ++k, ++it) {
      T* vk = W.V.p + (int64_t)k * ld;
      T* vn = W.V.p + (int64_t)(k + 1) * ld;
      HD_TRY(launch_matvec(A, vk, vn, 1, st));
      // classical Gram-Schmidt, twice
      HD_TRY(dots<T>(W, ld, k + 1, vn, N, h1, st));
      HD_CUDA(cudaMemcpyAsync(W.c.p, h1.data(), (k + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
      k_sub_combination<T><<<grid, 256, 0, st>>>(W.V.p, ld, k + 1, W.c.p, vn, N);
      HD_TRY(dots<T>(W, ld, k + 1, vn, N, h2, st));
      HD_CUDA(cudaMemcpyAsync(W.c.p, h2.data(), (k + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
      k_sub_combination<T><<<grid, 256, 0, st>>>(W.V.p, ld, k + 1, W.c.p, vn, N);
      double hn = 0.0;
      HD_TRY(norm2<T>(vn, N, W.part, W.c, &hn, st));
      for (int j = 0; j <= k; ++j) H[(size_t)j * m + k] = h1[j] + h2[j];
      H[(size_t)(k + 1) * m + k] = hn;
      if (hn > 0.0) k_axpby<T, T, T><<<grid, 256, 0, st>>>(N, 1.0 / hn, vn, 0.0, (const T*)nullptr, vn);
      // Givens rotations on column k
      for (int j = 0; j < k; ++j) {
        const double a = H[(size_t)j * m + k], b = H[(size_t)(j + 1) * m + k];
        H[(size_t)j * m + k] = cs[j] * a + sn[j] * b;
        H[(size_t)(j + 1) * m + k] = -sn[j] * a + cs[j] * b;
      }
      const double a = H[(size_t)k * m + k], b = H[(size_t)(k + 1) * m + k];
      const double rr = std::hypot(a, b);
      cs[k] = rr > 0.0 ? a / rr : 1.0;
      sn[k] = rr > 0.0 ? b / rr : 0.0;
      H[(size_t)k * m + k] = rr;
      H[(size_t)(k + 1) * m + k] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      if (std::fabs(g[k + 1]) <= tol_in * beta0 || hn == 0.0) {
        ++k;
        ++it;
        done = true;
        break;
      }
    }
    // y = H(0:k, 0:k)^{-1} g(0:k); d += V(:, 0:k) y
    std::vector<double> y(k, 0.0);
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int j = i + 1; j < k; ++j) s -= H[(size_t)i * m + j] * y[j];
      y[i] = H[(size_t)i * m + i] != 0.0 ? s / H[(size_t)i * m + i] : 0.0;
    }
    for (double& v : y) v = -v;  // k_sub_combination subtracts
    HD_CUDA(cudaMemcpyAsync(W.c.p, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, st));
    k_sub_combination<T><<<grid, 256, 0, st>>>(W.V.p, ld, k, W.c.p, d, N);
    HD_CUDA(cudaGetLastError());
    if (done || it >= max_it) break;
    // restart from the true residual of the fast operator: w = r - A d
    HD_TRY(launch_matvec(A, d, W.w.p, 1, st));
    k_axpby<T, T, T><<<grid, 256, 0, st>>>(N, 1.0, r, -1.0, W.w.p, W.w.p);
    HD_TRY(norm2<T>(W.w.p, N, W.part, W.c, &beta, st));
    if (beta <= tol_in * beta0) break;
  }
  *iters += it;
  return HODLRDD_OK;
}

// Solver scratch kept in the inner handle between solves (grown on demand), so
// that repeated solves allocate nothing: a cudaMalloc / cudaFree per solve would
// synchronise the device under every other stream's work.
template <class T>
struct SolveScratch {
  Work<T> W;
  DevBuf<T> r_in, d_in;
  DevBuf<double> r, y;
  int64_t N = 0;
  int m = 0;
  int fit(int64_t n, int mm) {
    if (n <= N && mm <= m) return HODLRDD_OK;
    N = std::max(N, n);
    m = std::max(m, mm);
    HD_TRY(W.V.alloc((size_t)N * (m + 1)));
    HD_TRY(W.w.alloc(N));
    HD_TRY(W.part.alloc((size_t)kDotBlocks * (m + 1)));
    HD_TRY(W.c.alloc(m + 1));
    HD_TRY(r_in.alloc(N));
    HD_TRY(d_in.alloc(N));
    HD_TRY(r.alloc(N));
    HD_TRY(y.alloc(N));
    return HODLRDD_OK;
  }
};

template <class T>
int solve_typed(hodlrdd_s* inner, hodlrdd_s* outer, const double* b, double* x, const hodlrdd_solve_options& o,
                hodlrdd_solve_stats* stats, cudaStream_t st) {
  const int64_t N = outer->N;
  const int m = o.restart;
  const int grid = grid_for(N);
  if (!inner->solve_scratch || inner->solve_scratch_f64 != std::is_same<T, double>::value) {
    inner->solve_scratch = std::shared_ptr<void>(new (std::nothrow) SolveScratch<T>(),
                                                 [](void* p) { delete static_cast<SolveScratch<T>*>(p); });
    inner->solve_scratch_f64 = std::is_same<T, double>::value;
    if (!inner->solve_scratch) return HODLRDD_ERR_OOM;
  }
  SolveScratch<T>& S = *static_cast<SolveScratch<T>*>(inner->solve_scratch.get());
  HD_TRY(S.fit(N, m));
  Work<T>& W = S.W;
  DevBuf<T>& r_in = S.r_in;
  DevBuf<T>& d_in = S.d_in;
  DevBuf<double>& r = S.r;
  DevBuf<double>& y = S.y;
  HD_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), st));
  double bnorm = 0.0, rnorm = 0.0;
  HD_TRY(norm2<double>(b, N, W.part, W.c, &bnorm, st));
  HD_CUDA(cudaMemcpyAsync(r.p, b, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  rnorm = bnorm;
  int refine = 0, iters = 0;
  while (bnorm > 0.0 && rnorm > o.tol * bnorm && refine < o.max_refine) {
    // inner solve on the fast operator: A d = r (r scaled to unit norm)
    k_axpby<T, double, double><<<grid, 256, 0, st>>>(N, 1.0 / rnorm, r.p, 0.0, (const double*)nullptr, r_in.p);
    HD_TRY(gmres<T>(inner, r_in.p, d_in.p, N, m, o.inner_tol, o.max_inner_iters, W, &iters, st));
    // x += rnorm * d; r = b - K x with the FP64 operator
    k_axpby<double, double, T><<<grid, 256, 0, st>>>(N, 1.0, x, rnorm, d_in.p, x);
    HD_TRY(launch_matvec(outer, x, y.p, 1, st));
    k_axpby<double, double, double><<<grid, 256, 0, st>>>(N, 1.0, b, -1.0, y.p, r.p);
    HD_CUDA(cudaGetLastError());
    HD_TRY(norm2<double>(r.p, N, W.part, W.c, &rnorm, st));
    ++refine;
  }
  if (stats) {
    stats->refinements = refine;
    stats->inner_iterations = iters;
    stats->residual = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  }
  HD_CUDA(cudaStreamSynchronize(st));
  // a bounded wait that expired in any product of this solve makes its
  // residuals and iterate invalid: report that before the convergence test
  int32_t code_in = 0, code_out = 0;
  HD_TRY(take_error_word(inner, st, &code_in));
  if (outer != inner) HD_TRY(take_error_word(outer, st, &code_out));
  if (code_in != 0 || code_out != 0) {
    set_error("hodlrdd_solve: a bounded device-side wait expired in a product; x is invalid");
    return HODLRDD_ERR_TIMEOUT;
  }
  if (bnorm > 0.0 && rnorm > o.tol * bnorm) {
    set_error("hodlrdd_solve: tolerance not reached within max_refine refinement steps");
    return HODLRDD_ERR_NUMERIC;
  }
  return HODLRDD_OK;
}

}  // namespace
}  // namespace hd

using namespace hd;

extern "C" int hodlrdd_solve_options_default(hodlrdd_solve_options* o) {
  if (!o) return HODLRDD_ERR_INVALID;
  *o = hodlrdd_solve_options{};
  o->tol = 1e-10;
  o->inner_tol = 1e-5;
  o->restart = 50;
  o->max_inner_iters = 500;
  o->max_refine = 20;
  return HODLRDD_OK;
}

extern "C" int hodlrdd_solve(hodlrdd_handle inner, hodlrdd_handle outer, const double* b, double* x,
                             const hodlrdd_solve_options* opt, hodlrdd_solve_stats* stats, void* stream) {
  if (!inner || !outer || !b || !x) {
    set_error("hodlrdd_solve: NULL handle or pointer");
    return HODLRDD_ERR_INVALID;
  }
  hodlrdd_solve_options o;
  hodlrdd_solve_options_default(&o);
  if (opt) o = *opt;
  if (!(o.tol > 0.0) || !(o.inner_tol > 0.0) || o.restart < 1 || o.restart > 1000 || o.max_inner_iters < 1 ||
      o.max_refine < 1) {
    set_error("hodlrdd_solve: tol, inner_tol > 0; 1 <= restart <= 1000; max_inner_iters, max_refine >= 1");
    return HODLRDD_ERR_INVALID;
  }
  if (inner->N != outer->N || inner->d != outer->d) {
    set_error("hodlrdd_solve: inner and outer handles must describe the same points");
    return HODLRDD_ERR_INVALID;
  }
  if (outer->opt.precision != HODLRDD_PREC_FP64) {
    set_error("hodlrdd_solve: the outer (refinement) handle must be FP64");
    return HODLRDD_ERR_INVALID;
  }
  const size_t bytes = (size_t)outer->N * sizeof(double);
  const char* ba = reinterpret_cast<const char*>(b);
  const char* xa = reinterpret_cast<const char*>(x);
  if (ba < xa + bytes && xa < ba + bytes) {
    set_error("hodlrdd_solve: b and x overlap");
    return HODLRDD_ERR_INVALID;
  }
  cudaPointerAttributes pa{}, px{};
  if (cudaPointerGetAttributes(&pa, b) != cudaSuccess || cudaPointerGetAttributes(&px, x) != cudaSuccess ||
      pa.type != cudaMemoryTypeDevice || px.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    set_error("hodlrdd_solve: b and x must be device memory");
    return HODLRDD_ERR_INVALID;
  }
  HD_TRY(check_device(inner, "hodlrdd_solve"));
  HD_TRY(check_device(outer, "hodlrdd_solve"));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (inner->opt.precision == HODLRDD_PREC_FP64) return solve_typed<double>(inner, outer, b, x, o, stats, st);
  return solve_typed<float>(inner, outer, b, x, o, stats, st);
}
