// Solve K x = b with GMRES on a fast (FP32 / 16-bit) HODLRdD operator inside
// iterative refinement with the FP64 operator: the integral-equation use of the
// hierarchical product (the second-kind system (I + K/N) u = b of the paper's
// numerical experiments). Everything of a GMRES cycle runs on the device: the
// Arnoldi step (product, two Gram-Schmidt passes, normalisation) and the
// Hessenberg column's Givens update with the convergence test are one CUDA
// graph body under a conditional WHILE node, which the update kernel stops;
// the triangular solve and the update of the iterate follow in the same graph.
// The host launches one graph per restart cycle and reads the step count and
// residual once per cycle.
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

// State of one GMRES cycle on the device. sc: beta0, beta, ||w||^2 of the
// step, tol; hd: k (columns done), it (steps of this solve), max_it, converged.
struct GmState {
  double* H;   // (m + 1) x m, row-major with row stride m
  double* cs;  // m
  double* sn;  // m
  double* g;   // m + 1
  double* y;   // m
  double* h1;  // m + 1: first Gram-Schmidt coefficients of the step
  double* h2;  // m + 1: second
  double* sc;  // 4
  int* hd;     // 4
  int m;
};

// part[blk * (m + 1) + j] = this block's share of V[:, j] . w for j < k + add.
template <class T>
__global__ void __launch_bounds__(kDotThreads) k_gm_dots(const T* __restrict__ V, int64_t ld, GmState G, int add,
                                                        const T* __restrict__ w, int64_t N,
                                                        double* __restrict__ part) {
  __shared__ double red[kDotThreads];
  const int nc = G.hd[0] + add;
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
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * (G.m + 1) + j] = red[0];
    __syncthreads();
  }
}

// out[j] = sum over blocks of part[blk * (m + 1) + j], in block order, j < k + add.
__global__ void k_gm_dots_sum(const double* __restrict__ part, GmState G, int add, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= G.hd[0] + add) return;
  double s = 0.0;
  for (int b = 0; b < kDotBlocks; ++b) s += part[(int64_t)b * (G.m + 1) + j];
  out[j] = s;
}

// w[i] -= sum_{j < k + add} V[i, j] c[j]
template <class T>
__global__ void k_gm_sub(const T* __restrict__ V, int64_t ld, GmState G, int add, const double* __restrict__ c,
                         T* __restrict__ w, int64_t N) {
  const int nc = G.hd[0] + add;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < nc; ++j) s += (double)V[(int64_t)j * ld + i] * c[j];
    w[i] = (T)((double)w[i] - s);
  }
}

// Start of a cycle: beta = ||w|| from its squared norm, g = beta e_1, k = 0.
__global__ void k_gm_begin(GmState G, const double* __restrict__ w2) {
  if (threadIdx.x != 0) return;
  const double beta = sqrt(fmax(*w2, 0.0));
  G.sc[1] = beta;
  G.g[0] = beta;
  for (int j = 1; j <= G.m; ++j) G.g[j] = 0.0;
  G.hd[0] = 0;
  G.hd[3] = 0;
}

// dst[i] = src[i] / s (s = sc[idx], or sqrt(sc[idx]) when root); dst = src where s == 0.
template <class T>
__global__ void k_gm_scale(T* __restrict__ dst, const T* __restrict__ src, int64_t N, const double* __restrict__ sc,
                           int idx, int root) {
  const double v = root ? sqrt(fmax(sc[idx], 0.0)) : sc[idx];
  const double inv = v > 0.0 ? 1.0 / v : 1.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (T)((double)src[i] * inv);
}

// dst = V[:, k] (the product's input, a fixed buffer of the captured graph).
template <class T>
__global__ void k_gm_take(const T* __restrict__ V, int64_t ld, GmState G, T* __restrict__ dst, int64_t N) {
  const T* src = V + (int64_t)G.hd[0] * ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// V[:, k + 1] = w / ||w|| (w itself when its norm is zero).
template <class T>
__global__ void k_gm_store(T* __restrict__ V, int64_t ld, GmState G, const T* __restrict__ w, int64_t N) {
  T* dst = V + (int64_t)(G.hd[0] + 1) * ld;
  const double hn = sqrt(fmax(G.sc[2], 0.0));
  const double inv = hn > 0.0 ? 1.0 / hn : 1.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (T)((double)w[i] * inv);
}

// Column k of the Hessenberg matrix (h1 + h2, ||w||), the earlier rotations
// applied to it, its own rotation, the rotated right-hand side g, the
// convergence test |g[k+1]| <= tol * beta0; k and the step count advance, and
// the WHILE node continues while the cycle has columns and steps left.
__global__ void k_gm_update(GmState G, cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0) return;
  const int m = G.m, k = G.hd[0];
  double* H = G.H;
  const double hn = sqrt(fmax(G.sc[2], 0.0));
  for (int j = 0; j <= k; ++j) H[(size_t)j * m + k] = G.h1[j] + G.h2[j];
  H[(size_t)(k + 1) * m + k] = hn;
  for (int j = 0; j < k; ++j) {
    const double a = H[(size_t)j * m + k], b = H[(size_t)(j + 1) * m + k];
    H[(size_t)j * m + k] = G.cs[j] * a + G.sn[j] * b;
    H[(size_t)(j + 1) * m + k] = -G.sn[j] * a + G.cs[j] * b;
  }
  const double a = H[(size_t)k * m + k], b = H[(size_t)(k + 1) * m + k];
  const double rr = hypot(a, b);
  G.cs[k] = rr > 0.0 ? a / rr : 1.0;
  G.sn[k] = rr > 0.0 ? b / rr : 0.0;
  H[(size_t)k * m + k] = rr;
  H[(size_t)(k + 1) * m + k] = 0.0;
  G.g[k + 1] = -G.sn[k] * G.g[k];
  G.g[k] = G.cs[k] * G.g[k];
  const int it = G.hd[1] + 1;
  const bool conv = fabs(G.g[k + 1]) <= G.sc[3] * G.sc[0] || hn == 0.0;
  G.hd[0] = k + 1;
  G.hd[1] = it;
  G.hd[3] = conv ? 1 : 0;
  cudaGraphSetConditional(cond, (!conv && k + 1 < m && it < G.hd[2]) ? 1u : 0u);
}

// y = -H(0:k, 0:k)^{-1} g(0:k) by back substitution (negated for k_gm_sub).
__global__ void k_gm_lsq(GmState G) {
  if (threadIdx.x != 0) return;
  const int m = G.m, k = G.hd[0];
  for (int i = k - 1; i >= 0; --i) {
    double s = G.g[i];
    for (int j = i + 1; j < k; ++j) s -= G.H[(size_t)i * m + j] * G.y[j];
    G.y[i] = G.H[(size_t)i * m + i] != 0.0 ? s / G.H[(size_t)i * m + i] : 0.0;
  }
  for (int i = 0; i < k; ++i) G.y[i] = -G.y[i];
}

// Device scratch of one solve.
template <class T>
struct Work {
  DevBuf<T> V;         // Krylov basis, N x (m + 1)
  DevBuf<T> w;         // N
  DevBuf<T> vin;       // N: the product's input inside the graph
  DevBuf<double> part; // kDotBlocks x (m + 1)
  DevBuf<double> c;    // m + 1
  DevBuf<double> gm;   // GMRES state: H, cs, sn, g, y, h1, h2, sc
  DevBuf<int> hd;      // 4
};

template <class T>
GmState gm_state(Work<T>& W, int m) {
  GmState G;
  double* p = W.gm.p;
  G.H = p;
  p += (size_t)(m + 1) * m;
  G.cs = p;
  p += m;
  G.sn = p;
  p += m;
  G.g = p;
  p += m + 1;
  G.y = p;
  p += m;
  G.h1 = p;
  p += m + 1;
  G.h2 = p;
  p += m + 1;
  G.sc = p;
  G.hd = W.hd.p;
  G.m = m;
  return G;
}

template <class T>
size_t gm_doubles(int m) {
  return (size_t)(m + 1) * m + 3 * (size_t)m + 3 * (size_t)(m + 1) + 4;
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

// One GMRES cycle as a CUDA graph: start (v_0 = w / beta), WHILE (Arnoldi
// step + Givens update), triangular solve and d += V y. Built once per solve
// by stream capture (the body on its own stream) and launched once per cycle.
template <class T>
struct CycleGraph {
  cudaGraphExec_t exec = nullptr;
  ~CycleGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

template <class T>
int capture_cycle(hodlrdd_s* A, Work<T>& W, const GmState& G, T* d, int64_t N, cudaStream_t cs, cudaStream_t cb,
                  CycleGraph<T>& out) {
  const int64_t ld = N;
  const int grid = grid_for(N);
  const int m = G.m;
  cudaGraph_t graph = nullptr, body = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = HODLRDD_OK;
  auto ck = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == HODLRDD_OK) rc = cuda_fail(e, what, __FILE__, __LINE__);
    return rc == HODLRDD_OK;
  };
  if (!ck(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed), "gmres capture")) return rc;
  // the cycle starts from the residual w and its squared norm in c[0]
  k_gm_begin<<<1, 32, 0, cs>>>(G, W.c.p);
  k_gm_scale<T><<<grid, 256, 0, cs>>>(W.V.p, W.w.p, N, G.sc, 1, 0);
  cudaStreamCaptureStatus status;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraphNode_t cnode = nullptr;
  cudaGraphConditionalHandle cond;
  bool ok = ck(cudaGetLastError(), "gmres start") &&
            ck(cudaStreamGetCaptureInfo(cs, &status, nullptr, &graph, &deps, nullptr, &ndeps), "capture info") &&
            ck(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault), "conditional handle");
  if (ok) {
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    ok = ck(cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp), "while node") &&
         ck(cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies), "dependencies");
    if (ok) body = cp.conditional.phGraph_out[0];
  }
  if (ok) {
    // the Arnoldi step with classical Gram-Schmidt applied twice
    ok = ck(cudaStreamBeginCaptureToGraph(cb, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed), "body");
    if (ok) {
      k_gm_take<T><<<grid, 256, 0, cb>>>(W.V.p, ld, G, W.vin.p, N);
      int r2 = launch_matvec(A, W.vin.p, W.w.p, 1, cb);
      if (r2 != HODLRDD_OK && rc == HODLRDD_OK) rc = r2;
      for (int pass = 0; pass < 2; ++pass) {
        double* h = pass == 0 ? G.h1 : G.h2;
        k_gm_dots<T><<<kDotBlocks, kDotThreads, 0, cb>>>(W.V.p, ld, G, 1, W.w.p, N, W.part.p);
        k_gm_dots_sum<<<(m + 1 + 127) / 128, 128, 0, cb>>>(W.part.p, G, 1, h);
        k_gm_sub<T><<<grid, 256, 0, cb>>>(W.V.p, ld, G, 1, h, W.w.p, N);
      }
      k_dots<T><<<kDotBlocks, kDotThreads, 0, cb>>>(W.w.p, N, 1, W.w.p, N, W.part.p);
      k_dots_sum<<<1, 128, 0, cb>>>(W.part.p, 1, G.sc + 2);
      k_gm_store<T><<<grid, 256, 0, cb>>>(W.V.p, ld, G, W.w.p, N);
      k_gm_update<<<1, 32, 0, cb>>>(G, cond);
      ck(cudaGetLastError(), "gmres step");
      cudaGraph_t b2 = body;
      ck(cudaStreamEndCapture(cb, &b2), "body capture");
      ok = rc == HODLRDD_OK;
    }
  }
  if (ok) {
    k_gm_lsq<<<1, 32, 0, cs>>>(G);
    k_gm_sub<T><<<grid, 256, 0, cs>>>(W.V.p, ld, G, 0, G.y, d, N);
    ck(cudaGetLastError(), "gmres update");
  }
  cudaGraph_t g2 = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &g2);
  if (rc == HODLRDD_OK) ck(e, "gmres capture end");
  if (rc == HODLRDD_OK) ck(cudaGraphInstantiate(&exec, g2, 0), "gmres instantiate");
  if (g2) cudaGraphDestroy(g2);
  if (rc != HODLRDD_OK) {
    cudaGetLastError();
    return rc;
  }
  out.exec = exec;
  return HODLRDD_OK;
}

// Inner GMRES(m) on the fast operator: d ~ A^{-1} r in precision T (FP32 for
// 16-bit and FP32 handles, FP64 for FP64 handles), to a relative residual
// reduction of tol_in or max_it steps (it counts steps over the whole solve's
// calls). d is overwritten. Two host reads per restart cycle.
template <class T>
int gmres(hodlrdd_s* A, const T* r, T* d, int64_t N, int m, double tol_in, int max_it, Work<T>& W,
          const GmState& G, CycleGraph<T>& cyc, int* iters, cudaStream_t st) {
  const int grid = grid_for(N);
  HD_CUDA(cudaMemsetAsync(d, 0, N * sizeof(T), st));
  double beta0 = 0.0;
  HD_TRY(norm2<T>(r, N, W.part, W.c, &beta0, st));  // leaves ||r||^2 in c[0]
  if (beta0 == 0.0) return HODLRDD_OK;
  // residual of the current d: starts as r
  HD_CUDA(cudaMemcpyAsync(W.w.p, r, N * sizeof(T), cudaMemcpyDeviceToDevice, st));
  const double sc[4] = {beta0, beta0, 0.0, tol_in};
  const int hd[4] = {0, 0, max_it, 0};
  HD_CUDA(cudaMemcpyAsync(G.sc, sc, sizeof sc, cudaMemcpyHostToDevice, st));
  HD_CUDA(cudaMemcpyAsync(G.hd, hd, sizeof hd, cudaMemcpyHostToDevice, st));
  int it = 0;
  while (it < max_it) {
    HD_CUDA(cudaGraphLaunch(cyc.exec, st));
    int h[4];
    HD_CUDA(cudaMemcpyAsync(h, G.hd, sizeof h, cudaMemcpyDeviceToHost, st));
    HD_CUDA(cudaStreamSynchronize(st));
    it = h[1];
    if (h[3] || it >= max_it) break;
    // restart from the true residual of the fast operator: w = r - A d
    HD_TRY(launch_matvec(A, d, W.w.p, 1, st));
    k_axpby<T, T, T><<<grid, 256, 0, st>>>(N, 1.0, r, -1.0, W.w.p, W.w.p);
    double beta = 0.0;
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
  cudaStream_t cs = nullptr, cb = nullptr;  // capture streams of the cycle graph and its body
  ~SolveScratch() {
    if (cs) cudaStreamDestroy(cs);
    if (cb) cudaStreamDestroy(cb);
  }
  int fit(int64_t n, int mm) {
    if (!cs) HD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    if (!cb) HD_CUDA(cudaStreamCreateWithFlags(&cb, cudaStreamNonBlocking));
    if (n <= N && mm == m) return HODLRDD_OK;
    // the sizes are recorded only once every buffer is in place, so that a
    // failed allocation leaves the scratch marked empty
    const int64_t nN = std::max(N, n);
    N = 0;
    m = 0;
    HD_TRY(alloc_buffers(nN, mm));
    N = nN;
    m = mm;
    return HODLRDD_OK;
  }
  int alloc_buffers(int64_t N, int m) {
    HD_TRY(W.V.alloc((size_t)N * (m + 1)));
    HD_TRY(W.w.alloc(N));
    HD_TRY(W.vin.alloc(N));
    HD_TRY(W.part.alloc((size_t)kDotBlocks * (m + 1)));
    HD_TRY(W.c.alloc(m + 1));
    HD_TRY(W.gm.alloc(gm_doubles<T>(m)));
    HD_TRY(W.hd.alloc(4));
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
  const GmState G = gm_state(W, m);
  // the cycle graph, captured on the solve's own streams after the caller's work
  CycleGraph<T> cyc;
  {
    cudaEvent_t ev = nullptr;
    HD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S.cs, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_fail(e, "hodlrdd_solve", __FILE__, __LINE__);
    // the products inside the graph record no stage events
    const bool prof = inner->profiling;
    inner->profiling = false;
    const int rc = capture_cycle<T>(inner, W, G, S.d_in.p, N, S.cs, S.cb, cyc);
    inner->profiling = prof;
    HD_TRY(rc);
  }
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
    HD_TRY(gmres<T>(inner, r_in.p, d_in.p, N, m, o.inner_tol, o.max_inner_iters, W, G, cyc, &iters, st));
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
