// Near field of the FP64 form in float-float arithmetic on the FP32 pipes
// (option fp64_near = 1): the same tasks as the FP32 packed tiles (Algorithm 2,
// leaf loop, and the dense IL blocks), evaluated with about 48-bit arithmetic
// at the FP32 instruction rate instead of GB300's FP64 rate (1/64 of FP32).
//
// Coordinates are in units of the level's box size: each point keeps its
// position inside its box as q + r, q on the grid 2^-21 (exact in FP32 for
// every offset the tasks use) and r = u - q as an FP32 remainder (|r| <= 2^-22,
// error 2^-46). A source in box J is moved into target box I's frame by the
// integer offset c_J - c_I, exactly. Per dimension the grid difference is then
// exact and the remainder difference carries 2^-46, so a squared distance R
// in box units is a float-float to about 2^-45 relative. The kernel value at
// s = h^2 R folds the box size h into a per-launch constant (see ff_launch_consts).
// Products with x_j (a float-float from the FP64 x) accumulate in float-float
// over one staged chunk (at most kTileCap sources per thread); chunk sums and
// the stripes' partial sums are added in FP64.
#include <algorithm>
#include <cmath>

#include "ffmath.cuh"
#include "internal.cuh"

namespace hd {
namespace {

constexpr int kFfThreads = 256;
constexpr size_t kFfSmem = (size_t)kTileCap * (2 * sizeof(float4) + sizeof(float2));
constexpr double kFfGrid = 2097152.0;  // 2^21

// Box-unit coordinates at level l: u = (p - corner) / h in [0, 1), split as
// q = round(u 2^21) 2^-21 and r = u - q.
__global__ void k_relq(const double* __restrict__ p64, int64_t N, int d, int l, const int32_t* __restrict__ bstart,
                       const uint64_t* __restrict__ bkey, int64_t nb, const double* __restrict__ lo, double h,
                       float4* __restrict__ Q, float4* __restrict__ R) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = 0, b = nb;  // last box with bstart <= i
    while (b - a > 1) {
      const int64_t mid = (a + b) >> 1;
      if (bstart[mid] <= i) a = mid; else b = mid;
    }
    const uint64_t key = bkey[a];
    float qv[4] = {0.f, 0.f, 0.f, 0.f}, rv[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < d && k < 4; ++k) {
      int64_t c = 0;
      for (int bit = 0; bit < l; ++bit) c |= (int64_t)((key >> (d * bit + k)) & 1u) << bit;
      const double u = (p64[(int64_t)k * N + i] - (lo[k] + (double)c * h)) / h;
      const double q = rint(u * kFfGrid) / kFfGrid;
      qv[k] = (float)q;  // exact: at most 22 significant bits
      rv[k] = __double2float_rn(u - q);
    }
    Q[i] = make_float4(qv[0], qv[1], qv[2], qv[3]);
    R[i] = make_float4(rv[0], rv[1], rv[2], rv[3]);
  }
}

__device__ __forceinline__ float comp(const float4& v, int k) {
  return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

// Squared distance in box units as a float-float. Grid differences are exact
// and at least 2^-21 when nonzero, remainders at most 2^-22 each, so Fast2Sum
// normalises each difference.
template <int D>
__device__ __forceinline__ ff ff_sqdist(const float4& tq, const float4& tr, const float4& sq, const float4& sr) {
  float hi = 0.f, lo = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float dq = __fsub_rn(comp(tq, k), comp(sq, k));
    const float dr = __fsub_rn(comp(tr, k), comp(sr, k));
    const ff u = ff_fast(dq, dr);
    const ff p = ff_prod(u.h, u.h);
    const float cross = __fmaf_rn(__fmul_rn(2.0f, u.h), u.l, p.l);
    if (k == 0) {
      hi = p.h;
      lo = cross;
    } else {
      const ff s = ff_two_sum(hi, p.h);
      hi = s.h;
      lo = __fadd_rn(lo, __fadd_rn(s.l, cross));
    }
  }
  return ff_fast(hi, lo);
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }

// g(R) with the kernel value F = m g(R) (the launch multiplies by m); beta is
// the per-level constant (see ff_launch_consts).
template <int KID>
__device__ __forceinline__ ff ffk(ff R, ff beta, const FfExp& E) {
  if constexpr (KID == HODLRDD_K_LOG) {
    if (R.h == 0.0f) return {0.f, 0.f};
    const ff g = ff_log(R, E);
    return ff_add({__fmul_rn(g.h, 0.5f), __fmul_rn(g.l, 0.5f)}, beta);  // log(r) = log(R)/2 + log(h)
  } else if constexpr (KID == HODLRDD_K_INV_R) {
    if (R.h == 0.0f) return {0.f, 0.f};
    return ff_rsqrt(R);
  } else if constexpr (KID == HODLRDD_K_INV_R2_4D) {
    if (R.h == 0.0f) return {0.f, 0.f};
    return ff_recip(R);
  } else if constexpr (KID == HODLRDD_K_R) {
    return ff_sqrt(R);
  } else if constexpr (KID == HODLRDD_K_GAUSS) {
    return ff_exp(ff_neg(ff_mul(beta, R)), E);
  } else if constexpr (KID == HODLRDD_K_EXP) {
    return ff_exp(ff_neg(ff_mul(beta, ff_sqrt(R))), E);
  } else if constexpr (KID == HODLRDD_K_MATERN32) {
    const ff a = ff_mul(beta, ff_sqrt(R));
    return ff_mul(ff_addf(a, 1.0f), ff_exp(ff_neg(a), E));
  } else {  // HODLRDD_K_INV_SQRT1P
    return ff_rsqrt(ff_addf(ff_mul(beta, ff_sqrt(R)), 1.0f));
  }
}

// One CTA per task, the same tasks and source chunks as the FP32 tiles; each
// thread holds two target rows and sweeps the staged chunk in stripes.
// ynear[i] += m * sum_j g(R_ij) x_j + kdiag * x_i (FP64).
template <int D, int KID>
__global__ void __launch_bounds__(kFfThreads, 2) k_tile_ff(const int4* __restrict__ tasks, int64_t t0, int64_t t1,
                                                          const int4* __restrict__ srcs,
                                                          const float4* __restrict__ soff,
                                                          const float4* __restrict__ Q, const float4* __restrict__ Rm,
                                                          const double* __restrict__ xt, float inv_h, ff beta,
                                                          FfExpConst K, double m, double kdiag,
                                                          double* __restrict__ ynear) {
  extern __shared__ float4 ff_dyn[];
  float4* sq = ff_dyn;
  float4* sr = ff_dyn + kTileCap;
  float2* sx = reinterpret_cast<float2*>(ff_dyn + 2 * kTileCap);
  __shared__ ff tab[64];
  __shared__ double red[kFfThreads], red2[kFfThreads];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < 64) tab[tid] = K.t[tid];
  __syncthreads();
  const FfExp E{K.c0, K.c1, K.c2, K.inv, tab};
  for (int64_t it = t0 + blockIdx.x; it < t1; it += gridDim.x) {
    const int4 T = tasks[it];
    // two rows per thread, G = ceil(m / 2) row pairs and S = kFfThreads / G
    // source stripes; the kFfThreads - S G threads left over sweep nothing
    const int G = max(1, (T.y + 1) / 2);
    const int S = kFfThreads / G;
    const int gi = tid % G, stripe = tid / G;
    const bool va = gi < T.y, vb = gi + G < T.y;
    const int ra = T.x + gi, rb = T.x + gi + G;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 tqa = va ? Q[ra] : z4, tra = va ? Rm[ra] : z4;
    const float4 tqb = vb ? Q[rb] : z4, trb = vb ? Rm[rb] : z4;
    double sum_a = 0.0, sum_b = 0.0;  // chunk sums, added in FP64
    for (int e = T.z; e < T.w;) {
      const int e1 = srcs[e].w;
      __syncthreads();  // the previous chunk has been consumed
      for (int b = e + warp; b < e1; b += kFfThreads / 32) {
        const int4 sj = srcs[b];
        const float4 of = soff[b];
        // the box offset in box units (an integer: the stored offset is (c_J - c_I) h)
        const float ox = rintf(of.x * inv_h), oy = rintf(of.y * inv_h), oz = rintf(of.z * inv_h),
                    ow = rintf(of.w * inv_h);
        for (int k = lane; k < sj.y; k += 32) {
          const float4 q = Q[sj.x + k];
          sq[sj.z + k] = make_float4(q.x + ox, q.y + oy, q.z + oz, q.w + ow);  // exact
          sr[sj.z + k] = Rm[sj.x + k];
          const ff xv = ff_from_double(xt[sj.x + k]);
          sx[sj.z + k] = make_float2(xv.h, xv.l);
        }
      }
      const int4 lastb = srcs[e1 - 1];
      const int n = lastb.z + lastb.y;
      __syncthreads();
      ff acc_a = {0.f, 0.f}, acc_b = {0.f, 0.f};
      for (int f = stripe < S ? stripe : n; f < n; f += S) {
        const float4 q = sq[f], r = sr[f];
        const float2 x2 = sx[f];
        const ff xv = {x2.x, x2.y};
        if (va) acc_a = ff_add(acc_a, ff_mul(ffk<KID>(ff_sqdist<D>(tqa, tra, q, r), beta, E), xv));
        if (vb) acc_b = ff_add(acc_b, ff_mul(ffk<KID>(ff_sqdist<D>(tqb, trb, q, r), beta, E), xv));
      }
      sum_a += (double)acc_a.h + (double)acc_a.l;
      sum_b += (double)acc_b.h + (double)acc_b.l;
      e = e1;
    }
    red[tid] = sum_a;
    red2[tid] = sum_b;
    __syncthreads();
    if (stripe == 0) {
      double sa = 0.0, sb = 0.0;
      for (int s = 0; s < S; ++s) {
        sa += red[s * G + gi];
        sb += red2[s * G + gi];
      }
      if (va) ynear[ra] += m * sa + kdiag * xt[ra];
      if (vb) ynear[rb] += m * sb + kdiag * xt[rb];
    }
    __syncthreads();  // red and the staging arrays are reused by the next task
  }
}

// y[perm[i] * ldy + c0] = near(i) + sum over the level slices of y_l(i).
__global__ void k_finish_ff(const double* __restrict__ ynear, const double* __restrict__ ylev, int slices, int64_t N,
                            const int32_t* __restrict__ perm, double* __restrict__ y, int ldy, int c0) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = ynear[i];
    for (int l = 0; l < slices; ++l) acc += ylev[(int64_t)l * N + i];
    y[(int64_t)perm[i] * ldy + c0] = acc;
  }
}

// The exp constants from the mathematics, in extended precision on the host:
// ln2 / 64 = c0 + c1 + c2 with c0 rounded to 11 significant bits, and
// 2^(j/64) split into FP32 pairs.
const FfExpConst& ff_exp_const() {
  static const FfExpConst K = [] {
    FfExpConst k{};
    const long double ln2 = std::log(2.0L);
    const long double L = ln2 / 64.0L;
    int e = 0;
    std::frexp(L, &e);
    const long double quantum = std::ldexp(1.0L, e - 11);
    const long double c0 = std::round(L / quantum) * quantum;
    const long double r1 = L - c0;
    k.c0 = (float)c0;
    k.c1 = (float)r1;
    k.c2 = (float)(r1 - (long double)k.c1);
    k.inv = (float)(64.0L / ln2);
    for (int j = 0; j < 64; ++j) {
      const long double v = std::exp2((long double)j / 64.0L);
      k.t[j].h = (float)v;
      k.t[j].l = (float)(v - (long double)k.t[j].h);
    }
    return k;
  }();
  return K;
}

// beta and m of F(s) = m g(R), s = h^2 R, for box size h (FP64, then split).
void ff_launch_consts(const KernelSpec& K, double h, double* beta, double* m) {
  const double c = kernel_const(K);
  *beta = 0.0;
  *m = 1.0;
  switch (K.id) {
    case HODLRDD_K_LOG: *beta = std::log(h); break;
    case HODLRDD_K_INV_R: *m = 1.0 / h; break;
    case HODLRDD_K_INV_R2_4D: *m = c / (h * h); break;
    case HODLRDD_K_R: *m = h; break;
    case HODLRDD_K_GAUSS: *beta = c * h * h; break;
    case HODLRDD_K_EXP:
    case HODLRDD_K_MATERN32: *beta = c * h; break;
    default: *beta = h; break;  // 1 / sqrt(1 + r)
  }
}

ff split_host(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

template <int D, int KID>
int launch_ff_k(hodlrdd_s* h, cudaStream_t st, const double* xt, double* yn) {
  static PerDeviceOnce attr;
  HD_TRY(attr.run([] {
    HD_CUDA(cudaFuncSetAttribute(k_tile_ff<D, KID>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFfSmem));
    return (int)HODLRDD_OK;
  }));
  const Plan& P = h->plan;
  const FfExpConst& EC = ff_exp_const();
  auto run = [&](const DenseLevel& DL, double scale, double diag) -> int {
    const int64_t n = DL.t1 - DL.t0;
    if (n <= 0) return HODLRDD_OK;
    double beta = 0.0, m = 1.0;
    ff_launch_consts(h->K, P.h_box[DL.level], &beta, &m);
    k_tile_ff<D, KID><<<(int)std::min<int64_t>(n, INT32_MAX), kFfThreads, kFfSmem, st>>>(
        P.tasks4.p, DL.t0, DL.t1, P.srcs4.p, P.soff4.p, P.hq4[DL.level].p, P.lq4[DL.level].p, xt,
        (float)(1.0 / P.h_box[DL.level]), split_host(beta), EC, scale * m, diag, yn);
    HD_CUDA(cudaGetLastError());
    h->launches += 1;
    return HODLRDD_OK;
  };
  const double ks = h->K.scale, kd = h->K.diag;
  for (const DenseLevel& DL : P.coarse4) HD_TRY(run(DL, ks, 0.0));
  if (P.excl4.t1 > P.excl4.t0) HD_TRY(run(P.excl4, -ks, 0.0));  // leaf blocks the parent tiles also cover
  HD_TRY(run(P.leaf4, ks, kd));
  return HODLRDD_OK;
}

template <int D>
int launch_ff_d(hodlrdd_s* h, cudaStream_t st, const double* xt, double* yn) {
  switch (h->K.id) {
    case HODLRDD_K_LOG: return launch_ff_k<D, HODLRDD_K_LOG>(h, st, xt, yn);
    case HODLRDD_K_INV_R: return launch_ff_k<D, HODLRDD_K_INV_R>(h, st, xt, yn);
    case HODLRDD_K_MATERN32: return launch_ff_k<D, HODLRDD_K_MATERN32>(h, st, xt, yn);
    case HODLRDD_K_GAUSS: return launch_ff_k<D, HODLRDD_K_GAUSS>(h, st, xt, yn);
    case HODLRDD_K_EXP: return launch_ff_k<D, HODLRDD_K_EXP>(h, st, xt, yn);
    case HODLRDD_K_INV_R2_4D: return launch_ff_k<D, HODLRDD_K_INV_R2_4D>(h, st, xt, yn);
    case HODLRDD_K_R: return launch_ff_k<D, HODLRDD_K_R>(h, st, xt, yn);
    case HODLRDD_K_INV_SQRT1P: return launch_ff_k<D, HODLRDD_K_INV_SQRT1P>(h, st, xt, yn);
    default:
      set_error("float-float near field: kernel not supported");
      return HODLRDD_ERR_UNSUPPORTED;
  }
}

}  // namespace

// The float-float near field of one right-hand side into ynear (zeroed here).
int launch_tiles_ff(hodlrdd_s* h, cudaStream_t st, const double* xt, double* ynear) {
  HD_CUDA(cudaMemsetAsync(ynear, 0, (size_t)h->N * sizeof(double), st));
  switch (h->d) {
    case 1: return launch_ff_d<1>(h, st, xt, ynear);
    case 2: return launch_ff_d<2>(h, st, xt, ynear);
    case 3: return launch_ff_d<3>(h, st, xt, ynear);
    default: return launch_ff_d<4>(h, st, xt, ynear);
  }
}

int launch_finish_ff(hodlrdd_s* h, cudaStream_t st, const double* ynear, const double* ylev, int slices, double* y,
                     int ldy, int c0) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  k_finish_ff<<<(int)std::min<int64_t>((h->N + 255) / 256, (int64_t)sms * 16), 256, 0, st>>>(
      ynear, ylev, slices, h->N, h->perm.p, y, ldy, c0);
  HD_CUDA(cudaGetLastError());
  h->launches += 1;
  return HODLRDD_OK;
}

// Box-unit coordinates of level l for the float-float near field.
int build_ffcoords(hodlrdd_s* h, int l, const double* dlo, cudaStream_t st) {
  Plan& P = h->plan;
  if ((int)P.hq4.size() != h->kappa + 1) {
    P.hq4.clear();
    P.lq4.clear();
    P.hq4.resize(h->kappa + 1);
    P.lq4.resize(h->kappa + 1);
  }
  HD_TRY(P.hq4[l].alloc(h->N));
  HD_TRY(P.lq4[l].alloc(h->N));
  const Level& L = h->lv[l];
  k_relq<<<(int)std::min<int64_t>((h->N + 255) / 256, 152 * 16), 256, 0, st>>>(
      h->pts64.p, h->N, h->d, l, L.bstart.p, L.bkey.p, L.nb, dlo, P.h_box[l], P.hq4[l].p, P.lq4[l].p);
  HD_CUDA(cudaGetLastError());
  return HODLRDD_OK;
}

namespace {

// Test entry: F(s) = m g(s / h^2) in float-float for n values of s.
template <int KID>
__global__ void k_ff_eval(int64_t n, const double* __restrict__ s, double h2, ff beta, FfExpConst K, double m,
                          double* __restrict__ out) {
  __shared__ ff tab[64];
  if (threadIdx.x < 64) tab[threadIdx.x] = K.t[threadIdx.x];
  __syncthreads();
  const FfExp E{K.c0, K.c1, K.c2, K.inv, tab};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const ff R = ff_from_double(s[i] / h2);
    const ff g = ffk<KID>(R, beta, E);
    out[i] = m * ((double)g.h + (double)g.l);
  }
}

}  // namespace
}  // namespace hd

using namespace hd;

extern "C" int hodlrdd_debug_ff_eval(int kernel_id, const double* params, double h, const double* s, double* out,
                                     int64_t n) {
  if (!params || !s || !out || n < 0 || !(h > 0.0)) {
    set_error("hodlrdd_debug_ff_eval: NULL pointer, n < 0 or h <= 0");
    return HODLRDD_ERR_INVALID;
  }
  if (kernel_id == HODLRDD_K_SIN || kernel_id < 0 || kernel_id > HODLRDD_K_INV_SQRT1P) {
    set_error("hodlrdd_debug_ff_eval: kernel not supported by the float-float evaluation");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  if (n == 0) return HODLRDD_OK;
  KernelSpec K{};
  K.id = kernel_id;
  K.scale = params[0];
  K.diag = params[1];
  K.p0 = params[2];
  K.p1 = params[3];
  double beta = 0.0, m = 1.0;
  ff_launch_consts(K, h, &beta, &m);
  DevBuf<double> ds, dout;
  HD_TRY(ds.alloc(n));
  HD_TRY(dout.alloc(n));
  HD_CUDA(cudaMemcpy(ds.p, s, n * sizeof(double), cudaMemcpyHostToDevice));
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
  const FfExpConst& EC = ff_exp_const();
  const ff b = split_host(beta);
  switch (kernel_id) {
    case HODLRDD_K_LOG: k_ff_eval<HODLRDD_K_LOG><<<grid, 256>>>(n, ds.p, h * h, b, EC, m, dout.p); break;
    case HODLRDD_K_INV_R: k_ff_eval<HODLRDD_K_INV_R><<<grid, 256>>>(n, ds.p, h * h, b, EC, m, dout.p); break;
    case HODLRDD_K_MATERN32: k_ff_eval<HODLRDD_K_MATERN32><<<grid, 256>>>(n, ds.p, h * h, b, EC, m, dout.p); break;
    case HODLRDD_K_GAUSS: k_ff_eval<HODLRDD_K_GAUSS><<<grid, 256>>>(n, ds.p, h * h, b, EC, m, dout.p); break;
    case HODLRDD_K_EXP: k_ff_eval<HODLRDD_K_EXP><<<grid, 256>>>(n, ds.p, h * h, b, EC, m, dout.p); break;
    case HODLRDD_K_INV_R2_4D: k_ff_eval<HODLRDD_K_INV_R2_4D><<<grid, 256>>>(n, ds.p, h * h, b, EC, m, dout.p); break;
    case HODLRDD_K_R: k_ff_eval<HODLRDD_K_R><<<grid, 256>>>(n, ds.p, h * h, b, EC, m, dout.p); break;
    default: k_ff_eval<HODLRDD_K_INV_SQRT1P><<<grid, 256>>>(n, ds.p, h * h, b, EC, m, dout.p); break;
  }
  HD_CUDA(cudaGetLastError());
  HD_CUDA(cudaMemcpy(out, dout.p, n * sizeof(double), cudaMemcpyDeviceToHost));
  return HODLRDD_OK;
}
